"""Combining the results of shards of one closest-pair / motif search.

A search split with ``tsmm_motif_shard`` / ``cpp_closest_pair_shard`` yields one exact result per
shard; the answer of the whole search is the lexicographically smallest (dist2, i, j) among them
(shards with no pair report i = j = -1).  ``reduce_results`` does that on one host;
``allreduce_result`` is the exchange step across the ranks of a torch.distributed group (each rank
contributes its shard's 24-byte key; every rank receives the combined answer).
"""
from __future__ import annotations

import math


def _key(r: dict):
    if r["i"] < 0:
        return (math.inf, math.inf, math.inf)
    return (r["dist2"], r["i"], r["j"])


def reduce_results(results: list) -> dict:
    """The lexicographic (dist2, i, j) minimum of shard results (i = j = -1 when none has a pair)."""
    best = None
    for r in results:
        if best is None or _key(r) < _key(best):
            best = r
    out = dict(best) if best is not None else {"i": -1, "j": -1, "dist2": math.inf, "dist": math.inf}
    out["n_emitted"] = sum(int(r.get("n_emitted", 0)) for r in results)
    out["n_rechecked"] = sum(int(r.get("n_rechecked", 0)) for r in results)
    return out


def allreduce_result(result: dict, group=None) -> dict:
    """Exchange step: gather every rank's shard result and reduce (works with gloo and nccl)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gathered = [None] * world
    dist.all_gather_object(gathered, {k: result[k] for k in ("i", "j", "dist2", "dist", "n_emitted",
                                                              "n_rechecked") if k in result}, group=group)
    return reduce_results(gathered)
