"""Combining the results of the shards of one search (the single exchange step of each row).

* Closest pair / motif (``tsmm_motif_shard``, ``cpp_closest_pair_shard``): every shard returns the
  exact best pair of its tiles; the answer is the lexicographically smallest (dist2, i, j)
  (``reduce_results``; ``allreduce_result`` across the ranks of a torch.distributed group).
* Two-locus (``twolocus_scan_shard``): the answer is the shard result with the largest score, then
  the smallest (i, j) (``reduce_twolocus`` / ``allreduce_twolocus``).
* FRNN on the grid (``frnn_query_shard``): each shard answers the points of its x-slab (slabs of
  equal point counts); the CSR of the whole query takes each point's row from its own shard
  (``merge_frnn`` on the host, ``merge_frnn_tensors`` on a device; ``allgather_frnn`` exchanges the
  pieces with tensor collectives and merges on the pieces' device).
* Two-locus on the tensor cores (``twolocus_scan_tc_shard``): as two-locus, with Pearson's results
  ranked by ``score_real`` (``reduce_twolocus``).
* Strings (``hamming_pair_shard``): the fewest (closest) or most (least correlated) mismatches, then
  the smallest (i, j) (``reduce_hamming`` / ``allreduce_hamming``).
* Light-bulb search (``mlba_pair`` on a subset of the iterations, i.e. of the rows of ``cols``): the
  same ranking as strings; the candidate counts add up (``reduce_mlba`` / ``allreduce_mlba``).

Shards with no pair report i = j = -1.
"""
from __future__ import annotations

import math

import numpy as np


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


def _tl_key(r: dict):
    if r["i"] < 0:
        return (1, 0, 0, 0)  # after every real pair
    if int(r["score"]) < 0:  # Pearson: the score is score_real
        return (0, -float(r["score_real"]), int(r["i"]), int(r["j"]))
    return (0, -int(r["score"]), int(r["i"]), int(r["j"]))


def reduce_twolocus(results: list) -> dict:
    """The two-locus shard result with the largest score, ties to the smallest (i, j)."""
    best = None
    for r in results:
        if best is None or _tl_key(r) < _tl_key(best):
            best = r
    if best is None:
        return {"i": -1, "j": -1, "score": -1, "countsA": np.zeros(9, np.int32), "countsB": np.zeros(9, np.int32)}
    return dict(best)


def allreduce_twolocus(result: dict, group=None) -> dict:
    """Exchange step of a sharded two-locus scan: gather every rank's result and max-reduce."""
    import torch.distributed as dist
    gathered = [None] * dist.get_world_size(group)
    local = {"i": int(result["i"]), "j": int(result["j"]), "score": int(result["score"]),
             "score_real": float(result.get("score_real", -1.0)),
             "countsA": np.asarray(result["countsA"]).tolist(), "countsB": np.asarray(result["countsB"]).tolist()}
    dist.all_gather_object(gathered, local, group=group)
    out = reduce_twolocus(gathered)
    out["countsA"] = np.asarray(out["countsA"], dtype=np.int32)
    out["countsB"] = np.asarray(out["countsB"], dtype=np.int32)
    return out


def _ham_key(r: dict, least: bool):
    if r["i"] < 0:
        return (1, 0, 0, 0)
    m = int(r["mismatches"])
    return (0, -m if least else m, int(r["i"]), int(r["j"]))


def reduce_hamming(results: list, least: bool = False) -> dict:
    """The string-pair shard result with the fewest (least=False) or most (least=True) mismatches,
    ties to the smallest (i, j); i = j = -1 when no shard has a pair."""
    best = None
    for r in results:
        if best is None or _ham_key(r, least) < _ham_key(best, least):
            best = r
    return dict(best) if best is not None else {"i": -1, "j": -1, "mismatches": -1}


def reduce_mlba(results: list, least: bool = False) -> dict:
    """Light-bulb searches over disjoint sets of iterations: the best candidate as in
    :func:`reduce_hamming`; the candidate counts add up."""
    out = reduce_hamming(results, least)
    out["candidates"] = sum(int(r.get("candidates", 0)) for r in results)
    return out


def _allgather(obj, group=None):
    import torch.distributed as dist
    gathered = [None] * dist.get_world_size(group)
    dist.all_gather_object(gathered, obj, group=group)
    return gathered


def allreduce_hamming(result: dict, least: bool = False, group=None) -> dict:
    """Exchange step of a sharded string-pair search across the ranks of a process group."""
    local = {k: int(result[k]) for k in ("i", "j", "mismatches")}
    return reduce_hamming(_allgather(local, group), least)


def allreduce_mlba(result: dict, least: bool = False, group=None) -> dict:
    """Exchange step of a light-bulb search whose iterations are split across the ranks."""
    local = {k: int(result[k]) for k in ("i", "j", "mismatches", "candidates")}
    return reduce_mlba(_allgather(local, group), least)


def merge_frnn(parts: list):
    """CSR of the whole query from the shards' (row_ptr, cols) pieces (numpy); each point's row is
    non-empty in at most one piece (its own slab's)."""
    if not parts:
        raise ValueError("no shard pieces")
    n = len(parts[0][0]) - 1
    deg = np.zeros(n, dtype=np.int64)
    for rp, _ in parts:
        deg += np.diff(np.asarray(rp, dtype=np.int64))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    cols = np.empty(int(row_ptr[-1]), dtype=np.int32)
    for rp, c in parts:
        rp = np.asarray(rp, dtype=np.int64)
        c = np.asarray(c, dtype=np.int32)
        m = int(rp[-1])
        if m == 0:
            continue
        r = np.repeat(np.arange(n), np.diff(rp))            # the row of every entry of this piece
        cols[row_ptr[r] + (np.arange(m) - rp[r])] = c[:m]
    return row_ptr, cols


def merge_frnn_tensors(rp_parts: list, col_parts: list):
    """merge_frnn on torch tensors (on any one device): each piece's entries are placed at their rows'
    offsets in the merged CSR by index arithmetic, without leaving the device."""
    import torch
    n = rp_parts[0].numel() - 1
    dev = rp_parts[0].device
    deg = torch.zeros(n, dtype=torch.int64, device=dev)
    degs = []
    for rp in rp_parts:
        dk = rp[1:].to(torch.int64) - rp[:-1].to(torch.int64)
        degs.append(dk)
        deg += dk
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(deg, 0, out=row_ptr[1:])
    cols = torch.empty(int(row_ptr[-1].item()), dtype=torch.int32, device=dev)
    rows = torch.arange(n, device=dev)
    for rp, dk, c in zip(rp_parts, degs, col_parts):
        m = int(rp[-1].item())
        if m == 0:
            continue
        r = torch.repeat_interleave(rows, dk)                  # the row of every entry of this piece
        cols[row_ptr[r] + (torch.arange(m, device=dev) - rp[r].to(torch.int64))] = c[:m].to(torch.int32)
    return row_ptr, cols


def allgather_frnn(row_ptr, cols, group=None):
    """Exchange step of a sharded FRNN query: every rank receives every slab's piece and merges.

    Tensor collectives only (NCCL for device tensors, gloo for host ones): the pieces' row degrees
    (n int32 each) and their columns, padded to the longest piece, are all-gathered, and the merge is
    index arithmetic on the same device.  numpy inputs give numpy outputs (through host tensors)."""
    import torch
    import torch.distributed as dist
    as_numpy = isinstance(row_ptr, np.ndarray)
    rp = torch.as_tensor(np.asarray(row_ptr) if as_numpy else row_ptr).to(torch.int64)
    cl = torch.as_tensor(np.asarray(cols, dtype=np.int32) if as_numpy else cols).to(torch.int32)
    world = dist.get_world_size(group)
    n = rp.numel() - 1
    m = int(rp[-1].item())
    deg = (rp[1:] - rp[:-1]).to(torch.int32)
    sizes = [torch.zeros(1, dtype=torch.int64, device=rp.device) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([m], dtype=torch.int64, device=rp.device), group=group)
    mmax = max(int(t.item()) for t in sizes)
    degs = [torch.empty(n, dtype=torch.int32, device=rp.device) for _ in range(world)]
    dist.all_gather(degs, deg.contiguous(), group=group)
    padded = torch.zeros(max(mmax, 1), dtype=torch.int32, device=rp.device)
    padded[:m] = cl[:m]
    pieces = [torch.empty(max(mmax, 1), dtype=torch.int32, device=rp.device) for _ in range(world)]
    dist.all_gather(pieces, padded, group=group)
    rps = []
    for dk in degs:
        r = torch.zeros(n + 1, dtype=torch.int64, device=rp.device)
        torch.cumsum(dk.to(torch.int64), 0, out=r[1:])
        rps.append(r)
    out_rp, out_cols = merge_frnn_tensors(rps, pieces)
    if as_numpy:
        return out_rp.cpu().numpy(), out_cols.cpu().numpy()
    return out_rp, out_cols
