"""The exchange step of a sharded search, on CPU: two gloo ranks each contribute the best pair of
their part of the pair space (computed by the oracle), and the all-reduce must give the answer of
the whole search.  Also the host-side reduction's edge cases."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1407_5609_gb300 import shards, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a = synth.make_random_walk(900, seed=81)
    l, excl = 40, 20
    n = a.shape[0] - l + 1
    rows = np.arange(rank, n, world)                    # this rank's part: pairs touching its rows
    bj, bd = oracle.tsmm_rows(a, l, excl, rows)
    keys = [(float(d), int(min(r, j)), int(max(r, j))) for r, j, d in zip(rows, bj, bd) if j >= 0]
    d2, i, j = min(keys)
    local = {"i": i, "j": j, "dist2": d2, "dist": math.sqrt(d2), "n_emitted": 1, "n_rechecked": 1}
    res = shards.allreduce_result(local)
    if rank == 0:
        np.save(out_path, np.array([res["i"], res["j"], res["dist2"], res["n_emitted"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_allreduce_two_gloo_ranks(tmp_path):
    out = str(tmp_path / "res.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    i, j, d2, ne = np.load(out)
    a = synth.make_random_walk(900, seed=81)
    oi, oj, od2 = oracle.tsmm(a, 40, 20)
    assert (int(i), int(j)) == (oi, oj) and d2 == od2 and ne == 2


def test_reduce_results_lexicographic_and_empty():
    none = {"i": -1, "j": -1, "dist2": math.inf, "dist": math.inf}
    r = shards.reduce_results([none, {"i": 5, "j": 9, "dist2": 1.0, "dist": 1.0},
                               {"i": 3, "j": 11, "dist2": 1.0, "dist": 1.0}, {"i": 0, "j": 1, "dist2": 2.0, "dist": 1.4}])
    assert (r["i"], r["j"]) == (3, 11)
    assert shards.reduce_results([none, none])["i"] == -1
    assert shards.reduce_results([])["i"] == -1


def _rank_main_twolocus_frnn(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # two-locus: each rank's part = the best pair (by the oracle) among SNP pairs (i, j) with
    # i % world == rank; the max-reduce must give the whole scan's answer
    g, _ = synth.make_genotypes(S=120, m1=90, m2=70, seed=98)
    best = {"i": -1, "j": -1, "score": -1, "countsA": np.zeros(9, np.int32), "countsB": np.zeros(9, np.int32)}
    for i in range(rank, 120, world):
        for j in range(i + 1, 120):
            ua = int(np.sum(g[i, :90] == g[j, :90]))
            ub = int(np.sum(g[i, 90:] == g[j, 90:]))
            sc = abs(ua * 70 - ub * 90)
            if sc > best["score"]:
                best = {"i": i, "j": j, "score": sc, "countsA": np.zeros(9, np.int32), "countsB": np.zeros(9, np.int32)}
    tl = shards.allreduce_twolocus(best)
    # FRNN: each rank's piece = the oracle's rows of the points in its half of x
    x = synth.make_frnn_mixture(n=800, d=3, k=4, sigma=0.05, seed=99).astype(np.float64)
    rp, cols = oracle.frnn(x, 0.03)
    own = (x[:, 0] >= np.median(x[:, 0])).astype(int) == rank
    deg = np.where(own, np.diff(rp), 0)
    prp = np.concatenate([[0], np.cumsum(deg)])
    pcols = np.concatenate([cols[rp[i]:rp[i + 1]] for i in range(800) if own[i]] or [np.zeros(0, np.int32)])
    mrp, mcols = shards.allgather_frnn(prp, pcols)
    import torch
    trp, tcols = shards.allgather_frnn(torch.from_numpy(prp), torch.from_numpy(pcols.astype(np.int32)))
    if rank == 0:
        np.savez(out_path, tl=np.array([tl["i"], tl["j"], tl["score"]]), rp=mrp, cols=mcols, trp=trp.numpy(),
                 tcols=tcols.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_twolocus_and_frnn_exchange_two_gloo_ranks(tmp_path):
    out = str(tmp_path / "res.npz")
    mp.start_processes(_rank_main_twolocus_frnn, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    z = np.load(out)
    g, _ = synth.make_genotypes(S=120, m1=90, m2=70, seed=98)
    oi, oj, osc, _, _ = oracle.twolocus(g, 90, 70)
    assert tuple(int(v) for v in z["tl"]) == (oi, oj, osc)
    x = synth.make_frnn_mixture(n=800, d=3, k=4, sigma=0.05, seed=99).astype(np.float64)
    rp, cols = oracle.frnn(x, 0.03)
    np.testing.assert_array_equal(z["rp"], rp)
    np.testing.assert_array_equal(z["cols"], cols)
    np.testing.assert_array_equal(z["trp"], rp)       # torch tensors in, torch tensors out
    np.testing.assert_array_equal(z["tcols"], cols)


def test_merge_frnn_tensors_matches_numpy_merge():
    """The on-device merge (index arithmetic on tensors) gives the same CSR as the numpy merge,
    including empty pieces and rows answered by no piece."""
    import torch
    x = synth.make_frnn_mixture(n=500, d=3, k=4, sigma=0.05, seed=131).astype(np.float64)
    rp, cols = oracle.frnn(x, 0.04)
    owner = synth.rng_for(132).integers(0, 4, size=500)        # 3 pieces + rows of no piece
    parts = []
    for k in range(3):
        deg = np.where(owner == k, np.diff(rp), 0)
        prp = np.concatenate([[0], np.cumsum(deg)])
        pcols = np.concatenate([cols[rp[i]:rp[i + 1]] for i in range(500) if owner[i] == k] or [np.zeros(0, np.int32)])
        parts.append((prp, pcols.astype(np.int32)))
    parts.append((np.zeros(501, np.int64), np.zeros(0, np.int32)))
    nrp, ncols = shards.merge_frnn(parts)
    trp, tcols = shards.merge_frnn_tensors([torch.from_numpy(p[0]) for p in parts],
                                           [torch.from_numpy(p[1]) for p in parts])
    np.testing.assert_array_equal(trp.numpy(), nrp)
    np.testing.assert_array_equal(tcols.numpy(), ncols)


def test_reduce_twolocus_order():
    none = {"i": -1, "j": -1, "score": -1, "countsA": np.zeros(9), "countsB": np.zeros(9)}
    a = {"i": 4, "j": 9, "score": 50, "countsA": np.zeros(9), "countsB": np.zeros(9)}
    b = {"i": 2, "j": 30, "score": 50, "countsA": np.zeros(9), "countsB": np.zeros(9)}
    c = {"i": 0, "j": 1, "score": 49, "countsA": np.zeros(9), "countsB": np.zeros(9)}
    r = shards.reduce_twolocus([none, a, c, b])
    assert (r["i"], r["j"], r["score"]) == (2, 30, 50)
    assert shards.reduce_twolocus([none])["i"] == -1 and shards.reduce_twolocus([])["i"] == -1


def _rank_main_strings(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = synth.make_strings(700, 20, 4, seed=120, plant=(3, 650), at=(0,))
    # light-bulb search: this rank runs every world-th iteration (the oracle stands in for the GPU)
    cols = synth.sample_columns(6, 5, 20, seed=121)
    i, j, h, c = oracle.mlba(s, 4, cols[rank::world])
    ml = shards.allreduce_mlba({"i": i, "j": j, "mismatches": h, "candidates": c})
    # strings: this rank's part = the pairs (i, j) with i % world == rank, searched by brute force
    best = {"i": -1, "j": -1, "mismatches": -1}
    for a in range(rank, 700, world):
        hd = (s[a + 1:] != s[a]).sum(axis=1)
        if hd.size:
            k = int(np.argmax(hd))
            if best["i"] < 0 or hd[k] > best["mismatches"]:
                best = {"i": a, "j": a + 1 + k, "mismatches": int(hd[k])}
    hm = shards.allreduce_hamming(best, least=True)
    if rank == 0:
        np.save(out_path, np.array([ml["i"], ml["j"], ml["mismatches"], ml["candidates"], hm["i"], hm["j"],
                                    hm["mismatches"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_strings_and_mlba_exchange_two_gloo_ranks(tmp_path):
    out = str(tmp_path / "res.npy")
    mp.start_processes(_rank_main_strings, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    z = [int(v) for v in np.load(out)]
    s = synth.make_strings(700, 20, 4, seed=120, plant=(3, 650), at=(0,))
    cols = synth.sample_columns(6, 5, 20, seed=121)
    assert tuple(z[:4]) == oracle.mlba(s, 4, cols)
    assert tuple(z[4:]) == oracle.hamming(s, 4, least=True)


def test_reduce_hamming_and_mlba_order():
    none = {"i": -1, "j": -1, "mismatches": -1, "candidates": 0}
    a = {"i": 4, "j": 9, "mismatches": 3, "candidates": 10}
    b = {"i": 2, "j": 30, "mismatches": 3, "candidates": 1}
    c = {"i": 0, "j": 1, "mismatches": 5, "candidates": 2}
    assert (shards.reduce_hamming([none, a, c, b])["i"], shards.reduce_hamming([a, b])["j"]) == (2, 30)
    assert shards.reduce_hamming([a, b, c], least=True)["i"] == 0
    r = shards.reduce_mlba([none, a, b, c])
    assert (r["i"], r["j"], r["candidates"]) == (2, 30, 13)
    assert shards.reduce_mlba([none])["i"] == -1 and shards.reduce_hamming([])["i"] == -1
