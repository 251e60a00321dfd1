"""Seeded synthetic workloads for the closest-pair, FRNN, motif and two-locus paths.

This module only draws random inputs and lays them out; it holds none of the
method's arithmetic (no distances, no normalisation, no counting), so both the
CUDA path and the CPU oracle can take their inputs from here.

Every generator uses ``numpy.random.Generator(PCG64(seed))``.  The default seeds
are ``14075609 + k`` where k is the workload's index in the list below:

  0  closest pair: n=4096 points, d=32, FP64 uniform in [0,1]^d, one planted pair
     at Euclidean distance 1e-3                                   (Sec. 3, CPP)
  1  FRNN: n=2^20 FP32 points in d=3 from a 64-component Gaussian mixture
     (centres uniform in [0,1]^3, sigma=0.01), R=0.002           (Sec. 3.5)
  2  motif mining: FP32 random walk (cumsum of N(0,1)) of length 262,144,
     l=512, exclusion |i-j| < 256                                (Sec. 2, 3.6)
  3  two-locus: 4096 SNPs x (4096 cases + 4096 controls), genotypes in {0,1,2}
     under Hardy-Weinberg with minor-allele frequency U[0.05,0.5], one planted
     pair                                                         (Sec. 6, 6.1)
  4  batch: 2048 independent CPP/FRNN instances with n log-uniform in
     [256, 65536] and d in {8,16,32,64,128}                       (Sec. 3, 3.5)

The paper's own data (the insect-behaviour series of Table 3 and the GWAS data
of Sec. 6.1) are not available; these generators stand in for them with the
shapes and distributions listed above.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 14075609


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------- CPP
def make_cpp(n: int = 4096, d: int = 32, seed: int = SEED_BASE + 0,
             plant_dist: float | None = 1e-3, dtype=np.float64):
    """Uniform points in [0,1]^d plus one planted pair.

    The plant copies point ``a`` to point ``b`` and moves it by ``plant_dist``
    along a random unit vector.  Returns ``(pts, (a, b))`` with a < b, or
    ``(pts, None)`` when ``plant_dist`` is None.
    """
    g = rng_for(seed)
    pts = g.random((n, d))
    plant = None
    if plant_dist is not None and n >= 2:
        a, b = sorted(int(v) for v in g.choice(n, size=2, replace=False))
        v = g.standard_normal(d)
        v /= np.linalg.norm(v)
        pts[b] = pts[a] + plant_dist * v
        plant = (a, b)
    return np.ascontiguousarray(pts.astype(dtype)), plant


# -------------------------------------------------------------------------- FRNN
def make_frnn_mixture(n: int = 1 << 20, d: int = 3, k: int = 64, sigma: float = 0.01,
                      seed: int = SEED_BASE + 1, dtype=np.float32):
    """Equal-weight isotropic Gaussian mixture with k centres uniform in [0,1]^d."""
    g = rng_for(seed)
    centres = g.random((k, d))
    comp = np.arange(n) % k
    g.shuffle(comp)
    pts = centres[comp] + sigma * g.standard_normal((n, d))
    return np.ascontiguousarray(pts.astype(dtype))


# ------------------------------------------------------------------------- TSMM
def make_random_walk(N: int = 262144, seed: int = SEED_BASE + 2, dtype=np.float32):
    """Random walk: cumulative sum of i.i.d. N(0,1) steps (Sec. 3.6)."""
    g = rng_for(seed)
    return np.ascontiguousarray(np.cumsum(g.standard_normal(N)).astype(dtype))


def plant_motif(series: np.ndarray, src: int, dst: int, l: int,
                scale: float = 3.0, offset: float = 7.0) -> np.ndarray:
    """Copy the l-mer at ``src`` onto ``dst`` after an affine change.

    An affine change with positive scale leaves the z-normalised l-mer unchanged,
    so (src, dst) becomes a pair at distance ~0.
    """
    out = series.copy()
    out[dst:dst + l] = (scale * series[src:src + l].astype(np.float64) + offset).astype(series.dtype)
    return out


# -------------------------------------------------------------------- two-locus
def make_genotypes(S: int = 4096, m1: int = 4096, m2: int = 4096,
                   seed: int = SEED_BASE + 3, maf_lo: float = 0.05, maf_hi: float = 0.5,
                   plant: bool = True):
    """Genotype matrix int8 [S][m1+m2]: minor-allele counts in {0,1,2}.

    Columns 0..m1-1 are cases, m1..m1+m2-1 controls.  Each SNP has its own
    minor-allele frequency p ~ U[maf_lo, maf_hi] and Hardy-Weinberg genotype
    probabilities ((1-p)^2, 2p(1-p), p^2), the same for cases and controls.
    The planted pair (a, b), following the injection idea of Sec. 6.1: in the
    cases SNP b copies SNP a; in the controls SNP b is an independent draw.
    Returns ``(geno, (a, b) or None)``.
    """
    g = rng_for(seed)
    p = g.uniform(maf_lo, maf_hi, size=S)
    m = m1 + m2
    u = g.random((S, m))
    p0 = (1.0 - p) ** 2
    p1 = p0 + 2.0 * p * (1.0 - p)
    geno = (u >= p0[:, None]).astype(np.int8) + (u >= p1[:, None]).astype(np.int8)
    pair = None
    if plant and S >= 2:
        a, b = sorted(int(v) for v in g.choice(S, size=2, replace=False))
        geno[b, :m1] = geno[a, :m1]
        pair = (a, b)
    return np.ascontiguousarray(geno), pair


def words_per_group(m: int) -> int:
    return (m + 63) // 64


def pack_planes(geno: np.ndarray, m1: int, m2: int, W: int | None = None) -> np.ndarray:
    """Lay genotypes out as the two-locus kernel's input planes.

    Output uint64 [S][2 groups][2 planes][W]: group 0 = cases, 1 = controls;
    plane 0 holds [g == 1], plane 1 holds [g == 2] (the g == 0 plane of the
    one-hot code of Sec. 5.3 is implied).  Bit b of word w is individual 64w+b
    of the group; pad bits are 0.  W defaults to the larger group's word count.
    """
    S = geno.shape[0]
    if W is None:
        W = max(words_per_group(m1), words_per_group(m2))
    out = np.zeros((S, 2, 2, W), dtype=np.uint64)
    shifts = np.arange(64, dtype=np.uint64)
    for grp, (lo, hi) in enumerate(((0, m1), (m1, m1 + m2))):
        sub = geno[:, lo:hi]
        mg = hi - lo
        for pl, val in enumerate((1, 2)):
            bits = np.zeros((S, W * 64), dtype=np.uint64)
            bits[:, :mg] = (sub == val)
            out[:, grp, pl, :] = (bits.reshape(S, W, 64) << shifts[None, None, :]).sum(axis=2, dtype=np.uint64)
    return np.ascontiguousarray(out)


def unpack_planes(planes: np.ndarray, m1: int, m2: int) -> np.ndarray:
    """Inverse of :func:`pack_planes` (used to check the layout)."""
    S, _, _, W = planes.shape
    geno = np.zeros((S, m1 + m2), dtype=np.int8)
    shifts = np.arange(64, dtype=np.uint64)
    for grp, (lo, hi) in enumerate(((0, m1), (m1, m1 + m2))):
        mg = hi - lo
        for pl, val in enumerate((1, 2)):
            w = planes[:, grp, pl, :]
            bits = ((w[:, :, None] >> shifts[None, None, :]) & np.uint64(1)).reshape(S, W * 64)
            geno[:, lo:hi] += (bits[:, :mg].astype(np.int8) * val)
    return geno


# ------------------------------------------------------------------------ batch
@dataclasses.dataclass
class BatchInstance:
    pts: np.ndarray          # float32 [n][d]
    plant: tuple[int, int]   # planted pair (a, b), a < b
    plant_dist: float
    R: float                 # FRNN radius: 2x the planted distance


def make_batch(count: int = 2048, seed: int = SEED_BASE + 4, n_lo: int = 256, n_hi: int = 65536,
               dims=(8, 16, 32, 64, 128), plant_dist: float = 1e-3, mix_k: int = 16,
               mix_sigma: float = 0.05):
    """Uneven batch of CPP/FRNN instances.

    n = floor(exp(U[ln n_lo, ln n_hi])), d uniform over ``dims``; half the
    instances are uniform in [0,1]^d, half a ``mix_k``-component Gaussian
    mixture with sigma ``mix_sigma``; each has a pair planted at ``plant_dist``
    and R = 2 * plant_dist.
    """
    g = rng_for(seed)
    out = []
    for _ in range(count):
        n = int(np.floor(np.exp(g.uniform(np.log(n_lo), np.log(n_hi)))))
        n = max(2, min(n, n_hi))
        d = int(g.choice(dims))
        if g.random() < 0.5:
            pts = g.random((n, d))
        else:
            centres = g.random((mix_k, d))
            pts = centres[g.integers(0, mix_k, size=n)] + mix_sigma * g.standard_normal((n, d))
        a, b = sorted(int(v) for v in g.choice(n, size=2, replace=False))
        v = g.standard_normal(d)
        v /= np.linalg.norm(v)
        pts[b] = pts[a] + plant_dist * v
        out.append(BatchInstance(np.ascontiguousarray(pts.astype(np.float32)), (a, b),
                                 plant_dist, 2.0 * plant_dist))
    return out


def make_strings(n: int = 65536, t: int = 64, sigma: int = 4, seed: int = SEED_BASE + 5,
                 plant: tuple | None = (12345, 54321), at: tuple = (7, 40)) -> np.ndarray:
    """Uniform strings uint8 [n][t] over {0, .., sigma-1} (Sec. 4's strings; four letters is the
    discretisation of its experiment).  With ``plant = (a, b)`` string b copies string a except at
    the positions ``at``, where its symbol is shifted by one: a pair at len(at) mismatches."""
    s = rng_for(seed).integers(0, sigma, (n, t)).astype(np.uint8)
    if plant is not None:
        a, b = plant
        s[b] = s[a]
        idx = list(at)
        s[b, idx] = ((s[b, idx].astype(np.int64) + 1) % sigma).astype(np.uint8)
    return np.ascontiguousarray(s)


def sample_columns(iters: int, L: int, width: int, seed: int) -> np.ndarray:
    """The columns the light-bulb algorithm samples (Sec. 4): int32 [iters][L], each drawn
    uniformly from [0, width) with replacement."""
    if L == 0 or width == 0:
        return np.zeros((iters, L), np.int32)
    return rng_for(seed).integers(0, width, (iters, L)).astype(np.int32)
