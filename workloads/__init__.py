"""Seeded synthetic inputs for the rational-program fit and search.

This module only draws random numbers and lays them out. It holds none of
the method's arithmetic (no normalisation, no least squares, no packing, no
MWP-CWP). Both the CUDA path's tests/bench and the FP64 oracle take their
inputs from here.

Shapes follow the paper's CUDA embodiment (Sec. 4): the data parameter N is a
power of two (Sec. 5 fits on N = 64..512; here 2^6..2^12), the program
parameters are 2-D thread-block formats (B0, B1) with B0*B1 <= 1024 (Sec. 4),
and all low-level metrics of one kernel are measured at the same sample points
(Sec. 3.3, Step 1). The PolyBench/GPU kernels the paper profiles are not
available; these synthetic rational metrics stand in for them.
"""
from __future__ import annotations

import numpy as np

# The 66 thread-block formats (2^a, 2^b) with a + b <= 10, canonical order
# a ascending then b ascending: index = a*11 - a*(a-1)/2 + b.
CONFIGS = np.array([(2 ** a, 2 ** b) for a in range(11) for b in range(11 - a)],
                   dtype=np.int64)
N_CONFIGS = 66
N_METRICS = 8
N_EXPONENTS = (6, 12)          # fit samples: N = 2^6 .. 2^12
LATTICE_CORNER = (4096.0, 1024.0, 1024.0)

# Metric order used by the program table (meanings after Sec. 4.1):
METRIC_NAMES = ("comp_insts", "coal_mem_insts", "uncoal_mem_insts",
                "uncoal_per_mw", "synch_insts", "load_bytes_per_warp",
                "regs_per_thread", "smem_words_per_block")
# Each synthetic metric is offset + scale * g with g a positive rational
# function, so the metric stays rational of the same degree.
_METRIC_AFFINE = ((20.0, 400.0), (2.0, 40.0), (0.0, 12.0), (1.0, 6.0),
                  (0.0, 2.0), (128.0, 1024.0), (16.0, 24.0), (0.0, 1024.0))

# Query record: 8 x float32 = 32 bytes (kernel id stored as int32 bits).
Q_N, Q_NSM, Q_FGHZ, Q_MEMLD, Q_BW, Q_DDC, Q_DDU, Q_KID = range(8)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def exponents(d: int) -> np.ndarray:
    """Graded-lex exponents (e_N, e_B0, e_B1) of total degree <= d.

    Order: total degree ascending; inside one degree, e_N descending, then
    e_B0 descending.  Index 0 is the constant monomial.
    """
    out = []
    for t in range(d + 1):
        for a in range(t, -1, -1):
            for b in range(t - a, -1, -1):
                out.append((a, b, t - a - b))
    return np.array(out, dtype=np.int64)


def n_monomials(d: int) -> int:
    return (d + 1) * (d + 2) * (d + 3) // 6


def lattice() -> np.ndarray:
    """The 7 x 66 = 462 (N, B0, B1) points of the training lattice."""
    ns = [2.0 ** k for k in range(N_EXPONENTS[0], N_EXPONENTS[1] + 1)]
    return np.array([(n, b0, b1) for n in ns for (b0, b1) in CONFIGS],
                    dtype=np.float64)


def _raw_monomials(pts: np.ndarray, e: np.ndarray) -> np.ndarray:
    return np.prod(pts[:, None, :] ** e[None, :, :], axis=2)


class Truth:
    """A ground-truth rational metric g = p/q in the RAW variables."""

    def __init__(self, d, e, cp, cq):
        self.d, self.e, self.cp, self.cq = d, e, np.asarray(cp, float), np.asarray(cq, float)

    def __call__(self, pts):
        m = _raw_monomials(np.asarray(pts, float), self.e)
        return (m @ self.cp) / (m @ self.cq)


def _positive_truth(d, rng, scale_off, density=0.35):
    """Sparse rational with nonnegative coefficients (positive on N,B > 0),
    at least one of p, q of exact total degree d."""
    e = exponents(d)
    corner = np.prod(np.array(LATTICE_CORNER)[None, :] ** e, axis=1)
    deg = e.sum(1)
    while True:
        cp = np.where(rng.random(len(e)) < density, rng.uniform(0.05, 1.0, len(e)), 0.0)
        cq = np.where(rng.random(len(e)) < density, rng.uniform(0.05, 2.0, len(e)), 0.0)
        cp[0] = rng.uniform(0.05, 1.0)
        cq[0] = 1.0
        if (cp[deg == d] != 0).any() or (cq[deg == d] != 0).any():
            break
    cp, cq = cp / corner, cq / corner
    off, sc = scale_off
    # metric = off + sc*p/q = (off*q + sc*p)/q
    return Truth(d, e, off * cq + sc * cp, cq)


def tiny_instance(seed: int = 20190601, n_metrics: int = 4, d: int = 2, m: int = 64):
    """Plain FP64 tiny case: integer coefficients in [-5, 5] in the raw
    variables, deg <= d numerator and denominator, p > 0 and q > 0 on the
    whole 462-point lattice (rejection), m noise-free samples drawn without
    replacement from the lattice."""
    rng = rng_for(seed)
    lat = lattice()
    e = exponents(d)
    mono = _raw_monomials(lat, e)
    truths, xs, ys = [], [], []
    for _ in range(n_metrics):
        while True:
            cp = rng.integers(-5, 6, len(e)).astype(float)
            cq = rng.integers(-5, 6, len(e)).astype(float)
            if np.all(mono @ cq > 0) and np.all(mono @ cp > 0):
                break
        t = Truth(d, e, cp, cq)
        idx = rng.choice(len(lat), size=m, replace=False)
        pts = lat[idx]
        truths.append(t)
        xs.append(pts)
        ys.append(t(pts))
    x = np.concatenate(xs).T.astype(np.float32)
    y64 = np.concatenate(ys)
    off = np.arange(n_metrics + 1, dtype=np.int64) * m
    return dict(x=np.ascontiguousarray(x), y=y64.astype(np.float32), y64=y64, fit_off=off,
                degree=np.full(n_metrics, d, np.int8), truths=truths,
                lattice=lat)


def _kernel_points(rng, m):
    n = 2.0 ** rng.integers(N_EXPONENTS[0], N_EXPONENTS[1] + 1, m)
    c = CONFIGS[rng.integers(0, N_CONFIGS, m)]
    return np.stack([n, c[:, 0].astype(float), c[:, 1].astype(float)], 1)


def batched_instance(n_kernels: int, seed: int, m=512, d=3, noise=0.01,
                     n_metrics=N_METRICS, degree_choices=None, m_range=None):
    """Batched fit input: n_kernels x n_metrics fits.  The metrics of one
    kernel share their sample points.  y = g(x) * exp(noise * xi),
    xi ~ N(0, 1).  With m_range=(lo, hi) each kernel draws its own sample
    count log-uniformly in [lo, hi]; with degree_choices each fit draws its
    own degree."""
    rng = rng_for(seed)
    xs, ys, degs, truths, counts = [], [], [], [], []
    for k in range(n_kernels):
        if m_range is not None:
            mk = int(round(np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1])))))
        else:
            mk = m
        pts = _kernel_points(rng, mk)
        for j in range(n_metrics):
            dj = int(rng.choice(degree_choices)) if degree_choices is not None else d
            t = _positive_truth(dj, rng, _METRIC_AFFINE[j % N_METRICS])
            yj = t(pts) * np.exp(noise * rng.standard_normal(mk))
            xs.append(pts)
            ys.append(yj)
            degs.append(dj)
            truths.append(t)
            counts.append(mk)
    off = np.zeros(len(counts) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    x = np.ascontiguousarray(np.concatenate(xs).T.astype(np.float32))
    y64 = np.concatenate(ys)
    return dict(x=x, y=y64.astype(np.float32), y64=y64, fit_off=off,
                degree=np.array(degs, np.int8), truths=truths,
                metric_map=np.arange(n_kernels * n_metrics, dtype=np.int32).reshape(n_kernels, n_metrics)
                if n_metrics == N_METRICS else None)


def shared_points(inst, n_metrics=N_METRICS):
    """The same batched instance with each kernel's sample points stored once
    (its metrics are measured at the same points): x_points float32 [3][P]
    holding the points of fits 0, n_metrics, 2 n_metrics, .., and
    point_off int64 [K+1] into it; y and fit_off are unchanged."""
    off = inst["fit_off"]
    K = (len(off) - 1) // n_metrics
    starts = off[0:K * n_metrics:n_metrics]
    counts = off[1:K * n_metrics + 1:n_metrics] - starts
    cols = np.concatenate([np.arange(a, a + c) for a, c in zip(starts, counts)]) if K else \
        np.zeros(0, np.int64)
    point_off = np.zeros(K + 1, np.int64)
    point_off[1:] = np.cumsum(counts)
    return np.ascontiguousarray(inst["x"][:, cols]), point_off


def queries(n_queries: int, n_kernels: int, seed: int, n_log2=(10, 26)):
    """Search queries, sorted by kernel id.  N log-uniform over 2^10..2^26
    rounded to an integer; SMs U{80..160}; clock U[1.2, 2.0] GHz; memory
    latency U[400, 800] cycles; bandwidth U[1, 8] TB/s (stored in GB/s);
    departure delay U[1, 20] cycles (coalesced = uncoalesced)."""
    rng = rng_for(seed)
    q = np.empty((n_queries, 8), np.float32)
    q[:, Q_N] = np.round(2.0 ** rng.uniform(n_log2[0], n_log2[1], n_queries))
    q[:, Q_NSM] = rng.integers(80, 161, n_queries)
    q[:, Q_FGHZ] = rng.uniform(1.2, 2.0, n_queries)
    q[:, Q_MEMLD] = rng.uniform(400.0, 800.0, n_queries)
    q[:, Q_BW] = rng.uniform(1000.0, 8000.0, n_queries)
    dd = rng.uniform(1.0, 20.0, n_queries)
    q[:, Q_DDC] = dd
    q[:, Q_DDU] = dd
    kid = np.sort(rng.integers(0, n_kernels, n_queries)).astype(np.int32)
    q[:, Q_KID] = kid.view(np.float32)
    return q


def query_kernel_ids(q: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(q[:, Q_KID]).view(np.int32)


def synthetic_program(n_kernels: int, d: int, seed: int):
    """A random program table in the packed layout, drawn directly (not
    produced by a fit): per (kernel, config, metric) a univariate rational
    in t = aN*N + bN whose numerator and denominator are positive for
    t >= -1 (constant term larger than the sum of the other coefficients).
    Returns dict(aN[K][8], bN[K][8], table[K][66][8][2][d+1], grid_dims[K])."""
    rng = rng_for(seed)
    K = n_kernels
    lo, hi = 64.0, 4096.0
    aN = np.full((K, N_METRICS), 2.0 / (hi - lo), np.float64)
    bN = -1.0 - lo * aN
    tab = np.zeros((K, N_CONFIGS, N_METRICS, 2, d + 1), np.float64)
    hi_c = rng.uniform(0.0, 1.0, (K, N_CONFIGS, N_METRICS, 2, d))
    hi_c *= (rng.random(hi_c.shape) < 0.6)
    hi_c[..., 1:] *= 10.0 ** rng.uniform(-6, -2, hi_c[..., 1:].shape)
    tab[..., 1:] = hi_c
    tab[..., 0] = hi_c.sum(-1) + rng.uniform(0.05, 1.0, hi_c.shape[:-1])
    # Denominator normalised to constant term 1 + ..., numerator scaled to
    # the metric's range.
    for j, (off, sc) in enumerate(_METRIC_AFFINE):
        den = tab[:, :, j, 1, :]
        den /= den[..., :1]
        num = tab[:, :, j, 0, :]
        num *= sc / np.maximum(num[..., :1], 1e-30)
        num += off * den
    # Thread-block dependence: scale uncoalesced transactions per warp
    # access with B0 (column-major style accesses), smem with T.
    b0 = CONFIGS[:, 0].astype(float)
    t_ = (CONFIGS[:, 0] * CONFIGS[:, 1]).astype(float)
    tab[:, :, 3, 0, :] *= np.minimum(b0, 32.0)[None, :, None] / 8.0
    tab[:, :, 7, 0, :] *= (t_ / 256.0)[None, :, None]
    gd = rng.integers(1, 3, K).astype(np.int32)
    return dict(aN=aN.astype(np.float32), bN=bN.astype(np.float32),
                table=tab.astype(np.float32), grid_dims=gd, d=d)


HW_FIXED_DEFAULT = dict(warp_size=32, t_max=1024, b_max=32, w_max=64,
                        r_sm=65536, z_sm=58368, issue_cycles=1.0)
