"""Seeded CSR matrix generators for the workloads SpGEMM is measured on.

Every random draw comes from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), evaluated as
``mix(key + (counter + 1) * GAMMA)`` where ``key`` is derived from (seed, stream). A
draw therefore depends only on (seed, stream, counter): the same matrix comes out on
any machine, any numpy version and in any evaluation order.

The workloads follow the evaluation form of the paper (Sec. V: C = A*A on sparse
matrices of a few to ~150 nonzeros per row), with synthetic stand-ins for the
SuiteSparse matrices of Table I:

* ``uniform_random``: per row k_i ~ Binomial(n, d), then k_i distinct uniform columns.
* ``laplacian2d`` / ``laplacian3d``: 5- and 7-point stencils with Dirichlet boundary
  (boundary rows lack the neighbours outside the grid), diagonal 4 or 6, off-diagonal -1.
* ``rmat``: R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with 2^scale vertices and
  edge_factor * 2^scale directed edge samples, no noise, no vertex permutation,
  self-loops kept and duplicates merged before values are drawn (values in CSR order).
* ``batch_job`` / ``serve_stream``: the batched and served job mixes.

Nothing here multiplies, merges or sorts partial products: this module only builds
inputs, so the CUDA path and the CPU oracle can share it.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)
_INV53 = 1.0 / float(1 << 53)

# stream ids (a stream separates independent uses of one seed)
_ST_ROWCOUNT = 1
_ST_COLUMNS = 2
_ST_VALUES = 3
_ST_RMAT_EDGE = 10
_ST_RMAT_VAL = 11
_ST_BATCH_PARAM = 20
_ST_SERVE = 30
_ST_JOB_BASE = 1 << 20


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = (z ^ (z >> _S30)) * _M1
    z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([int(stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    k = _mix(s + GAMMA)
    k = _mix(k ^ np.array([int(seed) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    return k[0]


def counter_u64(seed: int, stream: int, counters) -> np.ndarray:
    """The counter-th 64-bit output of the SplitMix64 sequence keyed by (seed, stream)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed, stream) + (c + np.uint64(1)) * GAMMA)


def counter_uniform(seed: int, stream: int, counters) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (counter_u64(seed, stream, counters) >> _S11).astype(np.float64) * _INV53


@dataclass
class CSR:
    """A CSR matrix on the host: int64 row_ptr, int32 col, float64 or float32 val."""

    rows: int
    cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.rows > 0 else 0

    def astype(self, dtype) -> "CSR":
        return CSR(self.rows, self.cols, self.row_ptr, self.col, self.val.astype(dtype))

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.rows, self.cols), dtype=np.float64)
        r = np.repeat(np.arange(self.rows), self.row_lengths())
        d[r, self.col] = self.val
        return d


def _csr_from_sorted_keys(m: int, n: int, rows: np.ndarray, cols: np.ndarray) -> tuple:
    counts = np.bincount(rows, minlength=m) if m > 0 else np.zeros(0, np.int64)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp, cols.astype(np.int32)


def _binomial_cdf(n: int, d: float) -> tuple:
    """(cdf, kmax): the Binomial(n, d) CDF on 0..kmax (tail beyond mean + 14 sd dropped), for
    0 < d < 1 and n > 0."""
    mean = n * d
    sd = math.sqrt(n * d * (1.0 - d))
    kmax = int(min(n, math.ceil(mean + 14.0 * sd + 30.0)))
    lg_n1 = math.lgamma(n + 1.0)
    ld, l1d = math.log(d), math.log1p(-d)
    logpmf = np.array(
        [lg_n1 - math.lgamma(k + 1.0) - math.lgamma(n - k + 1.0) + k * ld + (n - k) * l1d
         for k in range(kmax + 1)]
    )
    cdf = np.cumsum(np.exp(logpmf - logpmf.max()))
    cdf /= cdf[-1]
    return cdf, kmax


def _binomial_counts(m: int, n: int, d: float, seed: int, stream: int) -> np.ndarray:
    """k_i ~ Binomial(n, d) by inverting the CDF at a counter uniform per row."""
    if m == 0:
        return np.zeros(0, dtype=np.int64)
    if d <= 0.0 or n == 0:
        return np.zeros(m, dtype=np.int64)
    if d >= 1.0:
        return np.full(m, n, dtype=np.int64)
    cdf, kmax = _binomial_cdf(n, d)
    u = counter_uniform(seed, stream, np.arange(m, dtype=np.uint64))
    k = np.searchsorted(cdf, u, side="right")
    return np.minimum(k, kmax).astype(np.int64)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (np.unique by sorting; numpy's hash-based unique is far slower
    on tens of millions of keys)."""
    a = np.sort(a)
    if a.shape[0] < 2:
        return a
    keep = np.empty(a.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _distinct_columns(k: np.ndarray, n: int, seed: int, stream: int) -> tuple:
    """For each row i, k[i] distinct columns drawn uniformly from [0, n); sorted per row.

    Sparse rows draw iid columns and redraw the shortfall left by duplicates (a uniform
    k-subset by symmetry). Rows with k > n/4 take the k smallest of n uniform keys.
    """
    m = k.shape[0]
    dense_rows = np.nonzero(k > max(n // 4, 0))[0] if n > 0 else np.zeros(0, np.int64)
    sparse_mask = np.ones(m, dtype=bool)
    sparse_mask[dense_rows] = False
    chosen = np.zeros(0, dtype=np.int64)
    need = np.where(sparse_mask, k, 0).astype(np.int64)
    rnd = 0
    while need.sum() > 0:
        if rnd >= 1023:
            raise RuntimeError("column sampling did not converge")
        rows_r = np.repeat(np.arange(m, dtype=np.int64), need)
        start = np.zeros(m + 1, dtype=np.int64)
        np.cumsum(need, out=start[1:])
        j = np.arange(rows_r.shape[0], dtype=np.int64) - start[rows_r]
        ctr = (rows_r.astype(np.uint64) << np.uint64(32)) | (np.uint64(rnd) << np.uint64(22)) | j.astype(np.uint64)
        c = np.minimum((counter_uniform(seed, stream, ctr) * n).astype(np.int64), n - 1)
        chosen = _sorted_unique(np.concatenate([chosen, rows_r * n + c]))
        have = np.bincount(chosen // n, minlength=m).astype(np.int64)
        need = np.where(sparse_mask, k - have, 0)
        rnd += 1
    parts = [chosen]
    for r in dense_rows:
        ctr = (np.uint64(int(r)) << np.uint64(32)) | np.uint64(1 << 31) | np.arange(n, dtype=np.uint64)
        u = counter_uniform(seed, stream, ctr)
        pick = np.sort(np.argsort(u, kind="stable")[: int(k[r])])
        parts.append(int(r) * n + pick.astype(np.int64))
    keys = np.sort(np.concatenate(parts)) if len(parts) > 1 else chosen
    rows = keys // n if n > 0 else keys
    cols = keys - rows * n
    return rows, cols


def uniform_random(m: int, n: int, density: float, seed: int = 0, *, stream_base: int = 0,
                   dtype=np.float64, lo: float = -1.0, hi: float = 1.0) -> CSR:
    """m x n matrix, per row Binomial(n, density) distinct uniform columns, values U[lo, hi)."""
    k = _binomial_counts(m, n, density, seed, stream_base + _ST_ROWCOUNT)
    rows, cols = _distinct_columns(k, n, seed, stream_base + _ST_COLUMNS)
    rp, col = _csr_from_sorted_keys(m, n, rows, cols)
    u = counter_uniform(seed, stream_base + _ST_VALUES, np.arange(col.shape[0], dtype=np.uint64))
    val = (lo + (hi - lo) * u).astype(dtype)
    return CSR(m, n, rp, col, val)


def random_small(m: int, n: int, density: float, seed: int, *, stream_base: int = 0,
                 dtype=np.float64, lo: float = -1.0, hi: float = 1.0) -> CSR:
    """Small test matrices of any density (same recipe as ``uniform_random``)."""
    return uniform_random(m, n, density, seed, stream_base=stream_base, dtype=dtype, lo=lo, hi=hi)


def identity(n: int, dtype=np.float64) -> CSR:
    return CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32),
               np.ones(n, dtype=dtype))


def from_dense(d: np.ndarray, pattern: np.ndarray | None = None, dtype=np.float64) -> CSR:
    """CSR of a dense array. ``pattern`` (bool) marks stored entries, so stored zeros are
    possible; without it the nonzeros are stored."""
    d = np.asarray(d, dtype=np.float64)
    mask = (d != 0) if pattern is None else np.asarray(pattern, dtype=bool)
    m, n = d.shape
    r, c = np.nonzero(mask)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=rp[1:])
    return CSR(m, n, rp, c.astype(np.int32), d[r, c].astype(dtype))


def _stencil(shape: tuple, diag: float, dtype) -> CSR:
    """Nearest-neighbour stencil on a row-major grid, neighbours listed in column order."""
    dims = len(shape)
    N = int(np.prod(shape))
    idx = np.arange(N, dtype=np.int64)
    coords = np.unravel_index(idx, shape)
    strides = [int(np.prod(shape[d + 1:])) for d in range(dims)]
    # offsets in increasing column order: -stride_0, ..., -stride_{dims-1}, 0, +stride_{dims-1}, ..., +stride_0
    offs = []
    for d in range(dims):
        offs.append((d, -1))
    offs.append((None, 0))
    for d in reversed(range(dims)):
        offs.append((d, +1))
    cols = np.empty((N, len(offs)), dtype=np.int64)
    valid = np.empty((N, len(offs)), dtype=bool)
    vals = np.empty((N, len(offs)), dtype=np.float64)
    for t, (d, s) in enumerate(offs):
        if d is None:
            cols[:, t] = idx
            valid[:, t] = True
            vals[:, t] = diag
        else:
            cols[:, t] = idx + s * strides[d]
            cd = coords[d] + s
            valid[:, t] = (cd >= 0) & (cd < shape[d])
            vals[:, t] = -1.0
    counts = valid.sum(axis=1)
    rp = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return CSR(N, N, rp, cols[valid].astype(np.int32), vals[valid].astype(dtype))


def laplacian2d(g: int, dtype=np.float64) -> CSR:
    """5-point Laplacian on a g x g grid (row-major), values 4 / -1."""
    return _stencil((g, g), 4.0, dtype)


def laplacian3d(g: int, dtype=np.float64) -> CSR:
    """7-point Laplacian on a g x g x g grid (row-major), values 6 / -1."""
    return _stencil((g, g, g), 6.0, dtype)


def aggregation_prolongator(g: int, dtype=np.float64) -> CSR:
    """Piecewise-constant prolongation of a 2D multigrid hierarchy: the (g*g) x ((g/2)*(g/2))
    matrix P with P[f, c] = 1 when fine node f = (y, x) of a row-major g x g grid lies in the
    2x2 aggregate c = (y // 2, x // 2) (g even). One entry per fine row."""
    if g % 2:
        raise ValueError("g must be even")
    h = g // 2
    f = np.arange(g * g, dtype=np.int64)
    y, x = f // g, f % g
    cols = (y // 2) * h + (x // 2)
    return CSR(g * g, h * h, np.arange(g * g + 1, dtype=np.int64), cols.astype(np.int32), np.ones(g * g, dtype=dtype))


def aggregation_restrictor(g: int, dtype=np.float64) -> CSR:
    """R = P^T for aggregation_prolongator(g): coarse row c lists its four fine nodes in order."""
    if g % 2:
        raise ValueError("g must be even")
    h = g // 2
    c = np.arange(h * h, dtype=np.int64)
    cy, cx = c // h, c % h
    base = (2 * cy) * g + 2 * cx
    cols = np.stack([base, base + 1, base + g, base + g + 1], axis=1).reshape(-1)
    return CSR(h * h, g * g, np.arange(0, 4 * h * h + 1, 4, dtype=np.int64), cols.astype(np.int32),
               np.ones(4 * h * h, dtype=dtype))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, dtype=np.float64, lo: float = 0.0, hi: float = 1.0,
         chunk: int = 1 << 22) -> CSR:
    """R-MAT graph adjacency as CSR: 2^scale vertices, edge_factor * 2^scale samples.

    Edge e at level l (most significant bit first) picks quadrant by the counter uniform
    (e * scale + l): [0,a) -> (0,0), [a,a+b) -> (0,1), [a+b,a+b+c) -> (1,0), else (1,1).
    """
    n = 1 << scale
    E = edge_factor * n
    keys_parts = []
    ab, abc = a + b, a + b + c
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        e = np.arange(e0, e1, dtype=np.uint64)
        r = np.zeros(e1 - e0, dtype=np.int64)
        q = np.zeros(e1 - e0, dtype=np.int64)
        for lvl in range(scale):
            u = counter_uniform(seed, _ST_RMAT_EDGE, e * np.uint64(scale) + np.uint64(lvl))
            rb = (u >= ab).astype(np.int64)
            cb = (((u >= a) & (u < ab)) | (u >= abc)).astype(np.int64)
            bit = scale - 1 - lvl
            r |= rb << bit
            q |= cb << bit
        keys_parts.append((r << scale) | q)
    keys = _sorted_unique(np.concatenate(keys_parts))
    rows = keys >> scale
    cols = keys & (n - 1)
    rp, col = _csr_from_sorted_keys(n, n, rows, cols)
    u = counter_uniform(seed, _ST_RMAT_VAL, np.arange(col.shape[0], dtype=np.uint64))
    val = (lo + (hi - lo) * u).astype(dtype)
    return CSR(n, n, rp, col, val)


def batch_job_params(i: int, seed: int = 0, n_lo: int = 100, n_hi: int = 50_000,
                     d_lo: float = 1e-4, d_hi: float = 1e-2) -> tuple:
    """(n_i, d_i) of batch job i: n log-uniform in [n_lo, n_hi], d log-uniform in [d_lo, d_hi]."""
    u = counter_uniform(seed, _ST_BATCH_PARAM, np.array([2 * i, 2 * i + 1], dtype=np.uint64))
    n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
    d = math.exp(math.log(d_lo) + u[1] * (math.log(d_hi) - math.log(d_lo)))
    return n, d


def batch_job(i: int, seed: int = 0, dtype=np.float64, **param_kw) -> tuple:
    """Independent square A_i, B_i with the job's (n_i, d_i); values U[-1, 1)."""
    n, d = batch_job_params(i, seed, **param_kw)
    base = _ST_JOB_BASE + 16 * i
    A = uniform_random(n, n, d, seed, stream_base=base, dtype=dtype)
    B = uniform_random(n, n, d, seed, stream_base=base + 8, dtype=dtype)
    return A, B


@dataclass
class Request:
    """One served SpGEMM request: arrival time (s) and how to build its inputs."""

    index: int
    arrival_s: float
    kind: str            # "batch" (A_i * B_i from the batch distribution) or "lap3d" (A*A)
    param: int           # batch job index, or grid size g


def serve_stream(num: int, rate_per_s: float, seed: int = 0, lap_fraction: float = 0.1,
                 g_lo: int = 64, g_hi: int = 128) -> list:
    """Poisson arrivals at ``rate_per_s``; (1 - lap_fraction) batch-distribution jobs and
    lap_fraction 3D Laplacian squares with g uniform in {g_lo..g_hi}."""
    c = np.arange(num, dtype=np.uint64)
    u_gap = counter_uniform(seed, _ST_SERVE, 3 * c)
    u_kind = counter_uniform(seed, _ST_SERVE, 3 * c + np.uint64(1))
    u_par = counter_uniform(seed, _ST_SERVE, 3 * c + np.uint64(2))
    gaps = -np.log1p(-u_gap) / rate_per_s
    t = np.cumsum(gaps)
    out = []
    for i in range(num):
        if u_kind[i] < lap_fraction:
            g = g_lo + min(int(u_par[i] * (g_hi - g_lo + 1)), g_hi - g_lo)
            out.append(Request(i, float(t[i]), "lap3d", g))
        else:
            out.append(Request(i, float(t[i]), "batch", 100_000 + i))
    return out
