"""The uniform-pattern generators of ``generators`` written with torch, so the batch-distribution
jobs can be built directly in device memory. Every draw is the same SplitMix64 counter output as
in ``generators`` (the counter layouts, the inverse-CDF row counts, the rounds of distinct-column
draws and the CSR-order values are the same), so the matrices are bit-identical to the numpy
ones on any device; a test compares them on the CPU.

Like ``generators``, this module only builds inputs: it never multiplies, merges or sorts partial
products.
"""

from __future__ import annotations

import numpy as np
import torch

from . import generators as G


def _signed(u: int) -> int:
    """The int64 with the bit pattern of the uint64 u."""
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


_GAMMA = _signed(int(G.GAMMA))
_M1 = _signed(int(G._M1))
_M2 = _signed(int(G._M2))


def _srl(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 holding uint64 bit patterns."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function (int64 arithmetic wraps modulo 2^64, as uint64 does)."""
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def counter_u64(seed: int, stream: int, counters: torch.Tensor) -> torch.Tensor:
    """The bit patterns of generators.counter_u64 as int64."""
    key = _signed(int(G._key(seed, stream)))
    return _mix(key + (counters + 1) * _GAMMA)


def counter_uniform(seed: int, stream: int, counters: torch.Tensor) -> torch.Tensor:
    """generators.counter_uniform: doubles in [0, 1) with 53 random bits."""
    return _srl(counter_u64(seed, stream, counters), 11).to(torch.float64) * G._INV53


def _binomial_counts(m: int, n: int, d: float, seed: int, stream: int, device) -> torch.Tensor:
    if m == 0:
        return torch.zeros(0, dtype=torch.int64, device=device)
    if d <= 0.0 or n == 0:
        return torch.zeros(m, dtype=torch.int64, device=device)
    if d >= 1.0:
        return torch.full((m,), n, dtype=torch.int64, device=device)
    cdf, kmax = G._binomial_cdf(n, d)
    u = counter_uniform(seed, stream, torch.arange(m, dtype=torch.int64, device=device))
    k = torch.searchsorted(torch.from_numpy(cdf).to(device), u, right=True)
    return torch.clamp(k, max=kmax)


def _distinct_columns(k: torch.Tensor, n: int, seed: int, stream: int) -> tuple:
    """generators._distinct_columns: rows (sorted) and columns of the chosen keys. Sparse rows draw
    iid columns and redraw the shortfall; rows with k > n/4 take the k smallest of n keys."""
    device = k.device
    m = k.shape[0]
    dense = torch.nonzero(k > max(n // 4, 0)).flatten() if n > 0 else torch.zeros(0, dtype=torch.int64)
    chosen = torch.zeros(0, dtype=torch.int64, device=device)
    need = k.clone()
    if dense.numel():
        need[dense] = 0
    rnd = 0
    while int(need.sum()) > 0:
        if rnd >= 1023:
            raise RuntimeError("column sampling did not converge")
        rows_r = torch.repeat_interleave(torch.arange(m, dtype=torch.int64, device=device), need)
        start = torch.cumsum(need, 0) - need
        j = torch.arange(rows_r.shape[0], dtype=torch.int64, device=device) - start[rows_r]
        ctr = (rows_r << 32) | (rnd << 22) | j
        c = torch.clamp((counter_uniform(seed, stream, ctr) * n).to(torch.int64), max=n - 1)
        chosen = torch.unique(torch.cat([chosen, rows_r * n + c]), sorted=True)
        have = torch.bincount(torch.div(chosen, n, rounding_mode="floor"), minlength=m)
        need = k - have
        if dense.numel():
            need[dense] = 0
        rnd += 1
    parts = [chosen]
    for r in dense.tolist():
        ctr = (r << 32) | (1 << 31) | torch.arange(n, dtype=torch.int64, device=device)
        u = counter_uniform(seed, stream, ctr)
        pick = torch.sort(torch.argsort(u, stable=True)[: int(k[r])]).values
        parts.append(r * n + pick)
    if len(parts) > 1:
        chosen = torch.sort(torch.cat(parts)).values
    rows = torch.div(chosen, n, rounding_mode="floor") if n > 0 else chosen
    return rows, chosen - rows * n


def uniform_random(m: int, n: int, density: float, seed: int = 0, *, stream_base: int = 0, device="cuda",
                   dtype=torch.float64, lo: float = -1.0, hi: float = 1.0) -> tuple:
    """generators.uniform_random on `device`: (row_ptr int64, col int32, val) tensors."""
    k = _binomial_counts(m, n, density, seed, stream_base + G._ST_ROWCOUNT, device)
    rows, cols = _distinct_columns(k, n, seed, stream_base + G._ST_COLUMNS)
    rp = torch.zeros(m + 1, dtype=torch.int64, device=device)
    if m:
        rp[1:] = torch.cumsum(torch.bincount(rows, minlength=m), 0)
    u = counter_uniform(seed, stream_base + G._ST_VALUES, torch.arange(cols.shape[0], dtype=torch.int64,
                                                                          device=device))
    val = (lo + (hi - lo) * u).to(dtype)
    return rp, cols.to(torch.int32), val


def batch_job(i: int, seed: int = 0, device="cuda", dtype=torch.float64) -> tuple:
    """generators.batch_job on `device`: (n, A tensors, B tensors), each (row_ptr, col, val)."""
    n, d = G.batch_job_params(i, seed)
    base = G._ST_JOB_BASE + 16 * i
    A = uniform_random(n, n, d, seed, stream_base=base, device=device, dtype=dtype)
    B = uniform_random(n, n, d, seed, stream_base=base + 8, device=device, dtype=dtype)
    return n, A, B
