"""The oracle against its frozen fixtures (tests/golden/), and the fixtures against facts
outside the oracle: the closed form of the squared 5-point stencil and a dense product."""

import os

import numpy as np

import oracle
import synth

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    with open(os.path.join(HERE, name + ".txt")) as f:
        lines = [ln.strip() for ln in f if not ln.startswith("#")]
    m, n, nnz = (int(x) for x in lines[0].split())
    rp = np.array([int(x) for x in lines[1].split()], dtype=np.int64)
    col = np.array([int(x) for x in lines[2].split()], dtype=np.int32)
    val = np.array([float.fromhex(x) for x in lines[3].split()], dtype=np.float64)
    assert rp.shape == (m + 1,) and col.shape == (nnz,) and val.shape == (nnz,)
    return m, n, rp, col, val


def test_uniform_fixture():
    m, n, rp, col, val = _read("uniform_40x40_d0.1_seed21")
    A = synth.uniform_random(40, 40, 0.1, 21)
    out = oracle.spgemm(A, A)
    assert np.array_equal(out.row_ptr, rp) and np.array_equal(out.col, col)
    assert np.array_equal(out.val, val)
    d = np.zeros((m, n))
    d[np.repeat(np.arange(m), np.diff(rp)), col] = val
    Ad = A.to_dense()
    assert np.all(np.abs(d - Ad @ Ad) <= 1e-12 * (np.abs(Ad) @ np.abs(Ad)))


def test_laplacian_fixture_closed_form():
    m, n, rp, col, val = _read("laplacian2d_g5_squared")
    L = synth.laplacian2d(5)
    out = oracle.spgemm(L, L)
    assert np.array_equal(out.row_ptr, rp) and np.array_equal(out.col, col)
    assert np.array_equal(out.val, val)
    g = 5
    for p in range(m):
        py, px = divmod(p, g)
        for q, v in zip(col[rp[p]:rp[p + 1]], val[rp[p]:rp[p + 1]]):
            qy, qx = divmod(int(q), g)
            dy, dx = qy - py, qx - px
            l1 = abs(dy) + abs(dx)
            if l1 == 0:
                nb = (py > 0) + (py < g - 1) + (px > 0) + (px < g - 1)
                assert v == 16 + nb
            elif l1 == 1:
                assert v == -8
            elif dy == 0 or dx == 0:
                assert v == 1
            else:
                assert v == 2
