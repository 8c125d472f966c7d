"""Pins of the CPU oracle to facts outside itself (no GPU).

The oracle is the row-by-row product of Algorithm 1 (Sec. III-A). Each test below checks
it against something it does not share code with:

* a dense matrix product of the same matrices (values, per-entry magnitude, term count);
* a dense boolean product of the stored patterns (structure, including stored zeros);
* A*I = A and I*B = B, exact;
* closed forms of the 2D and 3D Laplacian squares (exact integers, counts and values);
* scipy's sparse product on all-ones copies (counts of partial products per entry);
* the O(n) identity sum_i P_i = sum_k nnz(column k of A) * nnz(row k of B);
* cancellation to an exact zero stays a stored entry (Algorithm 1 emits every column of
  COLB, Sec. III-A);
* degenerate shapes (empty matrices, empty rows, 1x1, rectangular).

A dropped term, a wrong sign or index, or a transposed operand fails the dense and the
rectangular tests; a missed or extra column fails the boolean-pattern test.
"""

import numpy as np
import pytest

import oracle
import synth


def _dense(M):
    return M.to_dense()


def _pattern(M):
    p = np.zeros((M.rows, M.cols), dtype=np.int64)
    r = np.repeat(np.arange(M.rows), M.row_lengths())
    p[r, M.col] = 1
    return p


def _to_dense_out(out, m, n):
    d = np.zeros((m, n))
    mg = np.zeros((m, n))
    t = np.zeros((m, n), dtype=np.int64)
    s = np.zeros((m, n), dtype=bool)
    r = np.repeat(np.arange(m), np.diff(out.row_ptr))
    d[r, out.col] = out.val
    mg[r, out.col] = out.mag
    t[r, out.col] = out.terms
    s[r, out.col] = True
    return d, mg, t, s


SHAPES = [(1, 1, 1), (3, 5, 2), (7, 7, 7), (16, 9, 23), (24, 24, 24), (40, 13, 31)]
DENSITIES = [0.05, 0.2, 0.5, 1.0]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("density", DENSITIES)
def test_dense_and_boolean_product(shape, density):
    m, k, n = shape
    seed = 1000 + m * 7 + k * 3 + n + int(density * 100)
    A = synth.random_small(m, k, density, seed, stream_base=0)
    B = synth.random_small(k, n, density, seed, stream_base=64)
    out = oracle.spgemm(A, B)
    d, mg, t, s = _to_dense_out(out, m, n)
    pa, pb = _pattern(A), _pattern(B)
    # structure: exactly the stored entries of the boolean product, sorted per row
    assert np.array_equal(s, (pa @ pb) > 0)
    for i in range(m):
        c = out.col[out.row_ptr[i]:out.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    # term counts: number of k with A_ik and B_kj stored
    assert np.array_equal(t, pa @ pb)
    # values and magnitudes against the dense product
    ref = _dense(A) @ _dense(B)
    refmag = np.abs(_dense(A)) @ np.abs(_dense(B))
    assert np.all(np.abs(d - ref) <= 1e-12 * refmag + 1e-300)
    assert np.allclose(mg, refmag, rtol=1e-13, atol=0)


def test_rectangular_not_square_catches_transpose():
    A = synth.random_small(5, 9, 0.5, 7)
    B = synth.random_small(9, 3, 0.5, 8)
    out = oracle.spgemm(A, B)
    d, _, _, _ = _to_dense_out(out, 5, 3)
    assert np.allclose(d, _dense(A) @ _dense(B), rtol=1e-13, atol=1e-15)
    with pytest.raises(ValueError):
        oracle.spgemm(B, A)


def test_identity_exact():
    A = synth.uniform_random(300, 200, 0.03, 11)
    I200 = synth.identity(200)
    I300 = synth.identity(300)
    out = oracle.spgemm(A, I200)
    assert np.array_equal(out.row_ptr, A.row_ptr)
    assert np.array_equal(out.col, A.col)
    assert np.array_equal(out.val, A.val)
    out2 = oracle.spgemm(I300, A)
    assert np.array_equal(out2.row_ptr, A.row_ptr)
    assert np.array_equal(out2.col, A.col)
    assert np.array_equal(out2.val, A.val)


def test_cancellation_keeps_structural_zero():
    # [1 1] * [1 -1]^T = 0, stored (Algorithm 1 emits every column of COLB)
    A = synth.from_dense(np.array([[1.0, 1.0]]))
    B = synth.from_dense(np.array([[1.0], [-1.0]]))
    out = oracle.spgemm(A, B)
    assert out.nnz == 1 and out.col[0] == 0 and out.val[0] == 0.0
    assert out.mag[0] == 2.0 and out.terms[0] == 2


def test_stored_zeros_are_structural():
    pat = np.array([[True, True, False], [False, True, True]])
    A = synth.from_dense(np.array([[0.0, 2.0, 0.0], [0.0, 0.0, 3.0]]), pattern=pat)
    B = synth.from_dense(np.eye(3), pattern=np.eye(3, dtype=bool))
    out = oracle.spgemm(A, B)
    assert list(out.col) == [0, 1, 1, 2]
    assert list(out.val) == [0.0, 2.0, 0.0, 3.0]


@pytest.mark.parametrize("m,k,n", [(0, 0, 0), (0, 5, 3), (4, 0, 3), (4, 5, 0), (1, 1, 1)])
def test_degenerate_shapes(m, k, n):
    A = synth.random_small(m, k, 0.5, 3)
    B = synth.random_small(k, n, 0.5, 4)
    out = oracle.spgemm(A, B)
    assert out.row_ptr.shape == (m + 1,)
    if m * n == 0 or k == 0:
        assert out.nnz == 0


def test_empty_rows_and_single_dense_row():
    D = np.zeros((6, 6))
    D[2, :] = np.arange(1, 7)
    A = synth.from_dense(D)
    B = synth.from_dense(np.arange(36.0).reshape(6, 6) - 17.0)
    out = oracle.spgemm(A, B)
    lens = np.diff(out.row_ptr)
    assert list(lens) == [0, 0, 6, 0, 0, 0]
    d, _, _, _ = _to_dense_out(out, 6, 6)
    assert np.array_equal(d[2], D[2] @ B.to_dense())


def _lap2d_closed_form(g):
    """(nnz(C), P) of C = L^2 for the 5-point Dirichlet Laplacian on a g x g grid.

    The pattern of L^2 is every pair at grid distance <= 2 whose length-2 path stays in
    the grid (the diagonal is stored): offsets (0,0), 4 axis-1, 4 axis-2 and 4 diagonal.
    P = sum_k deg(k)^2 with deg = 1 + number of in-grid neighbours.
    """
    nnz = g * g + 4 * g * (g - 1) + 4 * g * max(g - 2, 0) + 4 * (g - 1) ** 2
    if g == 1:
        P = 1
    else:
        P = 4 * 9 + 4 * (g - 2) * 16 + (g - 2) ** 2 * 25
    return nnz, P


def _lap_square_value(shape, diag, p, q):
    """Closed-form entry (p, q) of L^2 for a d-dimensional grid stencil L."""
    dims = len(shape)
    cp = np.unravel_index(p, shape)
    cq = np.unravel_index(q, shape)
    delta = [int(cq[d]) - int(cp[d]) for d in range(dims)]
    l1 = sum(abs(x) for x in delta)
    if l1 == 0:
        nb = sum(int(cp[d] > 0) + int(cp[d] < shape[d] - 1) for d in range(dims))
        return diag * diag + nb
    if l1 == 1:
        return -2.0 * diag
    nz = [d for d in range(dims) if delta[d] != 0]
    if len(nz) == 1:
        return 1.0          # axis +-2: one path through the middle point
    return 2.0              # two different axes +-1: two paths, both in the grid


@pytest.mark.parametrize("g", [1, 2, 3, 4, 7, 16])
def test_laplacian2d_square_closed_form_small(g):
    L = synth.laplacian2d(g)
    out = oracle.spgemm(L, L)
    nnz, P = _lap2d_closed_form(g)
    assert out.nnz == nnz
    assert int(oracle.products_per_row(L, L).sum()) == P
    assert int(out.terms.astype(np.int64).sum()) == P
    r = np.repeat(np.arange(L.rows), np.diff(out.row_ptr))
    for p, q, v in zip(r, out.col, out.val):
        assert v == _lap_square_value((g, g), 4.0, int(p), int(q))
        cp, cq = np.unravel_index(p, (g, g)), np.unravel_index(q, (g, g))
        assert abs(cp[0] - cq[0]) + abs(cp[1] - cq[1]) <= 2


def test_laplacian2d_1024_counts_and_interior_values():
    """The 2D Laplacian config at full size: nnz(C) = 13,611,012, P = 26,177,544, and the
    interior 13-point stencil 20 / -8 / 1 / 2."""
    g = 1024
    L = synth.laplacian2d(g)
    assert L.nnz == 5 * g * g - 4 * g
    assert int(oracle.products_per_row(L, L).sum()) == 26_177_544
    rows = np.array([0, 1, g - 1, g, g + 1, 5 * g + 7, g * g // 2 + 300, g * g - 1])
    out = oracle.spgemm(L, L, rows=rows)
    for t, p in enumerate(rows):
        cs = out.col[out.row_ptr[t]:out.row_ptr[t + 1]]
        vs = out.val[out.row_ptr[t]:out.row_ptr[t + 1]]
        for q, v in zip(cs, vs):
            assert v == _lap_square_value((g, g), 4.0, int(p), int(q))
    interior = out.val[out.row_ptr[6]:out.row_ptr[7]]
    assert sorted(interior.tolist()) == sorted([20.0] + [-8.0] * 4 + [1.0] * 4 + [2.0] * 4)
    assert _lap2d_closed_form(g) == (13_611_012, 26_177_544)


@pytest.mark.slow
def test_laplacian2d_1024_full_nnz():
    L = synth.laplacian2d(1024)
    out = oracle.spgemm(L, L)
    assert out.nnz == 13_611_012


@pytest.mark.parametrize("g", [2, 3, 5, 8])
def test_laplacian3d_square_closed_form(g):
    L = synth.laplacian3d(g)
    out = oracle.spgemm(L, L)
    r = np.repeat(np.arange(L.rows), np.diff(out.row_ptr))
    for p, q, v in zip(r, out.col, out.val):
        assert v == _lap_square_value((g, g, g), 6.0, int(p), int(q))
    # pattern = all pairs at L1 distance <= 2 (every such pair has an in-grid 2-path)
    coords = np.stack(np.unravel_index(np.arange(g ** 3), (g, g, g)), axis=1)
    dist = np.abs(coords[:, None, :] - coords[None, :, :]).sum(axis=2)
    assert out.nnz == int((dist <= 2).sum())
    if g >= 5:
        c = (g // 2) * (g * g + g + 1)
        vs = out.val[out.row_ptr[c]:out.row_ptr[c + 1]]
        assert sorted(vs.tolist()) == sorted([42.0] + [-12.0] * 6 + [1.0] * 6 + [2.0] * 12)


@pytest.mark.parametrize("seed", [0, 1])
def test_scipy_pattern_counts(seed):
    sp = pytest.importorskip("scipy.sparse")
    A = synth.uniform_random(400, 300, 0.02, seed)
    B = synth.uniform_random(300, 500, 0.02, seed + 50)
    out = oracle.spgemm(A, B, values=False)
    SA = sp.csr_matrix((np.ones(A.nnz), A.col, A.row_ptr), shape=(A.rows, A.cols))
    SB = sp.csr_matrix((np.ones(B.nnz), B.col, B.row_ptr), shape=(B.rows, B.cols))
    SC = (SA @ SB).tocsr()
    SC.sort_indices()
    assert np.array_equal(SC.indptr.astype(np.int64), out.row_ptr)
    assert np.array_equal(SC.indices, out.col)
    assert np.array_equal(SC.data, out.val)          # path counts, exact
    assert np.array_equal(out.terms.astype(np.float64), out.val)


def test_products_sum_identity():
    A = synth.uniform_random(500, 400, 0.01, 5)
    B = synth.uniform_random(400, 700, 0.02, 6)
    P = oracle.products_per_row(A, B)
    colcount = np.bincount(A.col, minlength=A.cols)
    assert int(P.sum()) == int((colcount * np.diff(B.row_ptr)).sum())
    out = oracle.spgemm(A, B)
    per_row_terms = np.add.reduceat(out.terms.astype(np.int64), out.row_ptr[:-1]) \
        if out.nnz else np.zeros(A.rows, np.int64)
    per_row_terms = np.where(np.diff(out.row_ptr) > 0, per_row_terms, 0)
    assert np.array_equal(per_row_terms, P)


def test_row_subset_matches_full():
    A = synth.uniform_random(800, 800, 0.01, 9)
    full = oracle.spgemm(A, A)
    rows = np.array([799, 0, 5, 5, 400])
    sub = oracle.spgemm(A, A, rows=rows)
    for t, i in enumerate(rows):
        a = slice(full.row_ptr[i], full.row_ptr[i + 1])
        b = slice(sub.row_ptr[t], sub.row_ptr[t + 1])
        assert np.array_equal(full.col[a], sub.col[b])
        assert np.array_equal(full.val[a], sub.val[b])


def test_fp32_inputs_widen_exactly():
    A = synth.uniform_random(200, 200, 0.05, 12, dtype=np.float32, lo=0.0, hi=1.0)
    out = oracle.spgemm(A, A)
    d, mg, _, _ = _to_dense_out(out, 200, 200)
    Ad = A.to_dense()
    ref = Ad @ Ad
    assert np.all(np.abs(d - ref) <= 1e-12 * (np.abs(Ad) @ np.abs(Ad)) + 1e-300)


# ---- exact_sum: every value the correctly rounded sum of the entry's rounded products ----

def _one_row(products):
    """A 1 x t row of ones times a t x 1 column holding the given products: one entry whose
    partial products are exactly `products`, in this order."""
    t = len(products)
    A = synth.CSR(1, t, np.array([0, t], np.int64), np.arange(t, dtype=np.int32), np.ones(t))
    B = synth.CSR(t, 1, np.arange(t + 1, dtype=np.int64), np.zeros(t, np.int32), np.array(products, np.float64))
    return A, B


def test_exact_sum_closed_forms():
    # 1e16 + 1 - 1e16: stored order loses the 1, the exact sum is 1
    A, B = _one_row([1e16, 1.0, -1e16])
    assert oracle.spgemm(A, B).val[0] == 0.0
    assert oracle.spgemm(A, B, exact_sum=True).val[0] == 1.0
    # a tie rounds to even; anything past the tie rounds away
    A, B = _one_row([1.0, 2.0 ** -53])
    assert oracle.spgemm(A, B, exact_sum=True).val[0] == 1.0
    A, B = _one_row([1.0, 2.0 ** -53, 2.0 ** -80])
    assert oracle.spgemm(A, B, exact_sum=True).val[0] == 1.0 + 2.0 ** -52
    A, B = _one_row([1.0 + 2.0 ** -52, 2.0 ** -53])   # odd last bit: the tie goes up
    assert oracle.spgemm(A, B, exact_sum=True).val[0] == 1.0 + 2.0 ** -51
    A, B = _one_row([-(1.0 + 2.0 ** -52), -(2.0 ** -53)])
    assert oracle.spgemm(A, B, exact_sum=True).val[0] == -(1.0 + 2.0 ** -51)
    # full cancellation of many terms stays a stored zero
    A, B = _one_row([0.1, 0.2, 0.3, -0.1, -0.2, -0.3])
    out = oracle.spgemm(A, B, exact_sum=True)
    assert out.nnz == 1 and out.val[0] == 0.0


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_exact_sum_equals_math_fsum(seed):
    """Against Python's math.fsum (an exactly rounded summation in the standard library) over
    the products of each entry, on values spread over 16 decades with signs mixed."""
    import math
    rng = np.random.default_rng(seed)
    A = synth.random_small(30, 40, 0.4, seed)
    B = synth.random_small(40, 25, 0.4, seed + 100)
    A = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, A.val * 10.0 ** rng.uniform(-8, 8, A.nnz))
    B = synth.CSR(B.rows, B.cols, B.row_ptr, B.col, B.val * 10.0 ** rng.uniform(-8, 8, B.nnz))
    out = oracle.spgemm(A, B, exact_sum=True)
    for i in range(A.rows):
        acc = {}
        for q in range(A.row_ptr[i], A.row_ptr[i + 1]):
            k = A.col[q]
            for t in range(B.row_ptr[k], B.row_ptr[k + 1]):
                acc.setdefault(int(B.col[t]), []).append(float(A.val[q]) * float(B.val[t]))
        s = slice(out.row_ptr[i], out.row_ptr[i + 1])
        assert list(out.col[s]) == sorted(acc)
        want = np.array([math.fsum(acc[int(j)]) for j in out.col[s]])
        assert np.array_equal(out.val[s], want)


def test_exact_sum_equals_stored_order_on_integers():
    A = synth.rmat(9, 8, seed=7)
    A = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, np.floor(A.val * 8.0) - 3.0)
    a = oracle.spgemm(A, A)
    b = oracle.spgemm(A, A, exact_sum=True)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.mag, b.mag) and np.array_equal(a.terms, b.terms)


@pytest.mark.parametrize("case", ["uniform", "rmat", "rect", "signed_wide", "empty"])
def test_dense_accumulator_equals_ordered_map(case):
    """The dense-accumulator path adds every entry's products in the same stored order as the
    ordered map: row pointers, columns, values, magnitudes and term counts are bit-identical."""
    if case == "uniform":
        A = B = synth.uniform_random(800, 800, 0.01, seed=31)
    elif case == "rmat":
        A = B = synth.rmat(11, 16, seed=32)
    elif case == "rect":
        A = synth.uniform_random(300, 700, 0.02, seed=33)
        B = synth.uniform_random(700, 5000, 0.004, seed=34)
    elif case == "signed_wide":
        rng = np.random.default_rng(35)
        A = synth.random_small(60, 80, 0.3, 36)
        A = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, A.val * 10.0 ** rng.uniform(-12, 12, A.nnz))
        B = synth.random_small(80, 50, 0.3, 37)
    else:
        A = synth.random_small(0, 5, 0.5, 38)
        B = synth.random_small(5, 9, 0.5, 39)
    a = oracle.spgemm(A, B, method="map")
    b = oracle.spgemm(A, B, method="dense")
    for f in ("row_ptr", "col", "mag", "terms"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert np.array_equal(a.val.view(np.uint64), b.val.view(np.uint64))
    rows = np.arange(0, A.rows, 3)
    assert np.array_equal(oracle.spgemm(A, B, rows=rows, method="dense").val,
                          oracle.spgemm(A, B, rows=rows, method="map").val)


@pytest.mark.parametrize("g", [2, 4, 10, 64])
def test_galerkin_coarse_laplacian_closed_form(g):
    """Multigrid Galerkin product R*(A*P) with 2x2 aggregation (P piecewise constant, R = P^T) of
    the 2D 5-point Laplacian: every coarse entry sums the fine couplings between two aggregates,
    16 - 8 = 8 on the diagonal and -2 between neighbouring aggregates, i.e. exactly twice the
    5-point Laplacian of the coarse grid (Dirichlet boundaries included)."""
    A = synth.laplacian2d(g)
    P = synth.aggregation_prolongator(g)
    R = synth.aggregation_restrictor(g)
    assert np.array_equal(R.to_dense(), P.to_dense().T)
    AP = oracle.spgemm(A, P)
    APc = synth.CSR(A.rows, P.cols, AP.row_ptr, AP.col, AP.val)
    Ac = oracle.spgemm(R, APc)
    L = synth.laplacian2d(g // 2)
    assert np.array_equal(Ac.row_ptr, L.row_ptr) and np.array_equal(Ac.col, L.col)
    assert np.array_equal(Ac.val, 2.0 * L.val)
