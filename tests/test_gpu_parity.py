"""CUDA path vs the CPU oracle, element by element (FP64).

Structure (row_ptr, col) must be bit-equal; every value within 1e-12 * sum|a_ik*b_kj| of
the oracle's. Every row class is exercised: by the natural size mix of the workloads and
by forcing paths through the tuning knobs (tiny rows off, warp/block tables off, every row
windowed, the int64 row_ptr path at a low limit).
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_parity, compare_all_rows, gpu_or_skip, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    gpu_or_skip()


def opts(**kw):
    import paper_2004_13907_gb300 as sp
    return sp.spgemm_opts_default(**kw)


@pytest.mark.parametrize("general", [0, 1])
def test_uniform_10k_full(general):
    """C = A*A, A 10,000 x 10,000 at density 1e-3 (~10 per row), values U[-1,1]: the small-product
    path and the general row classes."""
    A = synth.uniform_random(10_000, 10_000, 1e-3, seed=0)
    rp, col, val, info0, info, _ = run_gpu(A, A, opts=opts(general_path=general))
    assert info["products"] == int(oracle.products_per_row(A, A).sum())
    assert_parity(A, A, rp, col, val)


@pytest.mark.parametrize("g", [1, 2, 7, 64, 300])
def test_laplacian2d_small(g):
    L = synth.laplacian2d(g)
    rp, col, val, *_ = run_gpu(L, L)
    assert_parity(L, L, rp, col, val)


def test_laplacian2d_1024_full():
    """The 2D Laplacian config at full size (1,048,576 rows), every entry compared."""
    L = synth.laplacian2d(1024)
    rp, col, val, info0, info, _ = run_gpu(L, L)
    assert info0["products"] == 26_177_544
    assert info["nnz_c"] == 13_611_012
    ref = assert_parity(L, L, rp, col, val)
    assert np.array_equal(val, ref.val)   # small exact integers: bit-exact in any order


@pytest.mark.parametrize("scale", [10, 13, 15])
@pytest.mark.parametrize("general", [0, 1])
def test_rmat_small_full(scale, general):
    A = synth.rmat(scale, 16, seed=3)
    rp, col, val, info0, info, _ = run_gpu(A, A, opts=opts(general_path=general))
    assert_parity(A, A, rp, col, val)


@pytest.mark.parametrize("kw", [
    dict(force_window=1),
    dict(tiny_max=0),
    dict(tiny_max=0, warp_max=0),
    dict(warp_max=64, block_max=64),
    dict(window_hash_fill=64),
    dict(force_window=1, window_hash_fill=1),
    dict(force_window=1, window_split_max_mb=0),
    dict(validate=0),
    dict(max_sms=7),
    dict(force_window=1, window_cols_max_mb=0),
    dict(force_window=1, window_cols_max_mb=1),
])
def test_forced_paths_rmat(kw):
    A = synth.rmat(12, 16, seed=5)
    B = synth.uniform_random(A.cols, 3000, 2e-3, seed=6)
    rp, col, val, *_ = run_gpu(A, B, opts=opts(**kw))
    assert_parity(A, B, rp, col, val)


@pytest.mark.parametrize("kw", [dict(force_window=1), dict(tiny_max=0, warp_max=0), dict()])
def test_forced_paths_uniform_rectangular(kw):
    A = synth.uniform_random(700, 3000, 5e-3, seed=7)
    B = synth.uniform_random(3000, 40_000, 2e-3, seed=8)
    rp, col, val, *_ = run_gpu(A, B, opts=opts(**kw))
    assert_parity(A, B, rp, col, val)


def test_window_columns_beyond_one_bitmap():
    """n > 2^20 columns: the symbolic bitmap slides over windows with cursors."""
    n = (1 << 20) + 70_000
    A = synth.uniform_random(300, 200, 0.05, seed=9)
    B = synth.uniform_random(200, n, 3e-3, seed=10)
    rp, col, val, *_ = run_gpu(A, B, opts=opts(force_window=1))
    assert_parity(A, B, rp, col, val)
    rp2, col2, val2, *_ = run_gpu(A, B)
    assert_parity(A, B, rp2, col2, val2)


def test_dense_small_n_window():
    """Rows denser than a hash window: dense windows on a narrow B."""
    A = synth.uniform_random(500, 400, 0.2, seed=11)
    B = synth.uniform_random(400, 20_000, 0.05, seed=12)
    rp, col, val, _, info, _ = run_gpu(A, B)
    assert_parity(A, B, rp, col, val)


def test_int64_rowptr_path():
    A = synth.uniform_random(2000, 2000, 4e-3, seed=13)
    rp, col, val, _, info, C = run_gpu(A, A, opts=opts(rowptr32_limit=1000), idx64_in=True)
    assert info["needs_rowptr64"] == 1 and C.row_ptr.dtype == torch.int64
    assert_parity(A, A, rp, col, val)


def test_int32_output_refused_when_too_large():
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(500, 500, 1e-2, seed=14)
    dA = sp.DeviceCSR.from_host(A, "cuda")
    plan = sp.spgemm_plan(dA, dA, "f64", opts(rowptr32_limit=100))
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan, idx64=False)
    with pytest.raises(sp.SpgemmError) as ei:
        sp.spgemm_numeric(plan, C)
    assert ei.value.name == "INDEX_OVERFLOW"


def _short_rows(m, k, n, na_of, blen_max, seed):
    """A with na_of(i) entries in row i, B with 0..blen_max entries per row over n columns."""
    rng = np.random.default_rng(seed)
    na = np.array([na_of(i) for i in range(m)], dtype=np.int64)
    arp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(na, out=arp[1:])
    acol = np.concatenate([np.sort(rng.choice(k, int(x), replace=False)) for x in na]).astype(np.int32)
    blen = rng.integers(0, blen_max + 1, k)
    brp = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(blen, out=brp[1:])
    bcol = np.concatenate([np.sort(rng.choice(n, int(x), replace=False)) for x in blen]).astype(np.int32)
    A = synth.CSR(m, k, arp, acol, rng.uniform(-1, 1, int(arp[-1])))
    B = synth.CSR(k, n, brp, bcol, rng.uniform(-1, 1, int(brp[-1])))
    return A, B


@pytest.mark.parametrize("kw", [dict(), dict(tiny_max=0), dict(validate=0)])
def test_micro_and_tiny_rows(kw):
    """Rows around the micro/tiny boundary (nnz(A_i) from 0 to 12, B rows of 0-3 entries over
    300 columns, so heads collide often and some rows exceed 32 products)."""
    A, B = _short_rows(4000, 5000, 300, lambda i: i % 13, 3, seed=40)
    rp, col, val, _, info, _ = run_gpu(A, B, opts=opts(general_path=1, **kw))
    assert_parity(A, B, rp, col, val)
    if not kw:
        import paper_2004_13907_gb300 as sp
        cls = dict(zip(sp._native.NUM_CLASSES, info["num_class_rows"]))
        assert cls["micro"] > 0 and cls["tiny"] > 0


def test_identity_exact():
    A = synth.uniform_random(3000, 2500, 3e-3, seed=15)
    I = synth.identity(2500)
    rp, col, val, *_ = run_gpu(A, I)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col) and np.array_equal(val, A.val)
    I3 = synth.identity(3000)
    rp, col, val, *_ = run_gpu(I3, A)
    assert np.array_equal(rp, A.row_ptr) and np.array_equal(col, A.col) and np.array_equal(val, A.val)


def test_cancellation_and_stored_zeros():
    A = synth.from_dense(np.array([[1.0, 1.0], [0.0, 2.0]]), pattern=np.array([[True, True], [True, True]]))
    B = synth.from_dense(np.array([[1.0, 3.0], [-1.0, 0.0]]), pattern=np.array([[True, False], [True, True]]))
    rp, col, val, *_ = run_gpu(A, B)
    assert list(rp) == [0, 2, 4]
    assert list(col) == [0, 1, 0, 1]
    assert list(val) == [0.0, 0.0, -2.0, 0.0]


@pytest.mark.parametrize("m,k,n", [(0, 0, 0), (0, 5, 7), (6, 0, 4), (5, 4, 0), (1, 1, 1), (3, 4, 2)])
def test_degenerate_shapes(m, k, n):
    A = synth.random_small(m, k, 0.6, seed=16)
    B = synth.random_small(k, n, 0.6, seed=17)
    rp, col, val, *_ = run_gpu(A, B)
    assert_parity(A, B, rp, col, val)


def test_empty_rows_mixed_with_heavy_rows():
    D = np.zeros((64, 50_000))
    rng = np.random.default_rng(0)
    for i in (3, 40):
        D[i, rng.choice(50_000, 9000, replace=False)] = rng.uniform(-1, 1, 9000)
    A = synth.from_dense(np.eye(64)[:, :64])
    B = synth.from_dense(D)
    rp, col, val, *_ = run_gpu(A, B)
    assert_parity(A, B, rp, col, val)


def test_invalid_csr_is_reported():
    """The general path reports invalid inputs at the plan (the small-product path, which plans
    without a host read, reports them at the symbolic pass: tests/test_gpu_small.py)."""
    import paper_2004_13907_gb300 as sp

    def plan(a, b):
        return sp.spgemm_plan(a, b, opts=sp.spgemm_opts_default(general_path=1))

    A = synth.uniform_random(50, 50, 0.1, seed=18)
    col = A.col.copy()
    r = int(np.argmax(np.diff(A.row_ptr) >= 2))
    s = A.row_ptr[r]
    col[s], col[s + 1] = col[s + 1], col[s]          # unsorted row
    bad = synth.CSR(A.rows, A.cols, A.row_ptr, col, A.val)
    dA = sp.DeviceCSR.from_host(bad, "cuda")
    with pytest.raises(sp.SpgemmError) as ei:
        plan(dA, dA)
    assert ei.value.name == "INVALID_CSR"
    col2 = A.col.copy()
    col2[0] = 50                                     # out of range
    dA = sp.DeviceCSR.from_host(synth.CSR(A.rows, A.cols, A.row_ptr, col2, A.val), "cuda")
    with pytest.raises(sp.SpgemmError) as ei:
        plan(dA, dA)
    assert ei.value.name == "INVALID_CSR"
    col3 = A.col.copy()
    col3[s + 1] = col3[s]                            # repeated column in a row
    dA = sp.DeviceCSR.from_host(synth.CSR(A.rows, A.cols, A.row_ptr, col3, A.val), "cuda")
    with pytest.raises(sp.SpgemmError) as ei:
        plan(dA, dA)
    assert ei.value.name == "INVALID_CSR"
    rp4 = A.row_ptr.copy()
    rp4[r + 1], rp4[r + 2] = rp4[r + 2], rp4[r + 1]  # decreasing row pointers (inside [0, nnz])
    if rp4[r + 1] != rp4[r + 2]:
        dA = sp.DeviceCSR.from_host(synth.CSR(A.rows, A.cols, rp4, A.col, A.val), "cuda")
        with pytest.raises(sp.SpgemmError) as ei:
            plan(dA, dA)
        assert ei.value.name == "INVALID_CSR"
    # a valid matrix whose rows start below the previous row's last column passes
    ok = synth.CSR(3, 6, np.array([0, 2, 3, 5]), np.array([3, 5, 0, 1, 4], dtype=np.int32), np.ones(5))
    sp.spgemm_plan_destroy(plan(sp.DeviceCSR.from_host(ok, "cuda"),
                                sp.DeviceCSR.from_host(synth.identity(6), "cuda")))


def test_host_entry_matches_oracle():
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(4000, 4000, 2e-3, seed=19)
    hA = sp.DeviceCSR(A.rows, A.cols, torch.from_numpy(A.row_ptr.astype(np.int32)).pin_memory(),
                      torch.from_numpy(A.col).pin_memory(), torch.from_numpy(A.val).pin_memory())
    C = sp.spgemm_multiply_host(hA, hA)
    rp = C.row_ptr.numpy().astype(np.int64)
    assert_parity(A, A, rp, C.col.numpy(), C.val.numpy())
    # reuse of the grown buffers
    C2 = sp.spgemm_multiply_host(hA, hA, out=C)
    assert np.array_equal(C2.col.numpy(), C.col.numpy())


def test_repeat_numeric_on_plan_and_changed_values():
    """The plan can be re-used for a new numeric pass when the values change."""
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(3000, 3000, 3e-3, seed=20)
    dA = sp.DeviceCSR.from_host(A, "cuda")
    plan = sp.spgemm_plan(dA, dA)
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan)
    sp.spgemm_numeric(plan, C)
    dA.val.mul_(2.0)
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    A2 = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, A.val * 2.0)
    H = C.to_host()
    assert_parity(A2, A2, H.row_ptr.numpy().astype(np.int64), H.col.numpy(), H.val.numpy())


@pytest.mark.slow
def test_rmat_2e20_every_row(capsys):
    """The R-MAT 2^20 / degree-16 config at full size (9.7e9 entries of C), in the bench's launch
    configuration: EVERY row against the oracle, streamed in row panels (structure bit-exact,
    values within 1e-12 * sum|a*b|)."""
    A = synth.rmat(20, 16, seed=0)
    import paper_2004_13907_gb300 as sp
    dA = sp.DeviceCSR.from_host(A, "cuda")
    plan = sp.spgemm_plan(dA, dA, opts=sp.spgemm_opts_default())
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan)
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    info = sp.spgemm_plan_get_info(plan)
    torch.cuda.synchronize()
    assert info["products"] == int(oracle.products_per_row(A, A).sum())
    worst = [0.0, 0]

    def check(ref, rp, col, val, r0, r1):
        assert np.array_equal(rp, ref.row_ptr), f"row offsets differ in rows [{r0}, {r1})"
        assert np.array_equal(col, ref.col), f"columns differ in rows [{r0}, {r1})"
        err = np.abs(val - ref.val)
        bad = err > 1e-12 * ref.mag
        assert not bad.any(), f"{int(bad.sum())} values out of tolerance in rows [{r0}, {r1})"
        nz = ref.mag > 0
        if nz.any():
            worst[0] = max(worst[0], float((err[nz] / ref.mag[nz]).max()))
        worst[1] += len(col)

    panels = compare_all_rows(A, A, C, check)
    assert worst[1] == info["nnz_c"]
    with capsys.disabled():
        print(f"\nR-MAT 2^20 FP64: all {A.rows} rows, {worst[1]} entries in {panels} panels match the oracle; "
              f"max |c - c_ref| / sum|p| = {worst[0]:.3e}")
    sp.spgemm_plan_destroy(plan)
    del C
    torch.cuda.empty_cache()


@pytest.mark.parametrize("accumulate", [0, 1])
def test_rmat_2e17_full_default_config(accumulate):
    """R-MAT 2^17 / degree 16 in the default launch configuration: every windowed sub-class,
    rows with more than 512 A entries among them, compared element by element (FP64 atomics and
    the exact fixed-point mode)."""
    import paper_2004_13907_gb300 as sp
    A = synth.rmat(17, 16, seed=0)
    dA = sp.DeviceCSR.from_host(A, "cuda")
    plan = sp.spgemm_plan(dA, dA, opts=sp.spgemm_opts_default(fp64_accumulate=accumulate))
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan)
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    info = sp.spgemm_plan_get_info(plan)
    torch.cuda.synchronize()
    cls = dict(zip(sp._native.NUM_CLASSES, info["num_class_rows"]))
    assert all(cls[c] > 0 for c in ("win1", "win2", "win3", "block8192", "warp1024"))
    assert int(np.diff(A.row_ptr).max()) > 512
    seen = [0]

    def check(ref, rp, col, val, r0, r1):
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col), f"rows [{r0}, {r1})"
        assert np.all(np.abs(val - ref.val) <= 1e-12 * ref.mag), f"values in rows [{r0}, {r1})"
        seen[0] += len(col)

    compare_all_rows(A, A, C, check)
    assert seen[0] == info["nnz_c"]
    sp.spgemm_plan_destroy(plan)


@pytest.mark.parametrize("g", [8, 96, 1024])
def test_galerkin_triple_product(g):
    """Multigrid coarse operator R*(A*P) with 2x2 aggregation on the 2D Laplacian, as two library
    products (the second takes the first's device output as its B): A*P matches the oracle and
    R*(A*P) is exactly 2 x the coarse 5-point Laplacian; then the values of A change and both
    numeric passes rerun on their plans."""
    import paper_2004_13907_gb300 as sp
    A = synth.laplacian2d(g)
    P = synth.aggregation_prolongator(g)
    R = synth.aggregation_restrictor(g)
    dA, dP, dR = (sp.DeviceCSR.from_host(M, "cuda") for M in (A, P, R))
    p1 = sp.spgemm_plan(dA, dP)
    sp.spgemm_symbolic(p1)
    AP = sp.alloc_output(p1)
    sp.spgemm_numeric(p1, AP)
    p2 = sp.spgemm_plan(dR, AP)
    sp.spgemm_symbolic(p2)
    Ac = sp.alloc_output(p2)
    sp.spgemm_numeric(p2, Ac)
    sp.spgemm_plan_check(p1)
    sp.spgemm_plan_check(p2)
    H = AP.to_host()
    assert_parity(A, P, H.row_ptr.numpy().astype(np.int64), H.col.numpy(), H.val.numpy())
    L = synth.laplacian2d(g // 2)
    Hc = Ac.to_host()
    assert np.array_equal(Hc.row_ptr.numpy().astype(np.int64), L.row_ptr)
    assert np.array_equal(Hc.col.numpy(), L.col)
    assert np.array_equal(Hc.val.numpy(), 2.0 * L.val)
    # plan reuse: A scaled by 3 in place (same pattern), both numeric passes again
    dA.val.mul_(3.0)
    sp.spgemm_numeric(p1, AP)
    sp.spgemm_numeric(p2, Ac)
    sp.spgemm_plan_check(p2)
    assert np.array_equal(Ac.val.cpu().numpy(), 6.0 * L.val)
    sp.spgemm_plan_destroy(p1)
    sp.spgemm_plan_destroy(p2)


@pytest.mark.parametrize("panels,idx64", [(2, False), (5, True), (64, False)])
def test_host_entry_in_row_panels(panels, idx64):
    """spgemm_multiply_host in row panels of A (each multiplied while the previous panels' C is
    copied back on a second stream): the same C as the oracle, with int32 or int64 row pointers,
    and a capacity too small reports nnz(C) for a second call."""
    import paper_2004_13907_gb300 as sp
    for A in (synth.uniform_random(3000, 2500, 3e-3, seed=21), synth.rmat(12, 16, seed=22)):
        B = A if A.rows == A.cols else synth.uniform_random(A.cols, 1800, 4e-3, seed=23)
        pin = lambda M: sp.DeviceCSR(M.rows, M.cols, torch.from_numpy(M.row_ptr.astype(np.int32)).pin_memory(),
                                     torch.from_numpy(M.col).pin_memory(), torch.from_numpy(M.val).pin_memory())
        o = opts(host_panels=panels)
        C = sp.spgemm_multiply_host(pin(A), pin(B), opts=o, idx64=idx64)
        assert C.row_ptr.dtype == (torch.int64 if idx64 else torch.int32)
        assert_parity(A, B, C.row_ptr.numpy().astype(np.int64), C.col.numpy(), C.val.numpy())
        ref = oracle.spgemm(A, B)
        small = sp.DeviceCSR(A.rows, B.cols, torch.empty(A.rows + 1, dtype=torch.int32).pin_memory(),
                             torch.empty(max(ref.nnz // 2, 1), dtype=torch.int32).pin_memory(),
                             torch.empty(max(ref.nnz // 2, 1), dtype=torch.float64).pin_memory())
        C2 = sp.spgemm_multiply_host(pin(A), pin(B), opts=o, out=small)
        assert np.array_equal(C2.col.numpy(), ref.col)


def test_host_entry_default_panels_on_a_large_product():
    """spgemm_multiply_host with default options on a product large enough to run in the default
    row panels (A's entries times B's mean row length above 1e8): every row against the oracle."""
    import paper_2004_13907_gb300 as sp
    A = synth.uniform_random(260_000, 260_000, 8e-5, seed=24)
    assert A.nnz * (A.nnz / A.rows) > 1e8
    hA = sp.DeviceCSR(A.rows, A.cols, torch.from_numpy(A.row_ptr.astype(np.int32)).pin_memory(),
                      torch.from_numpy(A.col).pin_memory(), torch.from_numpy(A.val).pin_memory())
    C = sp.spgemm_multiply_host(hA, hA)
    seen = [0]

    def check(ref, rp, col, val, r0, r1):
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col), f"rows [{r0}, {r1})"
        assert np.all(np.abs(val - ref.val) <= 1e-12 * ref.mag), f"values in rows [{r0}, {r1})"
        seen[0] += len(col)

    compare_all_rows(A, A, C, check)
    assert seen[0] == C.nnz


def test_stage_timings_per_plan_with_reused_events():
    """record_timings: every stage a plan ran reports a positive device time and its launches,
    the small-product path none of the general path's stages, and plans made one after another
    (whose timing events come back to a shared pool) each their own. Without the option nothing
    is recorded."""
    import paper_2004_13907_gb300 as sp
    big = synth.rmat(12, 16, seed=25)                    # general row classes
    small = synth.uniform_random(2000, 2000, 2e-3, seed=26)   # small-product path
    for rep in range(3):
        for M, expect in ((big, {"count", "num_rowptr"}), (small, {"sym_warp", "num_warp"})):
            dM = sp.DeviceCSR.from_host(M, "cuda")
            plan = sp.spgemm_plan(dM, dM, opts=opts(record_timings=1))
            sp.spgemm_symbolic(plan)
            C = sp.alloc_output(plan)
            sp.spgemm_numeric(plan, C)
            t = sp.spgemm_plan_get_timings(plan)
            ran = {k for k, (ms, nl) in t.items() if nl > 0}
            assert expect <= ran, (expect, t)
            assert all(ms > 0 for k, (ms, nl) in t.items() if k in ran)
            if M is small:
                assert not ran & {"count", "num_rowptr", "num_window"}
            sp.spgemm_plan_destroy(plan)
    dM = sp.DeviceCSR.from_host(small, "cuda")
    plan = sp.spgemm_plan(dM, dM)
    sp.spgemm_symbolic(plan)
    assert all(ms == 0 and nl == 0 for ms, nl in sp.spgemm_plan_get_timings(plan).values())
    sp.spgemm_plan_destroy(plan)
