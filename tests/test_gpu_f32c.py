"""FP32-compensated path vs the FP64 oracle (FP32 inputs, FP32 output).

Each value is either a compensated FP32 sum (error-free product with fmaf, two-sum
accumulation: Ogita, Rump and Oishi's Dot2) that passed its error bound, or, for a row with
an entry over that bound, the FP64 sum rounded once to FP32. So every entry must satisfy
|c_gpu - c| <= 2u|c| + (FP64 rounding), u = 2^-24, against the exact sum c (the FP64 oracle on
the same FP32 inputs, whose products are exact in FP64). With the rerun switched off, every
entry must still meet Dot2's published bound u|c| + gamma_t^2 * sum|p|. The structure is
bit-exact as in FP64.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import compare_all_rows, gpu_or_skip, run_gpu

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(autouse=True)
def _gpu():
    gpu_or_skip()


def opts(**kw):
    import paper_2004_13907_gb300 as sp
    return sp.spgemm_opts_default(**kw)


def _f32(M):
    return M.astype(np.float32)


def _check(A, B, rp, col, val, bound="final"):
    ref = oracle.spgemm(A, B)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    err = np.abs(val.astype(np.float64) - ref.val)
    if bound == "final":
        lim = 2.001 * U32 * np.abs(ref.val) + 2e-12 * ref.mag
    else:   # Dot2 bound for every entry
        t = ref.terms.astype(np.float64)
        g = t * U32 / (1 - t * U32)
        lim = 1.001 * U32 * np.abs(ref.val) + g * g * ref.mag * 1.001 + 1e-30
    bad = err > lim
    assert not bad.any(), f"{bad.sum()} entries over the bound; worst excess {(err - lim).max()}"
    rel = err / np.maximum(np.abs(ref.val), 1e-300)
    return float(rel[np.abs(ref.val) > 0].max()) if ref.nnz else 0.0


@pytest.mark.parametrize("scale", [10, 14])
def test_rmat_f32c(scale):
    A = _f32(synth.rmat(scale, 16, seed=41))
    rp, col, val, _, info, _ = run_gpu(A, A, prec="f32c")
    _check(A, A, rp, col, val)


def test_uniform_signed_f32c_and_tiny_rows():
    A = _f32(synth.uniform_random(4000, 4000, 2e-3, seed=42))
    rp, col, val, _, info, _ = run_gpu(A, A, prec="f32c")
    _check(A, A, rp, col, val)
    L = _f32(synth.laplacian2d(100))
    rp, col, val, _, info, _ = run_gpu(L, L, prec="f32c")
    _check(L, L, rp, col, val)


@pytest.mark.parametrize("A_kind", ["rmat", "uniform"])
def test_rerun_off_meets_dot2_bound(A_kind):
    A = _f32(synth.rmat(13, 16, seed=43) if A_kind == "rmat" else
             synth.uniform_random(3000, 3000, 5e-3, seed=44))
    rp, col, val, _, info, _ = run_gpu(A, A, prec="f32c", opts=opts(f32c_rerun_none=1))
    assert info["f32c_rerun_rows"] == 0
    _check(A, A, rp, col, val, bound="dot2")


def test_cancellation_forces_rerun():
    """Rows whose products cancel (to exactly 0, or to a tiny remainder) exceed the compensated
    bound and are recomputed in FP64; rows without cancellation are not."""
    rng = np.random.default_rng(0)
    m, n = 400, 3000
    A = np.zeros((m, 2 * m))
    Bd = np.zeros((2 * m, n))
    for i in range(m):
        A[i, 2 * i] = A[i, 2 * i + 1] = 1.0
        cols = rng.choice(n, 12, replace=False)
        v = rng.uniform(0.5, 1.0, 12).astype(np.float32).astype(np.float64)
        Bd[2 * i, cols] = v
        if i % 2 == 0:     # cancelling rows: exact zero or a 2^-20 remainder
            Bd[2 * i + 1, cols] = -v
            Bd[2 * i + 1, cols[0]] = -v[0] + 2.0 ** -20
        else:              # plain rows: same sign, no cancellation
            Bd[2 * i + 1, cols] = v
    pat_b = Bd != 0
    Af = synth.from_dense(A, dtype=np.float32)
    Bf = synth.from_dense(Bd, pattern=pat_b, dtype=np.float32)
    rp, col, val, _, info, _ = run_gpu(Af, Bf, prec="f32c")
    assert info["f32c_rerun_rows"] == m // 2
    _check(Af, Bf, rp, col, val)


def test_rerun_all_gives_rounded_fp64():
    A = _f32(synth.uniform_random(2000, 2000, 4e-3, seed=45))
    rp, col, val, _, info, _ = run_gpu(A, A, prec="f32c", opts=opts(f32c_rerun_all=1))
    assert info["f32c_rerun_rows"] == int(np.count_nonzero(np.diff(rp)))
    ref = oracle.spgemm(A, A)
    err = np.abs(val.astype(np.float64) - ref.val)
    assert np.all(err <= 1.0001 * U32 * np.abs(ref.val) + 2e-12 * ref.mag)


def test_forced_window_classes_f32c():
    A = _f32(synth.rmat(12, 16, seed=46))
    B = _f32(synth.uniform_random(A.cols, 5000, 2e-3, seed=47))
    rp, col, val, *_ = run_gpu(A, B, prec="f32c", opts=opts(force_window=1, window_hash_fill=1))
    _check(A, B, rp, col, val)


@pytest.mark.slow
def test_rmat_2e20_f32c_every_row_and_error_report(capsys):
    """The R-MAT 2^20 FP32 config at full size in its launch configuration: EVERY row against the
    FP64 oracle, streamed in row panels (structure bit-exact, each value within 2u|c| of the exact
    sum); prints the max relative entry error and the number of rows rerun in FP64."""
    import paper_2004_13907_gb300 as sp
    A = _f32(synth.rmat(20, 16, seed=0))
    dA = sp.DeviceCSR.from_host(A, "cuda", dtype=torch.float32)
    plan = sp.spgemm_plan(dA, dA, "f32c")
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan)
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    info = sp.spgemm_plan_get_info(plan)
    torch.cuda.synchronize()
    assert info["f32c_rerun_rows"] > 0
    worst = [0.0, 0]

    def check(ref, rp, col, val, r0, r1):
        assert np.array_equal(rp, ref.row_ptr), f"row offsets differ in rows [{r0}, {r1})"
        assert np.array_equal(col, ref.col), f"columns differ in rows [{r0}, {r1})"
        err = np.abs(val - ref.val)
        bad = err > 2.001 * U32 * np.abs(ref.val) + 2e-12 * ref.mag
        assert not bad.any(), f"{int(bad.sum())} values out of tolerance in rows [{r0}, {r1})"
        nz = np.abs(ref.val) > 0
        if nz.any():
            worst[0] = max(worst[0], float((err[nz] / np.abs(ref.val[nz])).max()))
        worst[1] += len(col)

    panels = compare_all_rows(A, A, C, check)
    assert worst[1] == info["nnz_c"]
    with capsys.disabled():
        print(f"\nR-MAT 2^20 FP32c: all {A.rows} rows, {worst[1]} entries in {panels} panels within 2u|c| of the "
              f"FP64 oracle; max rel err {worst[0]:.3e}; rows rerun in FP64: {info['f32c_rerun_rows']} of "
              f"{info['rows']}")
    sp.spgemm_plan_destroy(plan)
    del C
    torch.cuda.empty_cache()


def test_rmat_2e17_f32c_full():
    """R-MAT 2^17 FP32 in the default launch configuration, every entry against the FP64 oracle."""
    import paper_2004_13907_gb300 as sp
    A = _f32(synth.rmat(17, 16, seed=0))
    dA = sp.DeviceCSR.from_host(A, "cuda", dtype=torch.float32)
    plan = sp.spgemm_plan(dA, dA, "f32c")
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan)
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    torch.cuda.synchronize()

    def check(ref, rp, col, val, r0, r1):
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col), f"rows [{r0}, {r1})"
        err = np.abs(val - ref.val)
        assert np.all(err <= 2.001 * U32 * np.abs(ref.val) + 2e-12 * ref.mag), f"values in rows [{r0}, {r1})"

    compare_all_rows(A, A, C, check)
    sp.spgemm_plan_destroy(plan)


@pytest.mark.parametrize("t,sign,rerun", [(1000, 1.0, 0), (5000, 1.0, 1), (1000, -1.0, 0)])
def test_term_count_bound_of_nonnegative_products(t, sign, rerun):
    """With no negative value in A or B every partial product is non-negative, so the bound of an
    entry depends on its term count alone (about 4,000 terms at most); a value of either sign
    sends the kernel back to the bound with sum|p|. C = [[sum of t products]]."""
    import paper_2004_13907_gb300 as sp
    a = np.ones((1, t), dtype=np.float32)
    a[0, 7] = sign
    A = synth.from_dense(a).astype(np.float32)
    B = synth.from_dense(np.ones((t, 1), dtype=np.float32)).astype(np.float32)
    rp, col, val, _, info, _ = run_gpu(A, B, prec="f32c")
    assert info["f32c_rerun_rows"] == rerun
    assert val.tolist() == [float(t - 1 + sign)]
    _check(A, B, rp, col, val)


def test_sign_change_after_the_plan_reruns_hash_rows():
    """A plan made on non-negative values sends the short FP32 rows to the hash kernels, whose bound
    needs non-negative products. When a value turns negative before a later numeric pass, those
    rows are recomputed in FP64 and every entry still meets the final bound."""
    import paper_2004_13907_gb300 as sp
    A = _f32(synth.rmat(13, 16, seed=43))
    dA = sp.DeviceCSR.from_host(A, "cuda", dtype=torch.float32)
    plan = sp.spgemm_plan(dA, dA, "f32c")
    sp.spgemm_symbolic(plan)
    C = sp.alloc_output(plan)
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    info = sp.spgemm_plan_get_info(plan)
    cls = dict(zip(sp._native.NUM_CLASSES, info["num_class_rows"]))
    assert cls["block2048"] + cls["warp1024"] + cls["warp256"] > 0
    H = C.to_host()
    _check(A, A, H.row_ptr.numpy().astype(np.int64), H.col.numpy(), H.val.numpy())
    val = A.val.copy()
    val[::97] *= -1.0
    dA.val.copy_(torch.from_numpy(val))
    sp.spgemm_numeric(plan, C)
    sp.spgemm_plan_check(plan)
    reruns = sp.spgemm_plan_get_info(plan)["f32c_rerun_rows"]
    torch.cuda.synchronize()
    sp.spgemm_plan_destroy(plan)
    assert reruns >= cls["block8192"] + cls["block2048"] + cls["warp1024"] + cls["warp256"] + cls["warp64"]
    A2 = synth.CSR(A.rows, A.cols, A.row_ptr, A.col, val)
    H = C.to_host()
    _check(A2, A2, H.row_ptr.numpy().astype(np.int64), H.col.numpy(), H.val.numpy())
