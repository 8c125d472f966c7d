"""The C-ABI library builds, loads and exports every symbol include/*.h declares, and the
ctypes mirrors of its structs have the C layout (no GPU needed, no compute call)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_13907_gb300 import build
    from paper_2004_13907_gb300 import _native
    build.build()
    return _native.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(spgemm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"


def test_ctypes_signatures_cover_header():
    from paper_2004_13907_gb300 import _native
    assert set(_declared_functions()) == set(_native.SIGNATURES)


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.spgemm_version()
    assert lib.spgemm_last_error() is not None


def test_struct_layout_matches_c(tmp_path):
    from paper_2004_13907_gb300 import _native
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "spgemm.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(spgemm_csr_in),"
        " sizeof(spgemm_csr_out), sizeof(spgemm_allocator), sizeof(spgemm_opts),"
        " sizeof(spgemm_plan_info), offsetof(spgemm_opts, rowptr32_limit),"
        " offsetof(spgemm_plan_info, workspace_bytes), sizeof(spgemm_server_cfg),"
        " offsetof(spgemm_server_cfg, opts), sizeof(spgemm_job_info), sizeof(spgemm_server_stats),"
        " offsetof(spgemm_server_stats, latency_p50_ms)); printf(\"%zu %zu\\n\", sizeof(spgemm_tune_report),"
        " offsetof(spgemm_tune_report, trial_window_fill)); return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(_native.CsrIn), ctypes.sizeof(_native.CsrOut), ctypes.sizeof(_native.Allocator),
            ctypes.sizeof(_native.Opts), ctypes.sizeof(_native.PlanInfo),
            _native.Opts.rowptr32_limit.offset, _native.PlanInfo.workspace_bytes.offset,
            ctypes.sizeof(_native.ServerCfg), _native.ServerCfg.opts.offset, ctypes.sizeof(_native.JobInfo),
            ctypes.sizeof(_native.ServerStats), _native.ServerStats.latency_p50_ms.offset,
            ctypes.sizeof(_native.TuneReport), _native.TuneReport.trial_window_fill.offset]
    assert got == want


def test_opts_default_without_gpu(lib):
    from paper_2004_13907_gb300 import _native
    o = _native.Opts()
    lib.spgemm_opts_default(ctypes.byref(o))
    assert o.validate == 1 and o.tiny_max == 32 and o.block_max == 2048
    assert o.rowptr32_limit == 2**31 - 1


def test_plan_rejects_bad_arguments_on_host(lib):
    """Argument checks happen on the host before any device work."""
    from paper_2004_13907_gb300 import _native
    h = ctypes.c_void_p()
    st = lib.spgemm_plan(None, None, 0, None, None, None, ctypes.byref(h))
    assert st == 1 and h.value is None
    a = _native.CsrIn(4, 5, 0, 0, 0, 1, 0, 0)
    b = _native.CsrIn(6, 3, 0, 0, 0, 1, 0, 0)
    st = lib.spgemm_plan(ctypes.byref(a), ctypes.byref(b), 0, None, None, None, ctypes.byref(h))
    assert st == 1 and b"A.cols" in lib.spgemm_last_error()
    bad = _native.CsrIn(-1, 5, 0, 0, 0, 1, 0, 0)
    st = lib.spgemm_plan(ctypes.byref(bad), ctypes.byref(a), 0, None, None, None, ctypes.byref(h))
    assert st == 1


def test_python_binding_fails_loudly_without_library(tmp_path):
    from paper_2004_13907_gb300 import _native
    with pytest.raises(ImportError):
        _native.load(str(tmp_path / "missing.so"))


def test_server_config_checks_on_host(lib):
    """Server defaults, and configurations refused before any device call."""
    from paper_2004_13907_gb300 import _native
    cfg = _native.ServerCfg()
    assert lib.spgemm_server_cfg_default(ctypes.byref(cfg)) == 0
    assert cfg.mem_cap_bytes == 32 << 30 and cfg.num_streams == 2 and cfg.prec == 0
    assert cfg.opts.validate == 1 and cfg.opts.window_hash_fill == 4096
    assert cfg.reserve_sms == 0 and cfg.opts.max_sms == 0
    assert cfg.small_products == 1 << 26 and cfg.max_defer_ms == 250 and cfg.host_panels == 1
    h = ctypes.c_void_p()
    for field, bad in [("num_streams", 0), ("num_streams", 9), ("mem_cap_bytes", 0), ("max_batch_jobs", 0),
                       ("prec", 7), ("batch_window_us", -1), ("reserve_sms", -1), ("small_products", -1), ("max_defer_ms", -1)]:
        c = _native.ServerCfg()
        lib.spgemm_server_cfg_default(ctypes.byref(c))
        setattr(c, field, bad)
        assert lib.spgemm_server_create(ctypes.byref(c), ctypes.byref(h)) == 1, field
        assert h.value is None
    job = ctypes.c_int64()
    a = _native.CsrIn(4, 5, 0, 0, 0, 1, 0, 0)
    assert lib.spgemm_server_submit(None, ctypes.byref(a), ctypes.byref(a), ctypes.byref(job)) == 1
    lib.spgemm_server_wait_any.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
    assert lib.spgemm_server_wait_any(None, 0.0, ctypes.byref(job)) == 1
    assert lib.spgemm_server_destroy(None) == 0
