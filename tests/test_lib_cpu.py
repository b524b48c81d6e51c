"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/wave.h declares, and its host-only entry points validate arguments
and compute what they state (no GPU work is issued here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_15744_gb300 import build
    build.build()
    return C.CDLL(build.LIB)


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "wave.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("wave_model_create", "wave_forward", "wave_adjoint_sensitivity", "misfit"):
        assert n in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_cfl_dt_matches_oracle(lib):
    import oracle as O
    f = lib.wave_cfl_dt
    f.restype = C.c_double
    f.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double]
    for nd in (2, 3):
        for order in (2, 4, 6, 8):
            got = f(nd, order, 10.0, 4500.0, 0.5)
            assert abs(got - O.cfl_dt(10.0, 4500.0, nd, order, 0.5)) < 1e-15 * got
    assert f(2, 5, 10.0, 4500.0, 0.5) == 0.0
    assert f(4, 2, 10.0, 4500.0, 0.5) == 0.0


def test_status_strings(lib):
    f = lib.wave_status_string
    f.restype = C.c_char_p
    f.argtypes = [C.c_int]
    seen = {f(i).decode() for i in range(8)}
    assert len(seen) == 8 and "ok" in seen
    assert f(99).decode() == "unknown status"


def test_host_validation_rejects_bad_descriptors(lib):
    from paper_2509_15744_gb300 import wave as W

    def ws(**kw):
        d = W.GridDesc()
        d.ndim, d.order = kw.get("ndim", 2), kw.get("order", 2)
        n = kw.get("n", (64, 64, 1))
        for i in range(3):
            d.n[i] = n[i]
        d.h, d.dt = kw.get("h", 10.0), kw.get("dt", 1e-3)
        d.physics, d.bc, d.storage = kw.get("physics", 0), kw.get("bc", 0), kw.get("storage", 0)
        size = C.c_size_t(0)
        st = W._model_ws(C.byref(d), C.byref(size))
        return st, size.value

    st, size = ws()
    assert st == 0 and size >= 128 * 64 * 4
    assert ws(order=3)[0] == 1
    assert ws(ndim=4)[0] == 1
    assert ws(n=(8, 64, 1), order=8)[0] == 1          # fewer than order + 1 cells
    assert ws(n=(9, 9, 1), order=8)[0] == 0           # the minimum is accepted
    assert ws(n=(64, 64, 2))[0] == 1                  # 2D needs nz = 1
    assert ws(h=0.0)[0] == 1
    assert ws(physics=1, order=4)[0] == 1             # density is second order
    assert ws(storage=7)[0] == 1
    # 3D pitched size: rows rounded up to 128 cells
    st, size = ws(ndim=3, n=(130, 10, 11), order=4)
    assert st == 0 and size >= 256 * 10 * 11 * 4


def test_model_create_rejects_null_param_without_touching_the_gpu(lib):
    from paper_2509_15744_gb300 import wave as W
    d = W.GridDesc()
    d.ndim, d.order = 2, 2
    d.n[0], d.n[1], d.n[2] = 64, 64, 1
    d.h, d.dt = 10.0, 1e-3
    h = C.c_void_p()
    assert W._model_create(C.byref(d), None, None, 0, None, C.byref(h)) == 1


def test_workloads_are_deterministic():
    from paper_2509_15744_gb300 import workloads as WL
    a = WL.workload0()
    b = WL.workload0()
    assert (a.init_param == b.init_param).all() and (a.true_param == b.true_param).all()
    w2 = WL.workload2(n=64, nshots=16)
    assert w2.nshots == 16 and len(set(w2.sources)) == 16
    assert all(1500 <= n <= 2500 for n in w2.nt)
    assert w2.receivers[0].size == 32 * 32
    import oracle as O
    # the stated time step of workload 0 is half the 2D second-order limit
    assert abs(O.cfl_dt(a.h, a.vmax, 2, 2, a.cfl_fraction) - 0.5 * 10 / (3000 * 2 ** 0.5)) < 1e-15


def test_plain_c_client_links_and_runs_the_host_checks(lib, tmp_path):
    # The boundary is usable from C99 alone: tests/c_abi/host_check.c includes
    # only wave.h, links libwave, and calls its host-side entry points.
    import shutil
    import subprocess
    from paper_2509_15744_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "host_check"
    libdir = os.path.dirname(build.LIB)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi", "host_check.c"), "-o", str(exe),
                    "-L", libdir, "-l:libwave.so", f"-Wl,-rpath,{libdir}", "-lm"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout


def test_workspace_checks_happen_before_any_device_work(lib):
    # An undersized or misaligned caller workspace is refused on the host
    # (WAVE_EWORKSPACE = 3) before anything touches the GPU; the pointers are
    # never dereferenced, so fake addresses serve.
    from paper_2509_15744_gb300 import wave as W
    d = W.GridDesc()
    d.ndim, d.order = 3, 8
    d.n[0], d.n[1], d.n[2] = 130, 20, 21
    d.h, d.dt = 10.0, W.cfl_dt(3, 8, 10.0, 4500.0, 0.5)
    need = C.c_size_t(0)
    assert W._model_ws(C.byref(d), C.byref(need)) == 0
    param = C.c_void_p(0x10000)
    h = C.c_void_p()
    aligned = C.c_void_p(0x7f0000000000)
    assert W._model_create(C.byref(d), param, C.c_void_p(0x7f0000000000 + 8), need.value, None,
                           C.byref(h)) == 3                  # not 256-byte aligned
    assert W._model_create(C.byref(d), param, aligned, need.value - 1, None, C.byref(h)) == 3   # one byte short
    assert not h.value
    # misfit: scratch smaller than wave_misfit_scratch_size(count), or misaligned
    n = 1 << 20
    small = W._misfit_scratch(n) - 8
    out = C.c_void_p(0x20000)
    assert W._misfit(C.c_void_p(0x30000), None, n, 1.0, 1.0, out, aligned, small, None) == 3
    assert W._misfit(C.c_void_p(0x30000), None, n, 1.0, 1.0, out, C.c_void_p(0x7f0000000004),
                     W._misfit_scratch(n), None) == 3


def test_metrics_calls_validate_on_the_host(lib):
    from paper_2509_15744_gb300 import wave as W
    m = W.GradMetrics()
    assert W._metrics_read(None, C.byref(m)) == 1
    assert W._set_metrics(None, 1) == 1
    assert W._model_set_param(None, None, None) == 1


def test_schedule_setter_validates_on_the_host(lib):
    # a null model is rejected before anything else is looked at
    assert lib.wave_model_set_schedule(None, 1) == 1
    assert lib.wave_model_set_schedule(None, 0) == 1
