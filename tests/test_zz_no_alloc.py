"""The allocation-free misfit entry point (wave_misfit_static).

Some callers cannot allocate device memory at the point where they need the
misfit (a plugin whose host framework owns all device memory, a loop that
must not enter an allocator).  wave_misfit_static serves them with scratch
that lives in the library itself.  This test calls it through the C ABI and
checks it against the scratch-taking `misfit` entry point on two calls in a
row -- the second smaller than the first, so partial sums left over from the
first call must not leak into the second -- and checks that a count beyond
the static scratch is refused.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MAX_COUNT = 4096 * 8192   # samples the static scratch can reduce (include/wave.h)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2509_15744_gb300 import build
    L = C.CDLL(build.LIB)
    f = L.wave_misfit_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p]
    m = L.misfit
    m.restype = C.c_int
    m.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                  C.c_size_t, C.c_void_p]
    s = L.wave_misfit_scratch_size
    s.restype = C.c_size_t
    s.argtypes = [C.c_int64]
    return L


def _ref(lib, syn, obs, dt, w, stream):
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    scratch = torch.empty(max(1, lib.wave_misfit_scratch_size(syn.numel())), dtype=torch.uint8, device="cuda")
    st = lib.misfit(syn.data_ptr(), obs.data_ptr() if obs is not None else None, syn.numel(), dt, w,
                    out.data_ptr(), scratch.data_ptr(), scratch.numel(), stream)
    assert st == 0
    return out


def test_static_scratch_misfit_matches_misfit(lib):
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(5_000_003, True, 0.25, 1.0), (70_001, False, 0.5, -2.0 / 3.0)]
    for n, with_obs, dt, w in cases:    # two calls in a row, the second smaller
        syn = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        obs = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() if with_obs else None
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.wave_misfit_static(syn.data_ptr(), obs.data_ptr() if obs is not None else None, n, dt, w,
                                    out.data_ptr(), stream)
        assert st == 0
        ref = _ref(lib, syn, obs, dt, w, stream)
        torch.cuda.synchronize()
        a, b = float(out.item()), float(ref.item())
        assert abs(a - b) <= 1e-12 * abs(b), (a, b)


def test_static_scratch_misfit_limits(lib):
    stream = torch.cuda.current_stream().cuda_stream
    syn = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.full((1,), 1.0, dtype=torch.float64, device="cuda")
    # beyond the static scratch: refused on the host, nothing launched
    assert lib.wave_misfit_static(syn.data_ptr(), None, MAX_COUNT + 1, 1.0, 1.0, out.data_ptr(), stream) == 1
    # empty input gives zero
    assert lib.wave_misfit_static(None, None, 0, 1.0, 1.0, out.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
