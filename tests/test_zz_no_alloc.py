"""clb_nusselt_noalloc: the Nusselt number for callers that cannot allocate device memory (for
example a monitor in a server whose HBM is already committed to resident lattices, or a loop that
must not let cudaMalloc/cudaFree synchronise the device). It uses a fixed scratch array that the
library keeps in device memory, and must agree with clb_nusselt, which works through a handle and
its own scratch. Called through the C ABI, twice in a row on the same state and once more after
stepping, so that a stale result left in the shared array would show."""
import ctypes

import pytest

from paper_1710_10569_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64, F32, F16 = W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def noalloc_nusselt(clb, lat, prob):
    cur, _, _, _ = lat.buffers()
    p = clb.params(prob.params)
    out = ctypes.c_double()
    st = clb.lib().clb_nusselt_noalloc(ctypes.c_void_p(cur), prob.nx, prob.ny, ctypes.byref(p),
                                       prob.nu_axis, ctypes.c_void_p(lat.stream), ctypes.byref(out))
    assert st == clb.CLB_OK, clb.lib().clb_last_error()
    return out.value


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("kind", ["cavity", "rb"])
def test_noalloc_nusselt_equals_handle_nusselt(clb, storage, kind):
    if kind == "cavity":
        prob = W.cavity(96, Ra=1e4, ny=80, storage=storage)
    else:
        prob = W.rayleigh_benard(130, 61, Ra=5e3, storage=storage)
    lat = clb.Lattice.from_problem(prob)
    lat.step(300)
    expect = lat.nusselt(prob.nu_axis)
    first = noalloc_nusselt(clb, lat, prob)
    second = noalloc_nusselt(clb, lat, prob)
    assert first == pytest.approx(expect, rel=1e-12, abs=1e-14)
    assert second == pytest.approx(expect, rel=1e-12, abs=1e-14)
    lat.step(200)
    expect2 = lat.nusselt(prob.nu_axis)
    assert expect2 != expect
    assert noalloc_nusselt(clb, lat, prob) == pytest.approx(expect2, rel=1e-12, abs=1e-14)


def test_noalloc_rejects_lattices_beyond_the_fixed_scratch(clb):
    L = clb.lib()
    rows = 8192 + 1
    p = clb.params(W.default_params())
    out = ctypes.c_double(-1.0)
    st = L.clb_nusselt_noalloc(ctypes.c_void_p(256), 4, rows, ctypes.byref(p), 1, None,
                               ctypes.byref(out))
    assert st == clb.CLB_EINVAL
    assert b"8192" in L.clb_last_error()
    assert out.value == -1.0
