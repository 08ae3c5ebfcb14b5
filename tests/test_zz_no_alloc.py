"""clb_nusselt_noalloc: the Nusselt number for callers that cannot allocate device memory (for
example a monitor in a server whose HBM is already committed to resident lattices, or a loop that
must not let cudaMalloc/cudaFree synchronise the device). It uses a fixed scratch array that the
library keeps in device memory, and must agree with clb_nusselt, which works through a handle and
its own scratch. Called through the C ABI, twice in a row on the same state and once more after
stepping, so that a stale result left in the shared array would show; on halfway and wet walls and
on rows wider than the handle's 2048-node diagnostics segments; and once directly against the
oracle."""
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


def problem(kind, storage):
    if kind == "cavity":
        return W.cavity(96, Ra=1e4, ny=80, storage=storage)
    if kind == "rb":
        return W.rayleigh_benard(130, 61, Ra=5e3, storage=storage)
    if kind == "wet":
        # the paper's own walls: wall rows at half weight in the average, H = ny - 1
        return W.rayleigh_benard_table1(5000.0, storage=storage, wet=True)
    # rows wider than one 2048-node segment of the handle's diagnostics pass, which then sums
    # each row in several partials: equal within rounding, not bitwise
    return W.rayleigh_benard(4100, 8, Ra=2e3, storage=storage)


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("kind", ["cavity", "rb", "wet", "wide"])
def test_noalloc_nusselt_equals_handle_nusselt(clb, storage, kind):
    prob = problem(kind, storage)
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
    lat.close()


def test_noalloc_nusselt_matches_the_oracle(clb):
    """Directly against the oracle's Eq. 29 on the oracle's own fields (FP64 storage)."""
    import oracle
    prob = W.cavity(40, Ra=2e4, ny=32, storage=F64)
    lat = clb.Lattice.from_problem(prob)
    lat.step(150)
    ref = oracle.Oracle.from_problem(prob)
    ref.step(150)
    _, ux, uy, T = ref.fields()
    expect = oracle.nusselt(ux, uy, T, prob.params, prob.nu_axis)
    assert noalloc_nusselt(clb, lat, prob) == pytest.approx(expect, rel=1e-11, abs=1e-13)
    lat.close()


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
