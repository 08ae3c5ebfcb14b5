"""Out-of-bounds checks without a sanitizer: a lattice built in caller-owned device memory with a
guard region of a known byte pattern on each side, and the padding of every row's last chunk
filled with NaN, is stepped, reduced, read, autotuned and checkpointed. Afterwards the guards and the
padding must be unchanged (nothing writes outside the nodes), and every field must equal that of
the same lattice run without canaries (nothing reads the padding: a NaN read would spread)."""
import ctypes

import numpy as np
import pytest

from paper_1710_10569_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64, F32, F16 = W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV
GUARD = 1 << 20  # bytes on each side (a multiple of 512: the lattice's base stays aligned)
PATTERN = 0xA5


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def guarded_lattice(clb, prob):
    """A clb.Lattice whose memory sits between two guard regions of one torch allocation."""
    import torch
    lat = object.__new__(clb.Lattice)
    lat.nx, lat.ny, lat.params = prob.nx, prob.ny, dict(prob.params)
    lat._p = clb.params(prob.params)
    nb = ctypes.c_size_t()
    assert clb.lib().clb_footprint(lat.nx, lat.ny, ctypes.byref(lat._p), ctypes.byref(nb)) == clb.CLB_OK
    lat.footprint = nb.value
    lat._mem = torch.full((lat.footprint + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
    lat.stream = clb._stream_handle(None)
    h = ctypes.c_void_p()
    base = lat._mem.data_ptr() + GUARD
    assert clb.lib().clb_create(lat.nx, lat.ny, ctypes.byref(lat._p), lat.stream, ctypes.c_void_p(base),
                                lat.footprint, ctypes.byref(h)) == clb.CLB_OK
    lat._h = h
    lat.init_fields(prob.rho, prob.ux, prob.uy, prob.T)
    return lat


def padding_views(clb, lat, storage):
    """Views of the padding elements (the nodes x >= nx of each row's last chunk, every population)
    of both buffers."""
    import torch
    dt = {F64: torch.float64, F32: torch.float32, F16: torch.float16}[storage]
    es = {F64: 8, F32: 4, F16: 2}[storage]
    cur, oth, row, chunk = lat.buffers()
    nchunk = -(-lat.nx // chunk)
    assert row == nchunk * 14 * chunk
    base = lat._mem.data_ptr()
    views = []
    for ptr in (cur, oth):
        off = ptr - base
        assert off % es == 0 and GUARD <= off < GUARD + lat.footprint
        buf = lat._mem[off:off + lat.ny * row * es].view(dt).view(lat.ny, nchunk, 14, chunk)
        views.append(buf[:, nchunk - 1, :, lat.nx - (nchunk - 1) * chunk:])
    return views, nchunk * chunk


CASES = {
    "random_37x19": lambda st: W.random_problem(37, 19, seed=0, storage=st),
    "random_100x7_moving": lambda st: W.random_problem(100, 7, seed=1, storage=st, moving=True),
    "random_65x33_moving": lambda st: W.random_problem(65, 33, seed=2, storage=st, moving=True),
    "random_3x5": lambda st: W.random_problem(3, 5, seed=3, storage=st),
    "wet_walls_37x21": lambda st: W.normal_plate_channel(L=20, nx=37, storage=st, wet=True),
}


@pytest.mark.parametrize("storage", [F32, F16, F64])
@pytest.mark.parametrize("case", sorted(CASES))
def test_guards_and_padding_untouched(clb, storage, case):
    import torch
    prob = CASES[case](storage)
    nx = prob.nx
    lat = guarded_lattice(clb, prob)
    views, pitch = padding_views(clb, lat, storage)
    for v in views:
        v.fill_(float("nan"))
    before = [v.clone() for v in views]
    lat.step(37)                        # one graph chunk and single launches
    lat.autotune()                      # every candidate launch shape, staged-rows kernels included
    lat.run(1e-30, 200, 100)            # diagnostics passes
    nu = lat.nusselt(prob.nu_axis)
    er = lat.residual()
    lat.load(lat.save())                # checkpoint round trip (restores the padding too)
    lat.step(3)
    got = lat.fields()
    torch.cuda.synchronize()

    g = lat._mem
    assert bool((g[:GUARD] == PATTERN).all()) and bool((g[GUARD + lat.footprint:] == PATTERN).all())
    for v, b in zip(views, before):
        assert torch.equal(v.contiguous().view(-1).view(torch.uint8), b.contiguous().view(-1).view(torch.uint8)), \
            "padding was written"

    ref = clb.Lattice.from_problem(prob)
    ref.step(37)
    ref.run(1e-30, 200, 100)
    assert ref.nusselt(prob.nu_axis) == nu and ref.residual() == er
    ref.step(3)
    for a, b in zip(got, ref.fields()):
        assert np.array_equal(a, b)
    assert pitch >= nx
