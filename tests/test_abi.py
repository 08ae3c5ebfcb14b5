"""The C ABI library without a GPU: it builds for sm_103a, loads, exports every entry point that
include/clb.h declares, and its host-side validation answers with status codes."""
import ctypes

import pytest

from paper_1710_10569_gb300 import build as B
from paper_1710_10569_gb300 import workloads as W


@pytest.fixture(scope="module")
def clb():
    B.build()
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def test_every_declared_entry_point_is_exported(clb):
    names = clb.declared_entry_points()
    assert len(names) >= 30
    L = clb.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing
    # and the binding types every one of them
    assert set(names) <= set(clb._SIGS)


def test_version_and_defaults(clb):
    L = clb.lib()
    assert b"sm_103a" in L.clb_version()
    p = clb.clb_params()
    assert L.clb_params_default(ctypes.byref(p)) == clb.CLB_OK
    assert (p.cs2_T, p.s_3, p.s_4, p.lambda2, p.s_b, p.rho0) == (0.25, 1.0, 1.0, 1.0, 1.0, 1.0)
    assert list(p.wall) == [0, 0, 0, 0] and p.storage == 0


def footprint(clb, nx, ny, **kw):
    p = clb.params(W.default_params(**kw))
    n = ctypes.c_size_t()
    st = clb.lib().clb_footprint(nx, ny, ctypes.byref(p), ctypes.byref(n))
    return st, n.value


def test_footprint_scales_with_storage(clb):
    sizes = {}
    for s in (W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV):
        st, n = footprint(clb, 2048, 1024, storage=s)
        assert st == clb.CLB_OK
        sizes[s] = n
    nodes = 2048 * 1024
    # two buffers of 14 populations plus FP64 snapshot (24 B) and staging (32 B) per node
    for s, b in ((W.STORAGE_F64, 8), (W.STORAGE_F32, 4), (W.STORAGE_F16DEV, 2)):
        assert sizes[s] >= nodes * (2 * 14 * b + 56)
        assert sizes[s] < nodes * (2 * 14 * b + 56) * 1.01


@pytest.mark.parametrize("kw,nx,ny", [
    (dict(nu=0.0), 8, 8),
    (dict(nu=-1.0), 8, 8),
    (dict(kappa=0.0), 8, 8),
    (dict(s_3=2.0), 8, 8),
    (dict(s_b=0.0), 8, 8),
    (dict(lambda2=2.5), 8, 8),
    (dict(cs2_T=0.5), 8, 8),
    (dict(wall=(0, 1, 0, 0)), 8, 8),
    (dict(wall=(1, 1, 0, 2)), 8, 8),
    (dict(wall=(7, 7, 0, 0)), 8, 8),
    (dict(wall=(3, 0, 0, 0)), 8, 8),      # wet walls come in pairs
    (dict(wall=(0, 0, 3, 1)), 8, 8),
    (dict(wall=(3, 3, 1, 1)), 8, 8),      # beside wet walls: periodic or wet sides only
    (dict(wall=(2, 2, 3, 3)), 8, 8),
    (dict(wall=(3, 3, 0, 0)), 2, 8),      # three nodes across a wet pair
    (dict(wall=(0, 0, 3, 3)), 8, 2),
    (dict(storage=5), 8, 8),
    (dict(nu=float("nan")), 8, 8),
    ({}, 1, 8),
    ({}, 8, 0),
    ({}, (1 << 20) + 1, 4),
    ({}, 1 << 16, 1 << 15),
])
def test_invalid_arguments_are_rejected(clb, kw, nx, ny):
    st, _ = footprint(clb, nx, ny, **kw)
    assert st == clb.CLB_EINVAL
    assert clb.lib().clb_last_error()
    h = ctypes.c_void_p()
    p = clb.params(W.default_params(**kw))
    assert clb.lib().clb_create(nx, ny, ctypes.byref(p), None, None, 0, ctypes.byref(h)) == clb.CLB_EINVAL
    assert not h.value


@pytest.mark.parametrize("wall,nx,ny", [((3, 3, 0, 0), 3, 2), ((0, 0, 3, 3), 2, 3), ((3, 3, 3, 3), 3, 3)])
def test_wet_walls_on_either_axis_and_closed_boxes_are_accepted(clb, wall, nx, ny):
    st, n = footprint(clb, nx, ny, wall=wall)
    assert st == clb.CLB_OK and n > 0


def test_null_handles_are_rejected(clb):
    L = clb.lib()
    assert L.clb_step(None, 1) == clb.CLB_EINVAL
    assert L.clb_sync(None) == clb.CLB_EINVAL
    assert L.clb_batch_step(None, 1) == clb.CLB_EINVAL
    assert L.clb_serve_progress(None, 2, None, None) == clb.CLB_EINVAL
    L.clb_destroy(None)
    L.clb_batch_destroy(None)
    L.clb_serve_close(None)


def test_binding_raises_without_library(monkeypatch, tmp_path):
    from paper_1710_10569_gb300 import clb as c
    monkeypatch.setattr(c, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(c, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        c.lib()


def footprint3(clb, nx, ny, nz, **kw):
    p = clb.params3(W.default_params3(**kw))
    n = ctypes.c_size_t()
    st = clb.lib().clb3d_footprint(nx, ny, nz, ctypes.byref(p), ctypes.byref(n))
    return st, n.value


def test_3d_defaults_and_footprint(clb):
    p = clb.clb3d_params()
    assert clb.lib().clb3d_params_default(ctypes.byref(p)) == clb.CLB_OK
    assert (p.cs2_T, p.s_3, p.s_6, p.g_axis, p.rho0) == (0.25, 1.0, 1.0, 2, 1.0)
    st, n64 = footprint3(clb, 256, 256, 128, storage=W.STORAGE_F64)
    st2, n32 = footprint3(clb, 256, 256, 128, storage=W.STORAGE_F32)
    assert st == st2 == clb.CLB_OK
    nodes = 256 * 256 * 128
    # two buffers of 34 populations, 5 FP64 staging fields and a 4-field FP64 residual snapshot per node
    assert nodes * (2 * 34 * 8 + 72) <= n64 < nodes * (2 * 34 * 8 + 72) * 1.01
    assert nodes * (2 * 34 * 4 + 72) <= n32 < nodes * (2 * 34 * 4 + 72) * 1.01


@pytest.mark.parametrize("kw,n", [
    (dict(nu=0.0), (8, 8, 8)),
    (dict(storage=3), (8, 8, 8)),
    (dict(wall=(W.WALL_PERIODIC, W.WALL_DIRICHLET) + (W.WALL_PERIODIC,) * 4), (8, 8, 8)),
    (dict(wall=(W.WALL_WET,) * 2 + (W.WALL_PERIODIC,) * 4), (8, 8, 8)),
    (dict(g_axis=3), (8, 8, 8)),
    (dict(s_5=2.0), (8, 8, 8)),
    (dict(wall=(W.WALL_PERIODIC,) * 4 + (W.WALL_ADIABATIC,) * 2,
          u_wall=((0.0, 0.0, 0.0),) * 5 + ((0.5, 0.0, 0.0),)), (8, 8, 8)),
    (dict(cs2_T=0.34), (8, 8, 8)),
    (dict(), (0, 8, 8)),
    (dict(), (1 << 11, 1 << 11, 1 << 10)),
])
def test_3d_invalid_arguments_are_rejected(clb, kw, n):
    st, _ = footprint3(clb, *n, **kw)
    assert st == clb.CLB_EINVAL
    assert clb.lib().clb_last_error()


def test_3d_largest_lattice_in_32_bit_offsets(clb):
    """A 3-D buffer must stay below 2^31 elements (offsets within it are 32-bit): 384 x 384 x 428
    in FP32 (34 planes of 63.1 M elements) is accepted, one more layer is refused."""
    assert footprint3(clb, 384, 384, 428, storage=W.STORAGE_F32)[0] == clb.CLB_OK
    assert footprint3(clb, 384, 384, 429, storage=W.STORAGE_F32)[0] == clb.CLB_EINVAL


def test_3d_batch_invalid_arguments_are_rejected(clb):
    """clb3d_batch_create checks its arguments before touching the device: no lattices, a bad
    lattice, or storages that differ."""
    L = clb.lib()
    out = ctypes.c_void_p()
    n3 = (ctypes.c_int * 2)(8, 8)
    good = clb.params3(W.default_params3(storage=W.STORAGE_F32))
    other = clb.params3(W.default_params3(storage=W.STORAGE_F64))
    bad = clb.params3(W.default_params3(nu=0.0, storage=W.STORAGE_F32))
    assert L.clb3d_batch_create(0, n3, n3, n3, ctypes.byref(good), None, ctypes.byref(out)) == clb.CLB_EINVAL
    for second in (other, bad):
        ps = (clb.clb3d_params * 2)(good, second)
        assert L.clb3d_batch_create(2, n3, n3, n3, ps, None, ctypes.byref(out)) == clb.CLB_EINVAL
        assert not out.value


@pytest.mark.parametrize("header", ["clb.h", "clb3d.h"])
def test_headers_are_plain_c(header):
    """The ABI headers compile as C99 (no C++ in the declarations a C caller sees)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    path = os.path.join(os.path.dirname(__file__), "..", "include", header)
    r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", "-x", "c", "-std=c99", path],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


PARTITION_WALLS = {
    "periodic": (W.WALL_PERIODIC,) * 4,
    "rb": (W.WALL_PERIODIC, W.WALL_PERIODIC, W.WALL_DIRICHLET, W.WALL_DIRICHLET),
    "cavity": (W.WALL_DIRICHLET, W.WALL_DIRICHLET, W.WALL_ADIABATIC, W.WALL_ADIABATIC),
    "channel": (W.WALL_PERIODIC, W.WALL_PERIODIC, W.WALL_ADIABATIC, W.WALL_ADIABATIC),
    "wet_y": (W.WALL_PERIODIC, W.WALL_PERIODIC, W.WALL_WET, W.WALL_WET),
    "wet_x": (W.WALL_WET, W.WALL_WET, W.WALL_PERIODIC, W.WALL_PERIODIC),
    "wet_box": (W.WALL_WET,) * 4,
}


@pytest.mark.parametrize("walls", sorted(PARTITION_WALLS))
@pytest.mark.parametrize("npt", [1, 2, 4])
def test_step_partition_covers_every_warp_once(clb, walls, npt):
    """The FP16 step's split (clb_step_partition): the interior warps and the warps the edge kernel
    enumerates cover every (row, warp column) of the lattice exactly once, and no interior warp has
    a wall next to any of its nodes or runs past the end of its row."""
    w = PARTITION_WALLS[walls]
    wall_y = w[2] != W.WALL_PERIODIC
    wall_x = w[0] != W.WALL_PERIODIC
    width = 32 * npt
    for nx, ny in [(3, 3), (4, 3), (31, 5), (127, 5), (128, 5), (129, 5), (256, 3), (257, 3), (384, 7),
                   (1000, 4), (33, 33), (64, 64), (4096, 6)]:
        g = clb.step_partition(nx, ny, W.default_params(wall=w, storage=W.STORAGE_F16DEV), npt)
        nw = g["warp_cols"]
        assert nw == -(-nx // width)
        (y0, y1), (c0, c1) = g["rows"], g["cols"]
        inner = {(y, c) for y in range(y0, y1) for c in range(c0, c1)}
        edge = [(y, c) for y in g["edge_rows"] for c in range(nw)]
        edge += [(y, c) for y in range(y0, y1) for c in g["edge_cols"]]
        assert len(edge) == len(set(edge)), (nx, ny, g)
        assert not inner & set(edge), (nx, ny, g)
        assert inner | set(edge) == {(y, c) for y in range(ny) for c in range(nw)}, (nx, ny, g)
        for y, c in inner:
            x0, x1 = c * width, c * width + width - 1
            assert x1 < nx
            assert not wall_y or 0 < y < ny - 1
            assert not wall_x or (x0 > 0 and x1 < nx - 1)


def test_step_partition_rejects_bad_arguments(clb):
    p = W.default_params(storage=W.STORAGE_F16DEV)
    with pytest.raises(clb.CLBError):
        clb.step_partition(64, 64, p, npt=3)
    with pytest.raises(clb.CLBError):
        clb.step_partition(1, 64, p)
