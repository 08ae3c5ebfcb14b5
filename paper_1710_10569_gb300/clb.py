"""ctypes binding of libclb (include/clb.h), the coupled D2Q9 + D2Q5 central-moment LBM of
arXiv:1710.10569 on a GB300. Argument marshalling only: every step of the method runs in the
library's CUDA kernels. There is no CPU fallback; without a built libclb.so every call raises.

The C entry points are exposed under their C names (``clb_create``, ``clb_step``, ...) through
``lib()``; the classes below (``Lattice``, ``Batch``, ``Server``) wrap a handle and convert
numpy/torch arrays to pointers. Device memory for a lattice is a torch uint8 tensor of
``clb_footprint`` bytes handed to ``clb_create`` (PyTorch is the allocator; the library owns the
layout), and work goes on torch's current CUDA stream unless a stream is given.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libclb.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
HEADER = os.path.join(INCLUDE, "clb.h")

CLB_OK, CLB_EINVAL, CLB_ENOMEM, CLB_ENAN, CLB_ETIMEOUT, CLB_ECUDA, CLB_EBUSY = range(7)
STATUS_NAMES = {0: "CLB_OK", 1: "CLB_EINVAL", 2: "CLB_ENOMEM", 3: "CLB_ENAN", 4: "CLB_ETIMEOUT",
                5: "CLB_ECUDA", 6: "CLB_EBUSY"}


class CLBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class clb_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("kappa", ctypes.c_double), ("g_beta", ctypes.c_double),
                ("T0", ctypes.c_double), ("rho0", ctypes.c_double), ("s_b", ctypes.c_double),
                ("s_3", ctypes.c_double), ("s_4", ctypes.c_double), ("lambda2", ctypes.c_double),
                ("cs2_T", ctypes.c_double), ("Fv", ctypes.c_double * 2), ("wall", ctypes.c_int * 4),
                ("T_wall", ctypes.c_double * 4), ("storage", ctypes.c_int), ("T_ref", ctypes.c_double),
                ("u_ref", ctypes.c_double), ("dT_ref", ctypes.c_double), ("u_wall", ctypes.c_double * 8)]


class clb3d_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("kappa", ctypes.c_double), ("g_beta", ctypes.c_double),
                ("T0", ctypes.c_double), ("rho0", ctypes.c_double), ("s_b", ctypes.c_double),
                ("s_3", ctypes.c_double), ("s_4", ctypes.c_double), ("s_5", ctypes.c_double),
                ("s_6", ctypes.c_double), ("lambda2", ctypes.c_double), ("cs2_T", ctypes.c_double),
                ("Fv", ctypes.c_double * 3), ("g_axis", ctypes.c_int), ("wall", ctypes.c_int * 6),
                ("T_wall", ctypes.c_double * 6), ("storage", ctypes.c_int), ("T_ref", ctypes.c_double),
                ("u_wall", ctypes.c_double * 18), ("u_ref", ctypes.c_double), ("dT_ref", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long
_S = ctypes.c_size_t
_P = ctypes.POINTER

# name -> argtypes (restype is clb_status = int unless listed in _RESTYPES)
_SIGS = {
    "clb_params_default": [_P(clb_params)],
    "clb_footprint": [_I, _I, _P(clb_params), _P(_S)],
    "clb_create": [_I, _I, _P(clb_params), _VP, _VP, _S, _P(_VP)],
    "clb_destroy": [_VP],
    "clb_init_fields": [_VP, _D, _D, _D, _D],
    "clb_init_fields_device": [_VP, _VP, _VP, _VP, _VP],
    "clb_step": [_VP, _L],
    "clb_fields": [_VP, _D, _D, _D, _D],
    "clb_fields_device": [_VP, _VP, _VP, _VP, _VP],
    "clb_populations": [_VP, _D, _D],
    "clb_nusselt": [_VP, _I, _D],
    "clb_residual": [_VP, _D],
    "clb_nusselt_noalloc": [_VP, _I, _I, _P(clb_params), _I, _VP, _D],
    "clb_run": [_VP, ctypes.c_double, _L, _L, _P(_L), _D],
    "clb_check": [_VP, _I, _D, _D],
    "clb_steps": [_VP, _P(_L)],
    "clb_sync": [_VP],
    "clb_save": [_VP, _VP, _P(_S)],
    "clb_load": [_VP, _VP, _S],
    "clb_set_launch": [_VP, _I, _I, _I],
    "clb_get_launch": [_VP, _P(_I), _P(_I), _P(_I)],
    "clb_autotune": [_VP, _P(_I), _P(_I), _P(_I)],
    "clb_set_pipeline": [_VP, _I, _I],
    "clb_get_pipeline": [_VP, _P(_I), _P(_I)],
    "clb_stream": [_VP],
    "clb_buffers": [_VP, _P(_VP), _P(_VP), _P(_S), _P(_I)],
    "clb_step_partition": [_I, _I, _P(clb_params), _I, _P(_I)],
    "clb_last_error": [],
    "clb_version": [],
    "clb_thermal_create": [_I, _I, _P(clb_params), _VP, _P(_VP)],
    "clb_thermal_destroy": [_VP],
    "clb_thermal_init": [_VP, _D, _D, _D],
    "clb_thermal_step": [_VP, _L],
    "clb_thermal_fields": [_VP, _D],
    "clb_thermal_populations": [_VP, _D],
    "clb_thermal_sync": [_VP],
    "clb_batch_create": [_I, _P(_I), _P(_I), _P(clb_params), _VP, _P(_VP)],
    "clb_batch_destroy": [_VP],
    "clb_batch_init_fields": [_VP, _I, _D, _D, _D, _D],
    "clb_batch_step": [_VP, _L],
    "clb_batch_fields": [_VP, _I, _D, _D, _D, _D],
    "clb_batch_diagnostics": [_VP, _P(_I), _D, _D],
    "clb_batch_run": [_VP, ctypes.c_double, _L, _L, _P(_L), _D, _P(_I)],
    "clb_batch_status": [_VP, _P(_I), _D, _P(_L), _D],
    "clb_batch_set_tile": [_VP, _I, _I, _I],
    "clb_batch_autotune": [_VP, _P(_I), _P(_I), _P(_I)],
    "clb_batch_get_launch": [_VP, _P(_I), _P(_I), _P(_I), _P(_I), _P(ctypes.c_long)],
    "clb_serve_open": [_S, _I, _I, _VP, _P(_VP)],
    "clb_serve_close": [_VP],
    "clb_serve_submit": [_VP, _I, _I, _P(clb_params), _D, _D, _D, _D, _I, _L, ctypes.c_double, _P(_L)],
    "clb_serve_progress": [_VP, _L, _P(_I), _P(_I)],
    "clb_serve_poll": [_VP, _L, _P(_I), _D, _P(_L), _D],
    "clb_serve_cancel": [_VP, _L],
    "clb_serve_fetch": [_VP, _L, _D, _D, _D, _D],
    "clb3d_params_default": [_P(clb3d_params)],
    "clb3d_footprint": [_I, _I, _I, _P(clb3d_params), _P(_S)],
    "clb3d_create": [_I, _I, _I, _P(clb3d_params), _VP, _P(_VP)],
    "clb3d_destroy": [_VP],
    "clb3d_init_fields": [_VP, _D, _D, _D, _D, _D],
    "clb3d_step": [_VP, _L],
    "clb3d_fields": [_VP, _D, _D, _D, _D, _D],
    "clb3d_populations": [_VP, _D, _D],
    "clb3d_nusselt": [_VP, _I, _D],
    "clb3d_set_launch": [_VP, _I, _I],
    "clb3d_residual": [_VP, _D],
    "clb3d_thermal_create": [_I, _I, _I, _P(clb3d_params), _VP, _P(_VP)],
    "clb3d_thermal_destroy": [_VP],
    "clb3d_thermal_init": [_VP, _D, _D, _D, _D],
    "clb3d_thermal_step": [_VP, _L],
    "clb3d_thermal_fields": [_VP, _D],
    "clb3d_thermal_populations": [_VP, _D],
    "clb3d_thermal_sync": [_VP],
    "clb3d_save": [_VP, _VP, _P(_S)],
    "clb3d_load": [_VP, _VP, _S],
    "clb3d_run": [_VP, ctypes.c_double, _L, _L, _P(_L), _D],
    "clb3d_sync": [_VP],
    "clb3d_stream": [_VP],
    "clb3d_buffers": [_VP, _P(_VP), _P(ctypes.c_longlong), _P(_I)],
    "clb3d_batch_create": [_I, _P(_I), _P(_I), _P(_I), _P(clb3d_params), _VP, _P(_VP)],
    "clb3d_batch_destroy": [_VP],
    "clb3d_batch_lattice": [_VP, _I, _P(_VP)],
    "clb3d_batch_init_fields": [_VP, _I, _D, _D, _D, _D, _D],
    "clb3d_batch_step": [_VP, _L],
    "clb3d_batch_set_tile": [_VP, _I, _I],
    "clb3d_batch_get_launch": [_VP, _P(_I), _P(_I), _P(_I), _P(ctypes.c_longlong)],
}
_RESTYPES = {"clb_destroy": None, "clb_batch_destroy": None, "clb_serve_close": None,
             "clb_thermal_destroy": None, "clb3d_destroy": None, "clb3d_stream": _VP,
             "clb3d_thermal_destroy": None, "clb3d_batch_destroy": None,
             "clb_last_error": ctypes.c_char_p, "clb_version": ctypes.c_char_p, "clb_stream": _VP}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libclb with typed entry points. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libclb.so is not built ({LIB_PATH}); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, ctypes.c_int)
            _lib = L
    return _lib


def _check(status: int):
    if status != CLB_OK:
        raise CLBError(status, lib().clb_last_error().decode(errors="replace"))


def step_partition(nx: int, ny: int, p: dict, npt: int = 4) -> dict:
    """clb_step_partition: how the FP16 form splits a step into interior and edge warps (host
    only). Returns the interior rows and warp columns, the warp columns per row, and the edge rows
    and edge columns."""
    g = (_I * 11)()
    cp = params(p)
    _check(lib().clb_step_partition(int(nx), int(ny), ctypes.byref(cp), int(npt), g))
    return {"rows": (g[0], g[1]), "cols": (g[2], g[3]), "warp_cols": g[4],
            "edge_rows": [g[6 + k] for k in range(g[5])], "edge_cols": [g[9 + k] for k in range(g[8])]}


def params(p: dict) -> clb_params:
    """clb_params from a parameter dict (see workloads.default_params)."""
    s = clb_params()
    for k in ("nu", "kappa", "g_beta", "T0", "rho0", "s_b", "s_3", "s_4", "lambda2", "cs2_T", "T_ref",
              "u_ref", "dT_ref"):
        setattr(s, k, float(p[k]))
    s.Fv[0], s.Fv[1] = (float(v) for v in p["Fv"])
    for i in range(4):
        s.wall[i] = int(p["wall"][i])
        s.T_wall[i] = float(p["T_wall"][i])
    s.storage = int(p["storage"])
    uw = p.get("u_wall", ((0.0, 0.0),) * 4)
    for side in range(4):
        s.u_wall[2 * side], s.u_wall[2 * side + 1] = float(uw[side][0]), float(uw[side][1])
    return s


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, "need C-contiguous float64"
    return a.ctypes.data_as(_D)


def _host(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"field has {a.size} values, lattice has {n} nodes")
    return a


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _tptr(t):
    if t is None:
        return None
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return t.data_ptr()


class Lattice:
    """One lattice on the GPU (handle of clb_create)."""

    def __init__(self, nx: int, ny: int, p: dict, stream=None, torch_memory: bool = True):
        import torch
        L = lib()
        self.nx, self.ny, self.params = int(nx), int(ny), dict(p)
        self._p = params(p)
        nbytes = _S()
        _check(L.clb_footprint(self.nx, self.ny, ctypes.byref(self._p), ctypes.byref(nbytes)))
        self.footprint = nbytes.value
        self._mem = None
        mem_ptr = None
        if torch_memory:
            # torch's caching allocator hands out 512-byte aligned blocks
            self._mem = torch.empty(self.footprint, dtype=torch.uint8, device="cuda")
            mem_ptr = self._mem.data_ptr()
        self.stream = _stream_handle(stream)
        h = _VP()
        _check(L.clb_create(self.nx, self.ny, ctypes.byref(self._p), self.stream, mem_ptr,
                            self.footprint if mem_ptr else 0, ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_problem(cls, prob: W.Problem, **kw) -> "Lattice":
        lat = cls(prob.nx, prob.ny, prob.params, **kw)
        lat.init_fields(prob.rho, prob.ux, prob.uy, prob.T)
        return lat

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def close(self):
        if getattr(self, "_h", None):
            lib().clb_destroy(self._h)
            self._h = None
            self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rho=None, ux=None, uy=None, T=None):
        n = self.nodes
        arrs = [_host(a, n) for a in (rho, ux, uy, T)]
        _check(lib().clb_init_fields(self._h, *[_dptr(a) for a in arrs]))

    def init_fields_device(self, rho=None, ux=None, uy=None, T=None):
        _check(lib().clb_init_fields_device(self._h, *[_tptr(t) for t in (rho, ux, uy, T)]))

    def step(self, n: int = 1):
        _check(lib().clb_step(self._h, int(n)))

    def fields(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        _check(lib().clb_fields(self._h, *[_dptr(a) for a in out]))
        return tuple(out)

    def fields_into(self, rho=None, ux=None, uy=None, T=None):
        """Host (numpy, e.g. pinned) outputs; any may be None."""
        _check(lib().clb_fields(self._h, *[_dptr(a) for a in (rho, ux, uy, T)]))

    def fields_device(self, rho=None, ux=None, uy=None, T=None):
        _check(lib().clb_fields_device(self._h, *[_tptr(t) for t in (rho, ux, uy, T)]))

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, self.ny, self.nx))
        _check(lib().clb_populations(self._h, _dptr(f), _dptr(g)))
        return f, g

    def nusselt(self, axis: int = 1) -> float:
        v = ctypes.c_double()
        _check(lib().clb_nusselt(self._h, int(axis), ctypes.byref(v)))
        return v.value

    def residual(self) -> float:
        v = ctypes.c_double()
        _check(lib().clb_residual(self._h, ctypes.byref(v)))
        return v.value

    def check(self, axis: int = 1):
        """(Nusselt number along axis, residual E_R) from one FP64 pass; the snapshot is retaken."""
        nu, er = ctypes.c_double(), ctypes.c_double()
        _check(lib().clb_check(self._h, int(axis), ctypes.byref(nu), ctypes.byref(er)))
        return nu.value, er.value

    def run(self, tol: float, max_steps: int, interval: int = 100):
        st, er = _L(), ctypes.c_double()
        _check(lib().clb_run(self._h, float(tol), int(max_steps), int(interval), ctypes.byref(st),
                             ctypes.byref(er)))
        return st.value, er.value

    @property
    def steps(self) -> int:
        v = _L()
        _check(lib().clb_steps(self._h, ctypes.byref(v)))
        return v.value

    def sync(self):
        _check(lib().clb_sync(self._h))

    def save(self) -> bytes:
        n = _S()
        _check(lib().clb_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().clb_save(self._h, ctypes.cast(buf, _VP), ctypes.byref(n)))
        return buf.raw[:n.value]

    def load(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(lib().clb_load(self._h, ctypes.cast(buf, _VP), len(data)))

    def set_launch(self, block_x: int = 0, block_y: int = 0, nodes_per_thread: int = 0):
        _check(lib().clb_set_launch(self._h, int(block_x), int(block_y), int(nodes_per_thread)))

    def launch(self):
        bx, by, npt = _I(), _I(), _I()
        _check(lib().clb_get_launch(self._h, ctypes.byref(bx), ctypes.byref(by), ctypes.byref(npt)))
        return bx.value, by.value, npt.value

    def autotune(self):
        bx, by, npt = _I(), _I(), _I()
        _check(lib().clb_autotune(self._h, ctypes.byref(bx), ctypes.byref(by), ctypes.byref(npt)))
        return bx.value, by.value, npt.value

    def set_pipeline(self, stages: int, rows: int = 0):
        _check(lib().clb_set_pipeline(self._h, int(stages), int(rows)))

    def pipeline(self):
        st, rows = _I(), _I()
        _check(lib().clb_get_pipeline(self._h, ctypes.byref(st), ctypes.byref(rows)))
        return st.value, rows.value

    def buffers(self):
        """(current buffer, other buffer, elements per chunked row, nodes per chunk): element
        (i, x, y) lies at y * row_elems + (x // chunk) * 14 * chunk + i * chunk + x % chunk."""
        cur, oth, row, chunk = _VP(), _VP(), _S(), _I()
        _check(lib().clb_buffers(self._h, ctypes.byref(cur), ctypes.byref(oth), ctypes.byref(row),
                                 ctypes.byref(chunk)))
        return cur.value, oth.value, row.value, chunk.value


class Thermal:
    """The D2Q5 equation alone with a prescribed velocity field (clb_thermal_*)."""

    def __init__(self, nx: int, ny: int, p: dict, stream=None):
        self.nx, self.ny, self.params = int(nx), int(ny), dict(p)
        self._p = params(p)
        self.stream = _stream_handle(stream)
        h = _VP()
        _check(lib().clb_thermal_create(self.nx, self.ny, ctypes.byref(self._p), self.stream, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().clb_thermal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, T=None, ux=None, uy=None):
        n = self.nx * self.ny
        arrs = [_host(a, n) for a in (T, ux, uy)]
        _check(lib().clb_thermal_init(self._h, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        _check(lib().clb_thermal_step(self._h, int(n)))

    def sync(self):
        _check(lib().clb_thermal_sync(self._h))

    def temperature(self):
        T = np.empty((self.ny, self.nx))
        _check(lib().clb_thermal_fields(self._h, _dptr(T)))
        return T

    def populations(self):
        g = np.empty((5, self.ny, self.nx))
        _check(lib().clb_thermal_populations(self._h, _dptr(g)))
        return g


class Batch:
    """Many lattices stepped in one launch per time step (clb_batch_*)."""

    def __init__(self, problems, stream=None):
        L = lib()
        self.problems = list(problems)
        n = len(self.problems)
        nx = (ctypes.c_int * n)(*[p.nx for p in self.problems])
        ny = (ctypes.c_int * n)(*[p.ny for p in self.problems])
        ps = (clb_params * n)(*[params(p.params) for p in self.problems])
        self.stream = _stream_handle(stream)
        h = _VP()
        _check(L.clb_batch_create(n, nx, ny, ps, self.stream, ctypes.byref(h)))
        self._h = h
        self._axis = (ctypes.c_int * n)(*[p.nu_axis for p in self.problems])
        for k, p in enumerate(self.problems):
            self.init_fields(k, p.rho, p.ux, p.uy, p.T)

    def __len__(self):
        return len(self.problems)

    def close(self):
        if getattr(self, "_h", None):
            lib().clb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, k, rho=None, ux=None, uy=None, T=None):
        n = self.problems[k].nodes
        arrs = [_host(a, n) for a in (rho, ux, uy, T)]
        _check(lib().clb_batch_init_fields(self._h, int(k), *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        _check(lib().clb_batch_step(self._h, int(n)))

    def fields(self, k):
        p = self.problems[k]
        out = [np.empty((p.ny, p.nx)) for _ in range(4)]
        _check(lib().clb_batch_fields(self._h, int(k), *[_dptr(a) for a in out]))
        return tuple(out)

    def diagnostics(self):
        n = len(self.problems)
        nu, er = np.empty(n), np.empty(n)
        _check(lib().clb_batch_diagnostics(self._h, self._axis, _dptr(nu), _dptr(er)))
        return nu, er

    def run(self, tol: float, max_steps: int, interval: int = 100):
        n = len(self.problems)
        steps = (ctypes.c_long * n)()
        er = np.empty(n)
        status = (ctypes.c_int * n)()
        _check(lib().clb_batch_run(self._h, float(tol), int(max_steps), int(interval), steps,
                                   _dptr(er), status))
        return np.array(steps[:], dtype=np.int64), er, np.array(status[:], dtype=np.int32)

    def status(self):
        """(status, residual, steps, Nusselt number) of every instance as of its last check."""
        n = len(self.problems)
        status = (ctypes.c_int * n)()
        steps = (ctypes.c_long * n)()
        er, nu = np.empty(n), np.empty(n)
        _check(lib().clb_batch_status(self._h, status, _dptr(er), steps, _dptr(nu)))
        return (np.array(status[:], dtype=np.int32), er, np.array(steps[:], dtype=np.int64), nu)

    def set_tile(self, tile_x: int, tile_y: int = 1, nodes_per_thread: int = 1):
        _check(lib().clb_batch_set_tile(self._h, int(tile_x), int(tile_y), int(nodes_per_thread)))

    def autotune(self):
        tx, ty, npt = _I(), _I(), _I()
        _check(lib().clb_batch_autotune(self._h, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(npt)))
        return tx.value, ty.value, npt.value

    def launch(self) -> dict:
        """Geometry of the next batched step: tile (threads x, threads y, nodes per thread), groups
        of rows each block steps, and blocks per launch."""
        tx, ty, npt, groups, blocks = _I(), _I(), _I(), _I(), ctypes.c_long()
        _check(lib().clb_batch_get_launch(self._h, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(npt),
                                          ctypes.byref(groups), ctypes.byref(blocks)))
        return dict(tile=(tx.value, ty.value, npt.value), groups=groups.value, blocks=blocks.value)


class Server:
    """Continuous-batching request server (clb_serve_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, storage: int, stream=None):
        self.stream = _stream_handle(stream)
        h = _VP()
        _check(lib().clb_serve_open(int(hbm_budget_bytes), int(max_slots), int(storage), self.stream,
                                    ctypes.byref(h)))
        self._h = h
        self.storage = storage

    def close(self):
        if getattr(self, "_h", None):
            lib().clb_serve_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prob: W.Problem, step_cap: int, tol: float) -> int:
        n = prob.nodes
        arrs = [_host(a, n) for a in prob.fields()]
        p = params(prob.params)
        rid = _L()
        _check(lib().clb_serve_submit(self._h, prob.nx, prob.ny, ctypes.byref(p),
                                      *[_dptr(a) for a in arrs], int(prob.nu_axis), int(step_cap),
                                      float(tol), ctypes.byref(rid)))
        return rid.value

    def progress(self, chunk: int):
        a, q = _I(), _I()
        _check(lib().clb_serve_progress(self._h, int(chunk), ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def cancel(self, rid: int):
        _check(lib().clb_serve_cancel(self._h, int(rid)))

    def poll(self, rid: int):
        done, nu, steps, er = _I(), ctypes.c_double(), _L(), ctypes.c_double()
        _check(lib().clb_serve_poll(self._h, int(rid), ctypes.byref(done), ctypes.byref(nu),
                                    ctypes.byref(steps), ctypes.byref(er)))
        return bool(done.value), nu.value, steps.value, er.value

    def fetch(self, rid: int, ny: int, nx: int):
        out = [np.empty((ny, nx)) for _ in range(4)]
        _check(lib().clb_serve_fetch(self._h, int(rid), *[_dptr(a) for a in out]))
        return tuple(out)


def declared_entry_points(header: str | None = None):
    """Names of the functions the headers in include/ declare (or the one header given)."""
    import glob
    import re
    names = set()
    for path in [header] if header else sorted(glob.glob(os.path.join(INCLUDE, "*.h"))):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(clb(?:3d)?_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def params3(p: dict) -> clb3d_params:
    """clb3d_params from a parameter dict (see workloads.default_params3)."""
    s = clb3d_params()
    for k in ("nu", "kappa", "g_beta", "T0", "rho0", "s_b", "s_3", "s_4", "s_5", "s_6", "lambda2",
              "cs2_T", "T_ref", "u_ref", "dT_ref"):
        setattr(s, k, float(p[k]))
    for i in range(3):
        s.Fv[i] = float(p["Fv"][i])
    s.g_axis = int(p["g_axis"])
    for i in range(6):
        s.wall[i] = int(p["wall"][i])
        s.T_wall[i] = float(p["T_wall"][i])
    uw = p.get("u_wall", ((0.0, 0.0, 0.0),) * 6)
    for face in range(6):
        for d in range(3):
            s.u_wall[3 * face + d] = float(uw[face][d])
    s.storage = int(p["storage"])
    return s


class Lattice3D:
    """One 3-D lattice (D3Q27 + D3Q7, include/clb3d.h). Fields are (nz, ny, nx) float64 arrays. The
    library allocates the lattice's device memory; work goes on torch's current stream unless a
    stream is given."""

    def __init__(self, nx: int, ny: int, nz: int, p: dict, stream=None):
        L = lib()
        self.nx, self.ny, self.nz = nx, ny, nz
        self.params = dict(p)
        self._p = params3(p)
        self.stream = _stream_handle(stream)
        h = _VP()
        _check(L.clb3d_create(nx, ny, nz, ctypes.byref(self._p), self.stream, ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_problem(cls, prob, stream=None) -> "Lattice3D":
        lat = cls(prob.nx, prob.ny, prob.nz, prob.params, stream)
        lat.init_fields(*prob.fields())
        return lat

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def close(self):
        if getattr(self, "_h", None):
            lib().clb3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rho, ux, uy, uz, T):
        n = self.nodes
        arrs = [_host(np.broadcast_to(np.asarray(a, dtype=np.float64), self.shape), n)
                for a in (rho, ux, uy, uz, T)]
        _check(lib().clb3d_init_fields(self._h, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        _check(lib().clb3d_step(self._h, int(n)))

    def sync(self):
        _check(lib().clb3d_sync(self._h))

    def fields(self):
        """(rho, ux, uy, uz, T), each (nz, ny, nx)."""
        out = [np.empty(self.shape) for _ in range(5)]
        _check(lib().clb3d_fields(self._h, *[_dptr(a) for a in out]))
        return tuple(out)

    def populations(self):
        f = np.empty((27,) + self.shape)
        g = np.empty((7,) + self.shape)
        _check(lib().clb3d_populations(self._h, _dptr(f), _dptr(g)))
        return f, g

    def nusselt(self, axis: int = 2) -> float:
        v = ctypes.c_double()
        _check(lib().clb3d_nusselt(self._h, int(axis), ctypes.byref(v)))
        return v.value

    def set_launch(self, block_x: int = 0, block_y: int = 0):
        _check(lib().clb3d_set_launch(self._h, int(block_x), int(block_y)))

    def residual(self) -> float:
        v = ctypes.c_double()
        _check(lib().clb3d_residual(self._h, ctypes.byref(v)))
        return v.value

    def save(self) -> bytes:
        n = _S()
        _check(lib().clb3d_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().clb3d_save(self._h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def load(self, data: bytes):
        _check(lib().clb3d_load(self._h, data, len(data)))

    def run(self, tol: float, max_steps: int, interval: int = 100):
        st, er = _L(), ctypes.c_double()
        _check(lib().clb3d_run(self._h, float(tol), int(max_steps), int(interval), ctypes.byref(st),
                               ctypes.byref(er)))
        return st.value, er.value


class _Member3D(Lattice3D):
    """A lattice owned by a Batch3D: read access through the single-lattice calls; its state changes
    only through the batch."""

    def __init__(self, batch, k: int, prob):
        self.nx, self.ny, self.nz = prob.nx, prob.ny, prob.nz
        self.params = dict(prob.params)
        self.stream = batch.stream
        h = _VP()
        _check(lib().clb3d_batch_lattice(batch._h, int(k), ctypes.byref(h)))
        self._h = h
        self._batch = batch  # the batch owns and destroys the handle

    def close(self):
        self._h = None

    def step(self, n: int = 1):
        raise RuntimeError("a batch member is stepped by its batch (Batch3D.step)")

    def init_fields(self, *a):
        raise RuntimeError("a batch member is initialised by its batch (Batch3D.init_fields)")


class Batch3D:
    """Many 3-D lattices (clb3d_batch_*) stepped by one launch per time step. `member(k)` gives a
    Lattice3D view of lattice k for fields, populations, Nusselt number and residual."""

    def __init__(self, problems, stream=None):
        L = lib()
        self.problems = list(problems)
        n = len(self.problems)
        self.stream = _stream_handle(stream)
        nx = (_I * n)(*[p.nx for p in self.problems])
        ny = (_I * n)(*[p.ny for p in self.problems])
        nz = (_I * n)(*[p.nz for p in self.problems])
        ps = (clb3d_params * n)(*[params3(p.params) for p in self.problems])
        h = _VP()
        _check(L.clb3d_batch_create(n, nx, ny, nz, ps, self.stream, ctypes.byref(h)))
        self._h = h
        self.members = [_Member3D(self, k, p) for k, p in enumerate(self.problems)]
        for k, p in enumerate(self.problems):
            self.init_fields(k, *p.fields())

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m.close()
            lib().clb3d_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def member(self, k: int) -> Lattice3D:
        return self.members[k]

    def init_fields(self, k: int, rho, ux, uy, uz, T):
        m = self.members[k]
        arrs = [_host(np.broadcast_to(np.asarray(a, dtype=np.float64), m.shape), m.nodes)
                for a in (rho, ux, uy, uz, T)]
        _check(lib().clb3d_batch_init_fields(self._h, int(k), *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        _check(lib().clb3d_batch_step(self._h, int(n)))

    def fields(self, k: int):
        return self.members[k].fields()

    def set_tile(self, block_x: int, block_y: int = 1):
        _check(lib().clb3d_batch_set_tile(self._h, int(block_x), int(block_y)))

    def launch(self) -> dict:
        bx, by, groups, blocks = _I(), _I(), _I(), ctypes.c_longlong()
        _check(lib().clb3d_batch_get_launch(self._h, ctypes.byref(bx), ctypes.byref(by), ctypes.byref(groups),
                                            ctypes.byref(blocks)))
        return dict(block=(bx.value, by.value), groups=groups.value, blocks=blocks.value)


class Thermal3D:
    """The D3Q7 equation alone with a prescribed velocity (include/clb3d.h, clb3d_thermal_*).
    Fields are (nz, ny, nx) float64 arrays."""

    def __init__(self, nx: int, ny: int, nz: int, p: dict, stream=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.params = dict(p)
        self._p = params3(p)
        self.stream = _stream_handle(stream)
        h = _VP()
        _check(lib().clb3d_thermal_create(nx, ny, nz, ctypes.byref(self._p), self.stream, ctypes.byref(h)))
        self._h = h

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None):
            lib().clb3d_thermal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, T, ux, uy, uz):
        n = self.nx * self.ny * self.nz
        arrs = [_host(np.broadcast_to(np.asarray(a, dtype=np.float64), self.shape), n) for a in (T, ux, uy, uz)]
        _check(lib().clb3d_thermal_init(self._h, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        _check(lib().clb3d_thermal_step(self._h, int(n)))

    def sync(self):
        _check(lib().clb3d_thermal_sync(self._h))

    def temperature(self):
        T = np.empty(self.shape)
        _check(lib().clb3d_thermal_fields(self._h, _dptr(T)))
        return T

    def populations(self):
        g = np.empty((7,) + self.shape)
        _check(lib().clb3d_thermal_populations(self._h, _dptr(g)))
        return g
