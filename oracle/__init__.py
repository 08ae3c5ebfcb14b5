"""FP64 CPU oracle of the coupled D2Q9 + D2Q5 central-moment lattice Boltzmann method
(Fei, Luo, Lin & Li, arXiv:1710.10569, Sec. 2) -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may import this module.
The arithmetic lives in ``clb_oracle.c`` (plain C, literal matrices of Eqs. 7, 17, 18); this wrapper
only marshals arguments, plus two diagnostics written out in numpy from their definitions:

* ``nusselt``: Eq. (29), Nu = 1 + <u_perp (T - T0)> H / (alpha dT), averaged over all nodes;
* ``residual``: the steady-state residual E_R. The paper defines it only by citation (Sec. 3.2); the
  reading used here is E_R = max over X in {u, T} of sqrt(sum |X(t) - X(t-D)|^2 / max(sum |X(t)|^2,
  N (1e-3 X_ref)^2)), with X_ref = u_ref for u and dT_ref for T (no floor when X_ref = 0).

Parity pins: every function here is checked by tests/test_oracle_pins.py against facts the paper and
the mathematics fix (brute-force moment sums, fixed points, conservation, decay rates, Poiseuille and
conduction profiles, Table 1 Nusselt numbers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "clb_oracle.c"), os.path.join(_HERE, "clb3d_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

PERIODIC, DIRICHLET, ADIABATIC, WET = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no host-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(map(os.path.getmtime, _SRCS)):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
                               "-fopenmp",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nu", ctypes.c_double), ("kappa", ctypes.c_double), ("g_beta", ctypes.c_double),
                ("T0", ctypes.c_double), ("rho0", ctypes.c_double),
                ("s_b", ctypes.c_double), ("s_3", ctypes.c_double), ("s_4", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("lambda2", ctypes.c_double), ("cs2_T", ctypes.c_double),
                ("Fv", ctypes.c_double * 2), ("wall", ctypes.c_int * 4), ("T_wall", ctypes.c_double * 4),
                ("thermal_only", ctypes.c_int), ("u_wall", ctypes.c_double * 8)]


class _Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nu", ctypes.c_double), ("kappa", ctypes.c_double), ("g_beta", ctypes.c_double),
                ("T0", ctypes.c_double), ("rho0", ctypes.c_double),
                ("s_b", ctypes.c_double), ("s_3", ctypes.c_double), ("s_4", ctypes.c_double),
                ("s_5", ctypes.c_double), ("s_6", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("lambda2", ctypes.c_double), ("cs2_T", ctypes.c_double),
                ("Fv", ctypes.c_double * 3), ("g_axis", ctypes.c_int), ("wall", ctypes.c_int * 6),
                ("T_wall", ctypes.c_double * 6), ("u_wall", ctypes.c_double * 18),
                ("thermal_only", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # Idle threads spin only briefly before they block: the node loops are short and the
            # oracle may share the host cores with other processes.
            os.environ.setdefault("GOMP_SPINCOUNT", "20000")
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d = P(ctypes.c_double)
            lib.orc_create.argtypes = [P(_Params), P(ctypes.c_void_p)]
            lib.orc_create.restype = ctypes.c_int
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_init.argtypes = [ctypes.c_void_p, d, d, d, d]
            lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            lib.orc_steps.argtypes = [ctypes.c_void_p]
            lib.orc_steps.restype = ctypes.c_long
            lib.orc_threads.argtypes = []
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_fields.argtypes = [ctypes.c_void_p, d, d, d, d]
            lib.orc_get_pops.argtypes = [ctypes.c_void_p, d, d]
            lib.orc_set_pops.argtypes = [ctypes.c_void_p, d, d]
            lib.orc_collide_node.argtypes = [P(_Params), d, d, d, d]
            lib.orc_collide_thermal_node.argtypes = [P(_Params), d, ctypes.c_double, ctypes.c_double, d]
            lib.orc_equilibrium_node.argtypes = [P(_Params), ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, d, d]
            lib.orc_matrices.argtypes = [P(_Params), ctypes.c_double, ctypes.c_double] + [d] * 11
            vp = ctypes.c_void_p
            lib.orc3_create.argtypes = [P(_Params3), P(vp)]
            lib.orc3_create.restype = ctypes.c_int
            lib.orc3_destroy.argtypes = [vp]
            lib.orc3_init.argtypes = [vp, d, d, d, d, d]
            lib.orc3_step.argtypes = [vp, ctypes.c_long]
            lib.orc3_fields.argtypes = [vp, d, d, d, d, d]
            lib.orc3_get_pops.argtypes = [vp, d, d]
            lib.orc3_set_pops.argtypes = [vp, d, d]
            lib.orc3_collide_node.argtypes = [P(_Params3), d, d, d, d]
            lib.orc3_equilibrium_node.argtypes = [P(_Params3)] + [ctypes.c_double] * 5 + [d, d]
            lib.orc3_collide_thermal_node.argtypes = [P(_Params3), d] + [ctypes.c_double] * 3 + [d]
            lib.orc3_matrices.argtypes = ([P(_Params3)] + [ctypes.c_double] * 3 + [d] * 9
                                          + [P(ctypes.c_int)] * 2)
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(p: dict, nx: int = 2, ny: int = 2) -> _Params:
    s = _Params()
    s.nx, s.ny = nx, ny
    for k in ("nu", "kappa", "g_beta", "T0", "rho0", "s_b", "s_3", "s_4", "lambda0", "lambda2",
              "cs2_T"):
        setattr(s, k, float(p.get(k, 1.0 if k == "lambda0" else 0.0)))
    s.Fv[0], s.Fv[1] = (float(v) for v in p["Fv"])
    for i in range(4):
        s.wall[i] = int(p["wall"][i])
        s.T_wall[i] = float(p["T_wall"][i])
    s.thermal_only = int(p.get("thermal_only", 0))
    uw = p.get("u_wall", ((0.0, 0.0),) * 4)
    for side in range(4):
        s.u_wall[2 * side], s.u_wall[2 * side + 1] = float(uw[side][0]), float(uw[side][1])
    return s


class Oracle:
    """One lattice stepped on the CPU in FP64. Fields are (ny, nx) float64 arrays. With
    params["thermal_only"] = 1 only the D2Q5 equation is stepped, with the velocity given to init()
    held fixed (the fields report that velocity)."""

    def __init__(self, nx: int, ny: int, params: dict):
        self._lib = _load()
        self.nx, self.ny, self.params = nx, ny, dict(params)
        self._p = _params(params, nx, ny)
        h = ctypes.c_void_p()
        rc = self._lib.orc_create(ctypes.byref(self._p), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle: invalid lattice {nx}x{ny} (code {rc})")
        self._h = h

    @classmethod
    def from_problem(cls, prob) -> "Oracle":
        o = cls(prob.nx, prob.ny, prob.params)
        o.init(prob.rho, prob.ux, prob.uy, prob.T)
        return o

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def init(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx)
                for a in (rho, ux, uy, T)]
        self._lib.orc_init(self._h, *[_ptr(a) for a in arrs])

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(self._lib.orc_steps(self._h))

    def fields(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        self._lib.orc_fields(self._h, *[_ptr(a) for a in out])
        return tuple(out)

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, self.ny, self.nx))
        self._lib.orc_get_pops(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == (5, self.ny, self.nx)
        self._lib.orc_set_pops(self._h, _ptr(f), _ptr(g))

    def nusselt(self, axis: int = 1) -> float:
        _, ux, uy, T = self.fields()
        return nusselt(ux, uy, T, self.params, axis)


def threads() -> int:
    """Number of OpenMP threads the oracle's node loops use (set with OMP_NUM_THREADS)."""
    return int(_load().orc_threads())


def collide_node(params: dict, f, g):
    """Post-collision populations (f*, g*) of one node (Eqs. 7-11, 16-21)."""
    lib = _load()
    p = _params(params)
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    fo, go = np.empty(9), np.empty(5)
    lib.orc_collide_node(ctypes.byref(p), _ptr(f), _ptr(g), _ptr(fo), _ptr(go))
    return fo, go


def collide_thermal_node(params: dict, g, ux, uy):
    """Post-collision D2Q5 populations of one node for a prescribed velocity (Eqs. 16-21)."""
    lib = _load()
    p = _params(params)
    g = np.ascontiguousarray(g, dtype=np.float64)
    go = np.empty(5)
    lib.orc_collide_thermal_node(ctypes.byref(p), _ptr(g), float(ux), float(uy), _ptr(go))
    return go


def equilibrium_node(params: dict, rho, ux, uy, T):
    """(f^eq, g^eq) = (M^-1 N(u)^-1 Gamma~eq, M_T^-1 N_T(u)^-1 Gamma~T,eq) at one node."""
    lib = _load()
    p = _params(params)
    f, g = np.empty(9), np.empty(5)
    lib.orc_equilibrium_node(ctypes.byref(p), float(rho), float(ux), float(uy), float(T), _ptr(f),
                             _ptr(g))
    return f, g


def matrices(params: dict, ux: float, uy: float) -> dict:
    """The matrices exactly as the oracle applies them (see clb_oracle.c)."""
    lib = _load()
    p = _params(params)
    shapes = dict(M=(9, 9), Minv=(9, 9), N=(9, 9), Ninv=(9, 9), MT=(5, 5), MTinv=(5, 5), NT=(5, 5),
                  NTinv=(5, 5), S=(9, 9), ST=(5, 5), wT=(5,))
    out = {k: np.empty(s) for k, s in shapes.items()}
    lib.orc_matrices(ctypes.byref(p), float(ux), float(uy),
                     *[_ptr(out[k]) for k in ("M", "Minv", "N", "Ninv", "MT", "MTinv", "NT",
                                               "NTinv", "S", "ST", "wT")])
    return out


def nusselt(ux, uy, T, params: dict, axis: int) -> float:
    """Eq. (29): Nu = 1 + <u_axis (T - T0)> H / (alpha dT), the average taken over the system.
    With walls halfway between nodes H is the node count along `axis` and the average is the plain
    mean over nodes. Wet walls lie on the end rows (columns) of nodes: along a wet direction the
    extent is one less and the average is the trapezoid rule (half weight on the two wall rows or
    columns), in every wet direction. dT is the difference of the wall temperatures on `axis`, the
    sign chosen so that heat flowing from the hot wall counts positive. alpha is the prescribed
    thermal diffusivity `kappa`."""
    u = ux if axis == 0 else uy
    ny, nx = T.shape
    lo, hi = (0, 1) if axis == 0 else (2, 3)
    Tl, Th = params["T_wall"][lo], params["T_wall"][hi]
    dT = abs(Tl - Th) or 1.0
    sign = 1.0 if Tl >= Th else -1.0
    q = u * (T - params["T0"])
    wx, wy = np.ones(nx), np.ones(ny)
    if params["wall"][0] == WET:
        wx[0] = wx[-1] = 0.5
    if params["wall"][2] == WET:
        wy[0] = wy[-1] = 0.5
    mean = float(np.sum(q * wy[:, None] * wx[None, :]) / (wx.sum() * wy.sum()))
    H = (wx if axis == 0 else wy).sum()
    return 1.0 + sign * mean * H / (params["kappa"] * dT)


def residual(prev, cur, u_ref: float, dT_ref: float) -> float:
    """E_R between two field snapshots (ux, uy, T) taken D steps apart (reading in module doc)."""
    pux, puy, pT = prev
    cux, cuy, cT = cur
    n = cT.size

    def ratio(num, den, ref):
        floor = n * (1e-3 * ref) ** 2
        den = max(den, floor)
        if num == 0.0:
            return 0.0
        return float(np.sqrt(num / den)) if den > 0 else float("inf")

    ru = ratio(float(np.sum((cux - pux) ** 2 + (cuy - puy) ** 2)),
               float(np.sum(cux ** 2 + cuy ** 2)), u_ref)
    rT = ratio(float(np.sum((cT - pT) ** 2)), float(np.sum(cT ** 2)), dT_ref)
    return max(ru, rT)


def run_to_steady(o: Oracle, tol: float, max_steps: int, interval: int = 100):
    """Step until E_R < tol (checked every `interval` steps) or `max_steps`. Returns (steps, E_R)."""
    p = o.params
    prev = o.fields()[1:]
    er = float("inf")
    while o.steps < max_steps:
        o.step(interval)
        cur = o.fields()[1:]
        er = residual(prev, cur, p.get("u_ref", 0.0), p.get("dT_ref", 0.0))
        prev = cur
        if er < tol:
            break
    return o.steps, er


# ------------------------------------------------------------------------------------------------
# Three-dimensional form (D3Q27 flow + D3Q7 temperature, clb3d_oracle.c). Fields are (nz, ny, nx)
# float64 arrays; params are those of the two-dimensional form plus s_5, s_6 (rates of the fifth-
# and sixth-order moments, default 1), Fv of length 3, g_axis (buoyancy along +g_axis, default 2)
# and six faces in wall / T_wall / u_wall (-x, +x, -y, +y, -z, +z).


def _params3(p: dict, nx: int = 1, ny: int = 1, nz: int = 1) -> _Params3:
    s = _Params3()
    s.nx, s.ny, s.nz = nx, ny, nz
    for k in ("nu", "kappa", "g_beta", "T0", "rho0", "s_b", "s_3", "s_4", "lambda2", "cs2_T"):
        setattr(s, k, float(p[k]))
    s.s_5 = float(p.get("s_5", 1.0))
    s.s_6 = float(p.get("s_6", 1.0))
    s.lambda0 = float(p.get("lambda0", 1.0))
    for i in range(3):
        s.Fv[i] = float(p["Fv"][i])
    s.g_axis = int(p.get("g_axis", 2))
    for i in range(6):
        s.wall[i] = int(p["wall"][i])
        s.T_wall[i] = float(p["T_wall"][i])
    uw = p.get("u_wall", ((0.0, 0.0, 0.0),) * 6)
    for face in range(6):
        for d in range(3):
            s.u_wall[3 * face + d] = float(uw[face][d])
    s.thermal_only = int(p.get("thermal_only", 0))
    return s


class Oracle3D:
    """One 3-D lattice stepped on the CPU in FP64."""

    def __init__(self, nx: int, ny: int, nz: int, params: dict):
        self._lib = _load()
        self.nx, self.ny, self.nz, self.params = nx, ny, nz, dict(params)
        self._p = _params3(params, nx, ny, nz)
        h = ctypes.c_void_p()
        rc = self._lib.orc3_create(ctypes.byref(self._p), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle: invalid lattice {nx}x{ny}x{nz} (code {rc})")
        self._h = h
        self.steps = 0

    @classmethod
    def from_problem(cls, prob) -> "Oracle3D":
        o = cls(prob.nx, prob.ny, prob.nz, prob.params)
        o.init(prob.rho, prob.ux, prob.uy, prob.uz, prob.T)
        return o

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc3_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def init(self, rho, ux, uy, uz, T):
        arrs = [np.ascontiguousarray(np.broadcast_to(a, self.shape), dtype=np.float64)
                for a in (rho, ux, uy, uz, T)]
        self._lib.orc3_init(self._h, *[_ptr(a) for a in arrs])
        self.steps = 0

    def step(self, n: int = 1):
        self._lib.orc3_step(self._h, int(n))
        self.steps += int(n)

    def fields(self):
        """(rho, ux, uy, uz, T), each (nz, ny, nx)."""
        out = [np.empty(self.shape) for _ in range(5)]
        self._lib.orc3_fields(self._h, *[_ptr(a) for a in out])
        return tuple(out)

    def populations(self):
        f = np.empty((27,) + self.shape)
        g = np.empty((7,) + self.shape)
        self._lib.orc3_get_pops(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (27,) + self.shape and g.shape == (7,) + self.shape
        self._lib.orc3_set_pops(self._h, _ptr(f), _ptr(g))

    def nusselt(self, axis: int = 2) -> float:
        _, ux, uy, uz, T = self.fields()
        return nusselt3((ux, uy, uz)[axis], T, self.params, axis)


def collide3_node(params: dict, f, g):
    """Post-collision (f*, g*) of one D3Q27 + D3Q7 node."""
    lib = _load()
    p = _params3(params)
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    fo, go = np.empty(27), np.empty(7)
    lib.orc3_collide_node(ctypes.byref(p), _ptr(f), _ptr(g), _ptr(fo), _ptr(go))
    return fo, go


def equilibrium3_node(params: dict, rho, ux, uy, uz, T):
    lib = _load()
    p = _params3(params)
    f, g = np.empty(27), np.empty(7)
    lib.orc3_equilibrium_node(ctypes.byref(p), float(rho), float(ux), float(uy), float(uz), float(T),
                              _ptr(f), _ptr(g))
    return f, g


def matrices3(params: dict, ux: float, uy: float, uz: float) -> dict:
    """M, Minv, N, S (27 x 27), MT, MTinv, NT, ST (7 x 7), wT (7), e27 (27 x 3), e7 (7 x 3)."""
    lib = _load()
    p = _params3(params)
    shapes = dict(M=(27, 27), Minv=(27, 27), N=(27, 27), S=(27, 27), MT=(7, 7), MTinv=(7, 7),
                  NT=(7, 7), ST=(7, 7), wT=(7,))
    out = {k: np.empty(s) for k, s in shapes.items()}
    e27 = np.empty((27, 3), dtype=np.int32)
    e7 = np.empty((7, 3), dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc3_matrices(ctypes.byref(p), float(ux), float(uy), float(uz),
                      *[_ptr(out[k]) for k in ("M", "Minv", "N", "S", "MT", "MTinv", "NT", "ST", "wT")],
                      e27.ctypes.data_as(ip), e7.ctypes.data_as(ip))
    out["e27"], out["e7"] = e27, e7
    return out


def nusselt3(u_axis, T, params: dict, axis: int) -> float:
    """Eq. (29) on a 3-D lattice: Nu = 1 + <u_axis (T - T0)> H / (alpha dT) over all nodes, H the
    node count along `axis` (walls halfway between nodes), dT the difference of the wall
    temperatures of that axis, heat from the hot wall counted positive."""
    H = T.shape[2 - axis]
    Tl, Th = params["T_wall"][2 * axis], params["T_wall"][2 * axis + 1]
    dT = abs(Tl - Th) or 1.0
    sign = 1.0 if Tl >= Th else -1.0
    return 1.0 + sign * float(np.mean(u_axis * (T - params["T0"]))) * H / (params["kappa"] * dT)


def residual3(prev, cur, u_ref: float, dT_ref: float) -> float:
    """E_R of the 3-D form between field snapshots (ux, uy, uz, T) taken some steps apart: the 2-D
    reading with u a 3-vector."""
    pux, puy, puz, pT = prev
    cux, cuy, cuz, cT = cur
    n = cT.size

    def ratio(num, den, ref):
        den = max(den, n * (1e-3 * ref) ** 2)
        if num == 0.0:
            return 0.0
        return float(np.sqrt(num / den)) if den > 0 else float("inf")

    ru = ratio(float(np.sum((cux - pux) ** 2 + (cuy - puy) ** 2 + (cuz - puz) ** 2)),
               float(np.sum(cux ** 2 + cuy ** 2 + cuz ** 2)), u_ref)
    rT = ratio(float(np.sum((cT - pT) ** 2)), float(np.sum(cT ** 2)), dT_ref)
    return max(ru, rT)


def collide3_thermal_node(params: dict, g, ux, uy, uz):
    """Post-collision D3Q7 populations of one node for a prescribed velocity."""
    lib = _load()
    p = _params3(params)
    g = np.ascontiguousarray(g, dtype=np.float64)
    go = np.empty(7)
    lib.orc3_collide_thermal_node(ctypes.byref(p), _ptr(g), float(ux), float(uy), float(uz), _ptr(go))
    return go
