"""Seeded synthetic problems shaped like the paper's workloads.

This module holds the problem statements only: lattice sizes, physical parameters derived from the
dimensionless groups the paper uses (Sec. 3.3: Ra = g*beta*dT*H^3/(nu*alpha), Pr = nu/alpha,
u_c = sqrt(g*beta*dT*H)), wall types and seeded initial fields. It contains none of the method's
arithmetic (no moments, no equilibria, no collision, no streaming), so that both the CUDA library and
the CPU oracle can be fed from it without sharing any of the computation.

Fields are float64 numpy arrays of shape (ny, nx), row-major (x fastest), node (x, y) at integer
coordinates; walls sit halfway between nodes, so a wall-bounded extent of n nodes has length n.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# wall kinds (per side, order -x, +x, -y, +y)
WALL_PERIODIC = 0
WALL_DIRICHLET = 1  # stationary no-slip wall at fixed temperature
WALL_ADIABATIC = 2  # stationary no-slip wall with zero heat flux
WALL_WET = 3        # wall on the end row of nodes (y sides, x periodic): the paper's own conditions

# population storage forms
STORAGE_F64 = 0
STORAGE_F32 = 1
STORAGE_F16DEV = 2
STORAGE_NAMES = {STORAGE_F64: "f64", STORAGE_F32: "f32", STORAGE_F16DEV: "f16dev"}

CS = 1.0 / math.sqrt(3.0)  # lattice sound speed of the D2Q9 lattice (Sec. 2.1, Eq. 9)


def default_params(**overrides) -> dict:
    """Default parameter set. High-order rates are 1 and the D2Q5 sound speed squared is 1/4,
    the defaults of Sec. 3 (first paragraph); the bulk rate s_b defaults to 1."""
    p = dict(
        nu=0.02, kappa=0.02, g_beta=0.0, T0=0.0, rho0=1.0,
        s_b=1.0, s_3=1.0, s_4=1.0, lambda0=1.0, lambda2=1.0, cs2_T=0.25,
        Fv=(0.0, 0.0),
        wall=(WALL_PERIODIC,) * 4, T_wall=(0.0,) * 4,
        storage=STORAGE_F64, T_ref=0.0, u_ref=0.0, dT_ref=0.0,
        u_wall=((0.0, 0.0),) * 4,
    )
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    params: dict
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    nu_axis: int = 1  # axis of the heat-flux for the Nusselt number (0 = x, 1 = y)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    def fields(self):
        return self.rho, self.ux, self.uy, self.T

    def with_storage(self, storage: int) -> "Problem":
        p = dict(self.params)
        p["storage"] = storage
        return dataclasses.replace(self, params=p)


def _grid(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def convection_params(H: float, Ra: float, Pr: float, u_c: float, dT: float = 1.0):
    """nu, alpha, g*beta from Ra, Pr and the characteristic velocity u_c = sqrt(g beta dT H)
    (Sec. 3.3: nu = u_c H sqrt(Pr/Ra) once u_c is fixed; alpha = nu/Pr)."""
    nu = u_c * H * math.sqrt(Pr / Ra)
    return nu, nu / Pr, u_c * u_c / (dT * H)


def taylor_green(n: int = 64, U: float = 0.01, nu: float = 0.02, kappa: float = 0.02,
                 T_amp: float = 0.01, noise: float = 1e-4, seed: int = 0, storage=STORAGE_F64,
                 ny: int | None = None) -> Problem:
    """Doubly periodic Taylor-Green vortex with a sinusoidal temperature, no gravity.
    u_x = -U cos(kx) sin(ky), u_y = U sin(kx) cos(ky), T = T_amp sin(kx) sin(ky), rho = 1, with
    independent seeded uniform noise of amplitude `noise` on u_x, u_y and T."""
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    ux = -U * np.cos(kx * x) * np.sin(ky * y) + rng.uniform(-noise, noise, (ny, nx))
    uy = U * np.sin(kx * x) * np.cos(ky * y) + rng.uniform(-noise, noise, (ny, nx))
    T = T_amp * np.sin(kx * x) * np.sin(ky * y) + rng.uniform(-noise, noise, (ny, nx))
    rho = np.ones((ny, nx))
    p = default_params(nu=nu, kappa=kappa, storage=storage, u_ref=U, dT_ref=T_amp)
    return Problem(f"taylor_green_{nx}x{ny}", nx, ny, p, rho, ux, uy, T, nu_axis=1,
                   meta=dict(U=U, seed=seed))


def cavity(n: int = 256, Ra: float = 1e5, Pr: float = 0.71, u_c: float = 0.1, noise: float = 1e-4,
           seed: int = 0, storage=STORAGE_F64, ny: int | None = None) -> Problem:
    """Differentially heated square cavity: left wall T=+0.5, right wall T=-0.5 (Dirichlet),
    top and bottom adiabatic, no-slip everywhere, fluid at rest, T = seeded noise of `noise`."""
    nx = n
    ny = n if ny is None else ny
    H = float(nx)  # heated walls are the x walls; the length scale is their distance
    nu, alpha, gb = convection_params(H, Ra, Pr, u_c)
    rng = np.random.default_rng(seed)
    T = rng.uniform(-noise, noise, (ny, nx))
    z = np.zeros((ny, nx))
    p = default_params(nu=nu, kappa=alpha, g_beta=gb, T0=0.0, storage=storage,
                       wall=(WALL_DIRICHLET, WALL_DIRICHLET, WALL_ADIABATIC, WALL_ADIABATIC),
                       T_wall=(0.5, -0.5, 0.0, 0.0), u_ref=u_c, dT_ref=1.0)
    return Problem(f"cavity_{nx}x{ny}_Ra{Ra:g}", nx, ny, p, np.ones((ny, nx)), z.copy(), z.copy(), T,
                   nu_axis=0, meta=dict(Ra=Ra, Pr=Pr, u_c=u_c, seed=seed))


def hydrostatic_density(s, g_beta: float, dT: float, H: float, rho0: float = 1.0):
    """Density in hydrostatic balance with the buoyancy of the conduction profile T - T0 =
    dT (1/2 - s) across a layer of height H (s = height / H in [0, 1]): the lattice equation of state
    p = c_s^2 rho turns dp/dy = rho0 g beta (T - T0) into c_s^2 d(rho)/dy = rho0 g beta (T - T0),
    integrated with the mean density rho0."""
    return rho0 * (1.0 + g_beta * dT * H / CS ** 2 * (s / 2 - s * s / 2 - 1.0 / 12.0))


def rayleigh_benard(nx: int = 2048, ny: int = 1024, Ra: float = 1e7, Pr: float = 0.71,
                    u_c: float = 0.1, perturb: float = 1e-3, seed: int = 0, storage=STORAGE_F64,
                    T0: float = 0.0, dT: float = 1.0, hydrostatic: bool = True) -> Problem:
    """Rayleigh-Benard convection: periodic in x, bottom wall T0+dT/2, top wall T0-dT/2, at rest,
    T = linear conduction profile + seeded uniform perturbation of amplitude `perturb`. With
    `hydrostatic` the density starts in balance with the buoyancy of the conduction profile, so the
    run starts from the conduction state; a uniform density is out of balance and sets the whole
    layer into a slow vertical acoustic oscillation that masks the onset of convection."""
    H = float(ny)
    nu, alpha, gb = convection_params(H, Ra, Pr, u_c, dT)
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    T = T0 + dT * (0.5 - (y + 0.5) / ny) + rng.uniform(-perturb, perturb, (ny, nx))
    rho = hydrostatic_density((y + 0.5) / ny, gb, dT, H) if hydrostatic else np.ones((ny, nx))
    z = np.zeros((ny, nx))
    p = default_params(nu=nu, kappa=alpha, g_beta=gb, T0=T0, storage=storage,
                       wall=(WALL_PERIODIC, WALL_PERIODIC, WALL_DIRICHLET, WALL_DIRICHLET),
                       T_wall=(0.0, 0.0, T0 + 0.5 * dT, T0 - 0.5 * dT), T_ref=T0, u_ref=u_c,
                       dT_ref=dT)
    return Problem(f"rayleigh_benard_{nx}x{ny}_Ra{Ra:g}", nx, ny, p, rho, z.copy(),
                   z.copy(), T, nu_axis=1, meta=dict(Ra=Ra, Pr=Pr, u_c=u_c, seed=seed))


def rayleigh_benard_table1(Ra: float, Ma: float = 0.3, nx: int = 60, ny: int = 30,
                           Pr: float = 0.71, storage=STORAGE_F64, wet: bool = False) -> Problem:
    """The Rayleigh-Benard set-up of Sec. 3.3 / Table 1: L x H = 60 x 30, Pr = 0.71,
    u_c = Ma * c_s, nu = Ma c_s H sqrt(Pr/Ra); density disturbed along the horizontal centre line,
    rho(x, H/2) = rho0 (1 + 0.001 cos(2 pi x / L)); the temperature starts from the conduction
    profile (the paper does not state it). Walls T = +-0.5 about T0 = 0 (a uniform shift of T from
    the paper's 1.05/0.95 about 1.0, with g*beta rescaled so Ra is unchanged)."""
    u_c = Ma * CS
    H = float(ny)
    if wet:
        ny = ny + 1  # walls on the end rows of nodes: H intervals need H + 1 rows
    nu, alpha, gb = convection_params(H, Ra, Pr, u_c)
    x, y = _grid(nx, ny)
    rho = np.ones((ny, nx))
    rho[ny // 2, :] = 1.0 + 0.001 * np.cos(2 * math.pi * np.arange(nx) / nx)
    T = 0.5 - (y / H if wet else (y + 0.5) / ny)
    z = np.zeros((ny, nx))
    kind = WALL_WET if wet else WALL_DIRICHLET
    p = default_params(nu=nu, kappa=alpha, g_beta=gb, T0=0.0, storage=storage,
                       wall=(WALL_PERIODIC, WALL_PERIODIC, kind, kind),
                       T_wall=(0.0, 0.0, 0.5, -0.5), u_ref=u_c, dT_ref=1.0)
    return Problem(f"rb_table1_Ra{Ra:g}" + ("_wet" if wet else ""), nx, ny, p, rho, z.copy(), z.copy(),
                   T, nu_axis=1, meta=dict(Ra=Ra, Pr=Pr, Ma=Ma, u_c=u_c))


def random_problem(nx: int, ny: int, seed: int, storage=STORAGE_F64, walls=None,
                   moving: bool = False) -> Problem:
    """A small problem with random-but-stable parameters and fields, used for parity sweeps
    (with `moving`, every wall also gets a random velocity of up to 0.05 per component)."""
    rng = np.random.default_rng(seed)
    if walls is None:
        walls = [(WALL_PERIODIC,) * 4,
                 (WALL_DIRICHLET, WALL_DIRICHLET, WALL_ADIABATIC, WALL_ADIABATIC),
                 (WALL_PERIODIC, WALL_PERIODIC, WALL_DIRICHLET, WALL_DIRICHLET),
                 (WALL_ADIABATIC, WALL_DIRICHLET, WALL_DIRICHLET, WALL_ADIABATIC)][seed % 4]
    T_wall = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 4))
    p = default_params(nu=float(rng.uniform(0.01, 0.1)), kappa=float(rng.uniform(0.01, 0.1)),
                       g_beta=float(rng.uniform(0.0, 1e-3)), T0=float(rng.uniform(-0.1, 0.1)),
                       s_b=float(rng.uniform(0.8, 1.6)), s_3=float(rng.uniform(0.8, 1.6)),
                       s_4=float(rng.uniform(0.8, 1.6)), lambda2=float(rng.uniform(0.8, 1.6)),
                       Fv=(float(rng.uniform(-1e-5, 1e-5)), float(rng.uniform(-1e-5, 1e-5))),
                       wall=tuple(walls), T_wall=T_wall, storage=storage, u_ref=0.05, dT_ref=1.0)
    rho = 1.0 + rng.uniform(-1e-3, 1e-3, (ny, nx))
    ux = rng.uniform(-0.05, 0.05, (ny, nx))
    uy = rng.uniform(-0.05, 0.05, (ny, nx))
    T = rng.uniform(-0.5, 0.5, (ny, nx))
    if moving:
        p["u_wall"] = tuple((float(a), float(b)) for a, b in rng.uniform(-0.05, 0.05, (4, 2)))
    return Problem(f"random_{nx}x{ny}_s{seed}", nx, ny, p, rho, ux, uy, T,
                   nu_axis=0 if walls[0] != WALL_PERIODIC else 1, meta=dict(seed=seed))


def normal_plate_channel(L: int = 50, Re: float = 10.0, Pr: float = 0.71, nu: float = 0.1,
                         nx: int = 5, storage=STORAGE_F64, lambda2=None, wet: bool = False) -> Problem:
    """Sec. 3.2: channel of width L, periodic in x; the bottom plate (y = 0, at rest, T_L = 0)
    injects a uniform normal flow v0 and the top plate (y = L, moving with u0, T_H = 1) withdraws it;
    u0 = v0 = Re nu / L. Walls lie halfway between nodes, so node j sits at y = j + 1/2 (with
    `wet`, the paper's own walls: on the end rows, node j at y = j, L + 1 rows). lambda2 defaults to
    the zero-numerical-slip value 12 (lambda1 - 2) / (lambda1 - 12) the paper uses."""
    ny = L + 1 if wet else L
    v0 = Re * nu / L
    alpha = nu / Pr
    lam1 = 1.0 / (alpha / 0.25 + 0.5)
    lam2 = 12 * (lam1 - 2) / (lam1 - 12) if lambda2 is None else lambda2
    y = (np.arange(ny) + (0.0 if wet else 0.5))[:, None] * np.ones((1, nx))
    kind = WALL_WET if wet else WALL_DIRICHLET
    p = default_params(nu=nu, kappa=alpha, lambda2=lam2, storage=storage,
                       wall=(WALL_PERIODIC, WALL_PERIODIC, kind, kind),
                       T_wall=(0.0, 0.0, 0.0, 1.0), u_wall=((0, 0), (0, 0), (0.0, v0), (v0, v0)),
                       u_ref=v0, dT_ref=1.0)
    ux = v0 * y / L
    uy = np.full((ny, nx), v0)
    T = y / L
    return Problem(f"normal_plate_L{L}_Re{Re:g}_Pr{Pr:g}" + ("_wet" if wet else ""), nx, ny, p,
                   np.ones((ny, nx)), ux, uy, T, nu_axis=1, meta=dict(L=L, Re=Re, Pr=Pr, v0=v0, wet=wet))


def normal_plate_analytic(prob: Problem):
    """Analytic steady profiles of Sec. 3.2 at the node heights: u/u0 = (exp(Re y/L) - 1)/(exp(Re) - 1)
    and (T - T_L)/dT = (exp(Re Pr y/L) - 1)/(exp(Re Pr) - 1); v = v0."""
    L, Re, Pr, v0 = (prob.meta[k] for k in ("L", "Re", "Pr", "v0"))
    y = np.arange(prob.ny) + (0.0 if prob.meta.get("wet") else 0.5)
    u = v0 * (np.exp(Re * y / L) - 1) / (math.exp(Re) - 1)
    T = (np.exp(Re * Pr * y / L) - 1) / (math.exp(Re * Pr) - 1)
    return u, T


def batch_cavities(count: int = 256, seed: int = 0, lo: int = 64, hi: int = 512,
                   Ra_range=(1e3, 1e6), Pr_range=(0.71, 7.0), u_c: float = 0.1,
                   nu_cap: float = 0.1, storage=STORAGE_F32) -> list[Problem]:
    """Independent side-heated cavities: edge log-uniform in [lo, hi], Ra log-uniform, Pr uniform.
    u_c is lowered where needed so that nu <= nu_cap (keeps the flow relaxation time moderate)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        Ra = math.exp(rng.uniform(math.log(Ra_range[0]), math.log(Ra_range[1])))
        Pr = float(rng.uniform(*Pr_range))
        uc = u_c
        nu = uc * n * math.sqrt(Pr / Ra)
        if nu > nu_cap:
            uc *= nu_cap / nu
        prob = cavity(n, Ra=Ra, Pr=Pr, u_c=uc, seed=seed * 100003 + k, storage=storage)
        prob.name = f"batch{k}_" + prob.name
        out.append(prob)
    return out


def request_trace(count: int = 64, seed: int = 0, rate_hz: float = 50.0, lo: int = 64,
                  hi: int = 512, Ra_range=(1e3, 1e6), storage=STORAGE_F32, nu_cap: float = 0.1,
                  rb_Ra_range=None):
    """A finite Poisson request stream: (arrival_time_s, Problem) pairs. Kind is uniform over
    periodic Taylor-Green, side-heated cavity and Rayleigh-Benard; edge log-uniform in [lo, hi];
    aspect ratio 1 or 2 with probability 1/2 each; Ra log-uniform in Ra_range (rb_Ra_range for
    the Rayleigh-Benard requests when given)."""
    rng = np.random.default_rng(seed)
    rb_lo, rb_hi = rb_Ra_range if rb_Ra_range is not None else Ra_range
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        kind = int(rng.integers(0, 3))
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        aspect = 1 + int(rng.integers(0, 2))
        Ra = math.exp(rng.uniform(math.log(Ra_range[0]), math.log(Ra_range[1])))
        s = seed * 1000003 + k
        if kind == 0:
            prob = taylor_green(n, ny=n * aspect if aspect == 2 else n, seed=s, storage=storage)
        elif kind == 1:
            uc = min(0.1, 0.1 * nu_cap / (0.1 * n * math.sqrt(0.71 / Ra)))
            prob = cavity(n, Ra=Ra, u_c=uc, ny=n * aspect, seed=s, storage=storage)
        else:
            if rb_Ra_range is not None:
                Ra = rb_lo * (rb_hi / rb_lo) ** (math.log(Ra / Ra_range[0]) / math.log(Ra_range[1] / Ra_range[0]))
            uc = min(0.1, 0.1 * nu_cap / (0.1 * n * math.sqrt(0.71 / Ra)))
            prob = rayleigh_benard(n * aspect, n, Ra=Ra, u_c=uc, seed=s, storage=storage)
        prob.name = f"req{k}_" + prob.name
        out.append((t, prob))
    return out


# ------------------------------------------------------------------------------------------------
# Three-dimensional problems (D3Q27 flow + D3Q7 temperature). Fields are float64 arrays of shape
# (nz, ny, nx), x fastest; faces in wall / T_wall are ordered -x, +x, -y, +y, -z, +z; buoyancy acts
# along +g_axis (z by default, gravity along -z).


def default_params3(**overrides) -> dict:
    """Defaults of the 3-D form: those of default_params, with the rates of the fifth- and
    sixth-order moments s_5 = s_6 = 1, a 3-vector Fv, g_axis = 2 and six faces."""
    p = dict(
        nu=0.02, kappa=0.02, g_beta=0.0, T0=0.0, rho0=1.0,
        s_b=1.0, s_3=1.0, s_4=1.0, s_5=1.0, s_6=1.0, lambda0=1.0, lambda2=1.0, cs2_T=0.25,
        Fv=(0.0, 0.0, 0.0), g_axis=2,
        wall=(WALL_PERIODIC,) * 6, T_wall=(0.0,) * 6, u_wall=((0.0, 0.0, 0.0),) * 6,
        storage=STORAGE_F64, T_ref=0.0, u_ref=0.0, dT_ref=0.0, thermal_only=0,
    )
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


@dataclasses.dataclass
class Problem3D:
    name: str
    nx: int
    ny: int
    nz: int
    params: dict
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    T: np.ndarray
    nu_axis: int = 2
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def fields(self):
        return self.rho, self.ux, self.uy, self.uz, self.T

    def with_storage(self, storage: int) -> "Problem3D":
        p = dict(self.params)
        p["storage"] = storage
        return dataclasses.replace(self, params=p)


def _grid3(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def rayleigh_benard3d(nx: int, ny: int, nz: int, Ra: float, Pr: float = 0.71, u_c: float = 0.1,
                      perturb: float = 1e-3, seed: int = 0, storage=STORAGE_F64,
                      hydrostatic: bool = True) -> Problem3D:
    """Rayleigh-Benard convection in a box periodic in x and y, Dirichlet walls on the z faces
    (T = +0.5 below, -0.5 above), H = nz, fluid at rest, T on the conduction line plus seeded
    uniform noise of amplitude `perturb`, density in hydrostatic balance with it (as in 2-D)."""
    H = float(nz)
    nu, alpha, gb = convection_params(H, Ra, Pr, u_c)
    rng = np.random.default_rng(seed)
    _, _, z = _grid3(nx, ny, nz)
    T = 0.5 - (z + 0.5) / H + rng.uniform(-perturb, perturb, (nz, ny, nx))
    rho = hydrostatic_density((z + 0.5) / H, gb, 1.0, H) if hydrostatic else np.ones((nz, ny, nx))
    zero = np.zeros((nz, ny, nx))
    p = default_params3(nu=nu, kappa=alpha, g_beta=gb, T0=0.0, storage=storage,
                        wall=(WALL_PERIODIC,) * 4 + (WALL_DIRICHLET,) * 2,
                        T_wall=(0.0,) * 4 + (0.5, -0.5), u_ref=u_c, dT_ref=1.0)
    return Problem3D(f"rayleigh_benard3d_{nx}x{ny}x{nz}", nx, ny, nz, p, rho,
                     zero.copy(), zero.copy(), zero.copy(), T, nu_axis=2,
                     meta=dict(Ra=Ra, Pr=Pr, u_c=u_c, seed=seed))


def batch_boxes3d(count: int = 48, seed: int = 0, lo: int = 24, hi: int = 128,
                  Ra_range=(1e3, 1e6), Pr_range=(0.71, 7.0), u_c: float = 0.1,
                  nu_cap: float = 0.1, storage=STORAGE_F32) -> list[Problem3D]:
    """Independent Rayleigh-Benard boxes for the 3-D batch: each extent log-uniform in [lo, hi]
    (drawn separately), Ra log-uniform, Pr uniform; u_c is lowered where needed so that
    nu <= nu_cap."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx, ny, nz = (int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3))
        Ra = math.exp(rng.uniform(math.log(Ra_range[0]), math.log(Ra_range[1])))
        Pr = float(rng.uniform(*Pr_range))
        uc = u_c
        nu = uc * nz * math.sqrt(Pr / Ra)
        if nu > nu_cap:
            uc *= nu_cap / nu
        prob = rayleigh_benard3d(nx, ny, nz, Ra=Ra, Pr=Pr, u_c=uc, seed=seed * 100003 + k, storage=storage)
        prob.name = f"box{k}_" + prob.name
        out.append(prob)
    return out


def taylor_green3d(n: int = 32, U: float = 0.01, nu: float = 0.02, kappa: float = 0.02,
                   T_amp: float = 0.01, noise: float = 1e-4, seed: int = 0,
                   storage=STORAGE_F64) -> Problem3D:
    """Triply periodic Taylor-Green vortex: u_x = U sin(kx) cos(ky) cos(kz), u_y = -U cos(kx)
    sin(ky) cos(kz), u_z = 0, T = T_amp sin(kx) sin(ky) sin(kz), rho = 1, plus seeded noise."""
    rng = np.random.default_rng(seed)
    x, y, z = _grid3(n, n, n)
    k = 2 * math.pi / n
    sh = (n, n, n)
    ux = U * np.sin(k * x) * np.cos(k * y) * np.cos(k * z) + rng.uniform(-noise, noise, sh)
    uy = -U * np.cos(k * x) * np.sin(k * y) * np.cos(k * z) + rng.uniform(-noise, noise, sh)
    uz = rng.uniform(-noise, noise, sh)
    T = T_amp * np.sin(k * x) * np.sin(k * y) * np.sin(k * z) + rng.uniform(-noise, noise, sh)
    p = default_params3(nu=nu, kappa=kappa, storage=storage, u_ref=U, dT_ref=T_amp)
    return Problem3D(f"taylor_green3d_{n}", n, n, n, p, np.ones(sh), ux, uy, uz, T,
                     meta=dict(U=U, seed=seed))


def random_problem3d(nx: int, ny: int, nz: int, seed: int = 0, storage=STORAGE_F64,
                     walls: tuple | None = None, moving: bool = False) -> Problem3D:
    """Seeded random parameters, faces and fields (for parity tests): rates drawn in their stable
    ranges, buoyancy along a random axis, each axis periodic or walled (Dirichlet or adiabatic per
    face), velocities up to 0.05, temperatures within +-0.5; with moving=True every wall face moves
    with a random velocity of up to 0.05 per component (tangential and normal)."""
    rng = np.random.default_rng(seed)
    if walls is None:
        walls = []
        for _ in range(3):
            if rng.uniform() < 0.5:
                walls += [WALL_PERIODIC, WALL_PERIODIC]
            else:
                walls += [int(rng.choice([WALL_DIRICHLET, WALL_ADIABATIC])) for _ in range(2)]
    sh = (nz, ny, nx)
    p = default_params3(nu=float(rng.uniform(0.01, 0.15)), kappa=float(rng.uniform(0.01, 0.15)),
                        g_beta=float(rng.uniform(0, 5e-3)), T0=float(rng.uniform(-0.1, 0.1)),
                        s_b=float(rng.uniform(0.8, 1.6)), s_3=float(rng.uniform(0.8, 1.6)),
                        s_4=float(rng.uniform(0.8, 1.6)), s_5=float(rng.uniform(0.8, 1.6)),
                        s_6=float(rng.uniform(0.8, 1.6)), lambda2=float(rng.uniform(0.8, 1.6)),
                        Fv=tuple(float(v) for v in rng.uniform(-1e-4, 1e-4, 3)),
                        g_axis=int(rng.integers(0, 3)), wall=tuple(walls),
                        T_wall=tuple(float(v) for v in rng.uniform(-0.5, 0.5, 6)),
                        storage=storage, T_ref=0.0, u_ref=0.05, dT_ref=0.5)
    if moving:
        p["u_wall"] = tuple((0.0, 0.0, 0.0) if walls[f] == WALL_PERIODIC else
                            tuple(float(v) for v in rng.uniform(-0.05, 0.05, 3)) for f in range(6))
    rho = 1.0 + rng.uniform(-1e-3, 1e-3, sh)
    ux, uy, uz = (rng.uniform(-0.05, 0.05, sh) for _ in range(3))
    T = rng.uniform(-0.5, 0.5, sh)
    return Problem3D(f"random3d_{nx}x{ny}x{nz}_s{seed}", nx, ny, nz, p, rho, ux, uy, uz, T,
                     meta=dict(seed=seed))
