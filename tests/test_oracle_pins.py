"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle by a route other than its own formulas: brute-force moment sums of
Eq. (5), the printed inverses of Appendix A, fixed points and conservation laws, analytic decay rates
(viscosity, Sec. 2.1; diffusivity in a moving frame, Sec. 3.1), the body-force Poiseuille and
pure-conduction profiles, and the Nusselt numbers of Table 1 (Sec. 3.3).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1710_10569_gb300 import workloads as W
from conftest import golden_path

P, D, A = W.WALL_PERIODIC, W.WALL_DIRICHLET, W.WALL_ADIABATIC

# Velocity set of Eq. (4), typed here from the paper for the brute-force sums.
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
ORDERS9 = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]  # Eq. (6)
ORDERS5 = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2)]                                  # Eq. (15)


def central_moments(f, ux, uy, orders, q):
    """Eq. (5b) by brute force: sum_i f_i (e_ix - u_x)^m (e_iy - u_y)^n."""
    return np.array([np.sum(f * (EX[:q] - ux) ** m * (EY[:q] - uy) ** n) for m, n in orders])


def raw_moments(f, orders, q):
    return np.array([np.sum(f * EX[:q] ** m * EY[:q] ** n) for m, n in orders])


def rand_params(rng, **kw):
    p = W.default_params(nu=float(rng.uniform(0.005, 0.2)), kappa=float(rng.uniform(0.005, 0.2)),
                         s_b=float(rng.uniform(0.5, 1.9)), s_3=float(rng.uniform(0.5, 1.9)),
                         s_4=float(rng.uniform(0.5, 1.9)), lambda2=float(rng.uniform(0.5, 1.9)),
                         g_beta=float(rng.uniform(0, 1e-2)), T0=float(rng.uniform(-0.2, 0.2)),
                         Fv=(float(rng.uniform(-1e-3, 1e-3)), float(rng.uniform(-1e-3, 1e-3))))
    p.update(kw)
    return p


def rand_pops(rng):
    f = rng.uniform(0.02, 0.5, 9)
    g = rng.uniform(-0.3, 0.6, 5)
    return f, g


def macro(f, g, p):
    """rho, u, T, F of Eqs. (3), (13), (23), typed from the paper for the checks."""
    rho = f.sum()
    T = g.sum()
    Fx = p["Fv"][0]
    Fy = p["Fv"][1] + p["rho0"] * p["g_beta"] * (T - p["T0"])
    ux = (np.dot(f, EX) + 0.5 * Fx) / rho
    uy = (np.dot(f, EY) + 0.5 * Fy) / rho
    return rho, ux, uy, T, Fx, Fy


# ----------------------------------------------------------------------------- transforms


def test_M_is_the_raw_moment_map():
    """Eq. (7a) against the definition of Eq. (5a) on random populations."""
    rng = np.random.default_rng(1)
    m = oracle.matrices(W.default_params(), 0.0, 0.0)
    for _ in range(20):
        f = rng.normal(size=9)
        np.testing.assert_allclose(m["M"] @ f, raw_moments(f, ORDERS9, 9), atol=1e-14)
        g = rng.normal(size=5)
        np.testing.assert_allclose(m["MT"] @ g, raw_moments(g, ORDERS5, 5), atol=1e-14)


def test_N_shifts_raw_to_central_moments():
    """N(u) M f equals the brute-force central moments of Eq. (5b) for random u. This fixes the
    k~02 row (the sign of its k01 entry is misprinted in Eq. 7b; Eq. 5b decides)."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        ux, uy = rng.uniform(-0.4, 0.4, 2)
        m = oracle.matrices(W.default_params(), ux, uy)
        f = rng.normal(size=9)
        np.testing.assert_allclose(m["N"] @ m["M"] @ f, central_moments(f, ux, uy, ORDERS9, 9),
                                   atol=1e-13)
        g = rng.normal(size=5)
        np.testing.assert_allclose(m["NT"] @ m["MT"] @ g, central_moments(g, ux, uy, ORDERS5, 5),
                                   atol=1e-13)


def test_inverses():
    """M^-1 M = I, N(u)^-1 = N(-u) (a shift by -u undoes a shift by u), and the 1-D tensor-product
    form of the D2Q9 inverse."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        ux, uy = rng.uniform(-0.4, 0.4, 2)
        m = oracle.matrices(W.default_params(), ux, uy)
        mneg = oracle.matrices(W.default_params(), -ux, -uy)
        np.testing.assert_allclose(m["Minv"] @ m["M"], np.eye(9), atol=1e-14)
        np.testing.assert_allclose(m["N"] @ m["Ninv"], np.eye(9), atol=1e-14)
        np.testing.assert_allclose(m["Ninv"], mneg["N"], atol=1e-14)
        np.testing.assert_allclose(m["NTinv"], mneg["NT"], atol=1e-14)
    # 1-D inverse of the moments (1, e, e^2) over e in (0, 1, -1): f0 = m0 - m2, f+- = (m2 +- m1)/2
    m = oracle.matrices(W.default_params(), 0.0, 0.0)
    inv1 = {0: np.array([1.0, 0.0, -1.0]), 1: np.array([0.0, 0.5, 0.5]), -1: np.array([0.0, -0.5, 0.5])}
    for i in range(9):
        for k, (a, b) in enumerate(ORDERS9):
            assert m["Minv"][i, k] == pytest.approx(inv1[int(EX[i])][a] * inv1[int(EY[i])][b], abs=1e-15)


def _read_appendix():
    mats, cur = {}, None
    for line in open(golden_path("appendixA_d2q5_inverses.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            mats[cur] = []
            continue
        mats[cur].append(line.split())
    return mats


def test_d2q5_inverses_match_appendix_a():
    mats = _read_appendix()
    rng = np.random.default_rng(4)
    for _ in range(10):
        ux, uy = rng.uniform(-0.4, 0.4, 2)
        m = oracle.matrices(W.default_params(), ux, uy)
        for key, name in (("MT_inv", "MTinv"), ("NT_inv", "NTinv")):
            ref = np.array([[eval(e, {"ux": ux, "uy": uy}) for e in row] for row in mats[key]])
            np.testing.assert_allclose(m[name], ref, atol=1e-14)


# ----------------------------------------------------------------------------- collision


def test_equilibrium_central_moments():
    """f^eq and g^eq carry exactly the central moments of Eqs. (9) and (20)."""
    rng = np.random.default_rng(5)
    p = W.default_params()
    cs2 = 1.0 / 3.0
    for _ in range(20):
        rho, T = rng.uniform(0.9, 1.1), rng.uniform(-1, 1)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        f, g = oracle.equilibrium_node(p, rho, ux, uy, T)
        np.testing.assert_allclose(central_moments(f, ux, uy, ORDERS9, 9),
                                   [rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 * cs2], atol=1e-14)
        c2 = p["cs2_T"]
        np.testing.assert_allclose(central_moments(g, ux, uy, ORDERS5, 5), [T, 0, 0, T * c2, T * c2],
                                   atol=1e-14)
    # rest weights at u = 0: D2Q9 4/9, 1/9, 1/36; D2Q5 with c_T,s^2 = 1/4: 1/2, 1/8
    f, g = oracle.equilibrium_node(p, 1.0, 0.0, 0.0, 1.0)
    np.testing.assert_allclose(f, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-15)
    np.testing.assert_allclose(g, [0.5] + [0.125] * 4, atol=1e-15)


def test_equilibrium_is_a_fixed_point_without_force():
    """With F = 0, collision maps (f^eq, g^eq) to itself for any relaxation rates."""
    rng = np.random.default_rng(6)
    for _ in range(30):
        p = rand_params(rng, g_beta=0.0, Fv=(0.0, 0.0))
        rho, T = rng.uniform(0.9, 1.1), rng.uniform(-1, 1)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        f, g = oracle.equilibrium_node(p, rho, ux, uy, T)
        fo, go = oracle.collide_node(p, f, g)
        np.testing.assert_allclose(fo, f, atol=1e-15)
        np.testing.assert_allclose(go, g, atol=1e-15)


def test_collision_conserves_mass_heat_and_adds_the_force():
    """sum f* = sum f, sum f* e = sum f e + F, sum g* = sum g (Eqs. 8, 11, 13, 19)."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        p = rand_params(rng)
        f, g = rand_pops(rng)
        rho, ux, uy, T, Fx, Fy = macro(f, g, p)
        fo, go = oracle.collide_node(p, f, g)
        assert fo.sum() == pytest.approx(f.sum(), abs=1e-14)
        assert np.dot(fo, EX) == pytest.approx(np.dot(f, EX) + Fx, abs=1e-14)
        assert np.dot(fo, EY) == pytest.approx(np.dot(f, EY) + Fy, abs=1e-14)
        assert go.sum() == pytest.approx(g.sum(), abs=1e-14)


def test_post_collision_central_moments():
    """Brute-force central moments of f* and g* (about the pre-collision u) equal Eq. (8) and
    Eq. (19) applied to brute-force central moments of f and g, for random rates."""
    rng = np.random.default_rng(8)
    cs2 = 1.0 / 3.0
    for _ in range(50):
        p = rand_params(rng)
        f, g = rand_pops(rng)
        rho, ux, uy, T, Fx, Fy = macro(f, g, p)
        fo, go = oracle.collide_node(p, f, g)
        s_nu = 1.0 / (3.0 * p["nu"] + 0.5)
        lam1 = 1.0 / (p["kappa"] / p["cs2_T"] + 0.5)
        k = central_moments(f, ux, uy, ORDERS9, 9)
        ko = central_moments(fo, ux, uy, ORDERS9, 9)
        sp, sm = 0.5 * (p["s_b"] + s_nu), 0.5 * (p["s_b"] - s_nu)
        a, b = k[3] - rho * cs2, k[4] - rho * cs2
        exp = [rho, k[1] + Fx, k[2] + Fy,
               k[3] - sp * a - sm * b, k[4] - sm * a - sp * b,
               (1 - s_nu) * k[5],
               (1 - p["s_3"]) * k[6] + (1 - p["s_3"] / 2) * cs2 * Fy,
               (1 - p["s_3"]) * k[7] + (1 - p["s_3"] / 2) * cs2 * Fx,
               (1 - p["s_4"]) * k[8] + p["s_4"] * rho * cs2 * cs2]
        np.testing.assert_allclose(ko, exp, atol=1e-14)
        kT = central_moments(g, ux, uy, ORDERS5, 5)
        koT = central_moments(go, ux, uy, ORDERS5, 5)
        c2 = p["cs2_T"]
        expT = [T, (1 - lam1) * kT[1], (1 - lam1) * kT[2],
                (1 - p["lambda2"]) * kT[3] + p["lambda2"] * T * c2,
                (1 - p["lambda2"]) * kT[4] + p["lambda2"] * T * c2]
        np.testing.assert_allclose(koT, expT, atol=1e-14)


# ----------------------------------------------------------------------------- lattice


def _run(nx, ny, p, rho, ux, uy, T, steps):
    o = oracle.Oracle(nx, ny, p)
    o.init(rho, ux, uy, T)
    o.step(steps)
    return o


def test_taylor_green_viscosity():
    """Kinetic energy of the Taylor-Green vortex decays as exp(-4 nu k^2 t) (nu = (1/s_nu - 1/2)/3,
    Sec. 2.1). Measured nu within 1% at N = 64 and the error shrinks with N (lattice error O(k^2))."""
    errs = []
    for n in (32, 64):
        prob = W.taylor_green(n, noise=0.0, T_amp=0.0)
        o = oracle.Oracle.from_problem(prob)
        _, ux, uy, _ = o.fields()
        e0 = np.sum(ux ** 2 + uy ** 2)
        steps = n * n // 4
        o.step(steps)
        _, ux, uy, _ = o.fields()
        e1 = np.sum(ux ** 2 + uy ** 2)
        k = 2 * math.pi / n
        nu = -math.log(e1 / e0) / (4 * k * k * steps)
        errs.append(abs(nu / 0.02 - 1))
    assert errs[1] < 0.01
    assert errs[1] < errs[0]


@pytest.mark.parametrize("Ma", [0.0, 0.1, 0.2, 0.3])
def test_diffusivity_in_moving_frame(Ma):
    """Sec. 3.1: a temperature wave T0 + B sin(phi (y - A t)) exp(-phi^2 alpha t) advected by the
    uniform flow u = (0, A), L = 100, alpha = 0.05, B = 0.01, T0 = 1. The measured diffusivity equals
    the prescribed alpha = (1/lambda1 - 1/2) c_T,s^2 independently of Ma = A / c_s, and the wave
    travels at speed A."""
    L, alpha, B = 100, 0.05, 0.01
    nx, ny = 2, L
    A_ = Ma * W.CS
    phi = 2 * math.pi / L
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    p = W.default_params(nu=0.05, kappa=alpha, T0=1.0)
    o = _run(nx, ny, p, np.ones((ny, nx)), np.zeros((ny, nx)), A_ * np.ones((ny, nx)),
             1.0 + B * np.sin(phi * y), 0)

    def mode():
        c = o.fields()[3][:, 0] - 1.0
        return np.sum(c * np.exp(-1j * phi * np.arange(ny))) * 2 / ny

    t1, t2 = 500, 2500
    o.step(t1)
    z1 = mode()
    o.step(t2 - t1)
    z2 = mode()
    a_meas = -math.log(abs(z2) / abs(z1)) / (phi * phi * (t2 - t1))
    assert a_meas == pytest.approx(alpha, rel=1e-3)
    # phase: sin(phi (y - A t)) has Fourier phase -phi A t - pi/2
    dphase = np.angle(z2 / z1)
    expect = -phi * A_ * (t2 - t1)
    assert abs((dphase - expect + math.pi) % (2 * math.pi) - math.pi) < 1e-3


def test_moving_uniform_flow_is_steady():
    """A uniform flow with uniform T in a periodic box is an exact steady state."""
    p = W.default_params(nu=0.03, kappa=0.03)
    n = 8
    o = _run(n, n, p, np.ones((n, n)), 0.1 * np.ones((n, n)), -0.15 * np.ones((n, n)),
             0.3 * np.ones((n, n)), 50)
    rho, ux, uy, T = o.fields()
    np.testing.assert_allclose(ux, 0.1, atol=1e-14)
    np.testing.assert_allclose(uy, -0.15, atol=1e-14)
    np.testing.assert_allclose(T, 0.3, atol=1e-14)
    np.testing.assert_allclose(rho, 1.0, atol=1e-14)


def _poiseuille_error(ny, s3):
    nu, F = 0.1, 1e-6
    p = W.default_params(nu=nu, kappa=0.05, Fv=(F, 0.0), wall=(P, P, A, A), s_3=s3)
    z = np.zeros((ny, 2))
    o = _run(2, ny, p, np.ones((ny, 2)), z, z, z, int(3 * ny * ny / nu))
    _, ux, uy, _ = o.fields()
    y = np.arange(ny)
    ua = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(uy)) < 1e-14
    return np.max(np.abs(ux[:, 0] - ua)) / np.max(ua)


def test_body_force_poiseuille_second_order():
    """Channel driven by F_v between halfway bounce-back walls: u(y) = F/(2 rho0 nu) (y+1/2)(ny-1/2-y).
    Relative error below 1e-3 at ny = 32 and second-order convergence from ny = 16."""
    for s3 in (1.0, 1.3):
        e16, e32 = _poiseuille_error(16, s3), _poiseuille_error(32, s3)
        assert e32 < 1e-3
        assert 3.5 < e16 / e32 < 4.5


@pytest.mark.parametrize("lambda2", [1.0, 1.5])
def test_conduction_between_dirichlet_walls_is_linear(lambda2):
    """g_beta = 0, walls at T = 0.7 (bottom) and -0.3 (top) halfway outside the end nodes: the
    steady temperature is the straight line through the wall values, to rounding."""
    ny = 20
    p = W.default_params(nu=0.1, kappa=0.1, wall=(P, P, D, D), T_wall=(0, 0, 0.7, -0.3),
                         lambda2=lambda2)
    z = np.zeros((ny, 2))
    o = _run(2, ny, p, np.ones((ny, 2)), z, z, z, 20000)
    T = o.fields()[3][:, 0]
    y = np.arange(ny)
    np.testing.assert_allclose(T, 0.7 - (y + 0.5) / ny, atol=1e-12)


def test_walls_conserve_mass_and_adiabatic_walls_conserve_heat():
    """Bounce-back walls conserve sum f exactly; with adiabatic walls on all sides sum g is
    conserved too (no flux through any wall)."""
    prob = W.random_problem(13, 11, seed=5, walls=(A, A, A, A))
    o = oracle.Oracle.from_problem(prob)
    f0, g0 = o.populations()
    o.step(300)
    f1, g1 = o.populations()
    assert f1.sum() == pytest.approx(f0.sum(), rel=1e-13)
    assert g1.sum() == pytest.approx(g0.sum(), rel=1e-13)


def _table1():
    rows = []
    for line in open(golden_path("table1_nusselt.txt")):
        if line.strip() and not line.startswith("#"):
            ra, an, pap, _ = line.split()
            rows.append((float(ra), float(an), float(pap)))
    return rows


def _rb_nusselt(Ra, Ma=0.3, nx=60, ny=30, tol=1e-6, max_steps=400000):
    prob = W.rayleigh_benard_table1(Ra, Ma=Ma, nx=nx, ny=ny)
    o = oracle.Oracle.from_problem(prob)
    hist = []
    while o.steps < max_steps:
        o.step(1000)
        hist.append(o.nusselt(1))
        if len(hist) > 3 and hist[-1] > 1.01 and abs(hist[-1] - hist[-2]) < tol \
                and abs(hist[-2] - hist[-3]) < tol:
            break
    return hist[-1], o


FAST_RA = (2500.0, 5000.0, 10000.0)


@pytest.mark.parametrize("row", [r for r in _table1() if r[0] in FAST_RA], ids=lambda r: f"Ra{r[0]:g}")
def test_table1_nusselt(row):
    """Sec. 3.3, Table 1: Nusselt numbers of Rayleigh-Benard convection at 60 x 30, Pr = 0.71,
    Ma = 0.3 within 0.5% of the analytic values (the paper's own errors are 0.08-0.41%)."""
    Ra, analytic, paper = row
    nu, _ = _rb_nusselt(Ra)
    assert nu == pytest.approx(analytic, rel=5e-3)
    assert nu == pytest.approx(paper, rel=6e-3)


@pytest.mark.slow
@pytest.mark.parametrize("row", [r for r in _table1() if r[0] not in FAST_RA], ids=lambda r: f"Ra{r[0]:g}")
def test_table1_nusselt_rest(row):
    """The remaining Table 1 rows. With walls halfway between nodes and only 30 nodes across, the
    error grows with Ra as the thermal boundary layer thins (about -2% at Ra = 5e4); bound 2.5%."""
    Ra, analytic, paper = row
    nu, _ = _rb_nusselt(Ra)
    assert nu == pytest.approx(analytic, rel=2.5e-2)


def test_wall_gradient_nusselt_matches_volume_average():
    """At steady state the conductive flux through the wall equals the convective + conductive
    flux averaged over the volume: Nu from the wall gradient (T_w - T(y=0)) / (1/2) H / dT matches
    Eq. (29) within the discretisation error."""
    nu_vol, o = _rb_nusselt(10000.0)
    T = o.fields()[3]
    grad_bottom = (0.5 - T[0, :]) / 0.5
    grad_top = (T[-1, :] - (-0.5)) / 0.5
    nu_wall = 0.5 * (grad_bottom.mean() + grad_top.mean()) * 30 / 1.0
    assert nu_wall == pytest.approx(nu_vol, rel=2e-2)


def test_subcritical_rayleigh_benard_decays_to_conduction():
    """Below the critical Rayleigh number (1707.76, Sec. 3.3) the convective roll decays: the
    horizontal velocity dies away and Nu -> 1. (An x-uniform odd-even mode of u_y of order 1e-5
    remains; it carries no roll and is neutral for lambda2 = lambda1, see the design notes.)"""
    prob = W.rayleigh_benard_table1(1500.0)
    o = oracle.Oracle.from_problem(prob)
    o.step(7500)
    v1 = np.max(np.abs(o.fields()[1]))
    o.step(7500)
    v2 = np.max(np.abs(o.fields()[1]))
    assert v2 < 0.5 * v1 and v1 < 1e-7
    assert o.nusselt(1) == pytest.approx(1.0, abs=1e-4)


def test_supercritical_rayleigh_benard_grows():
    """Above the critical Rayleigh number the same disturbance grows into a roll (Nu > 1)."""
    prob = W.rayleigh_benard_table1(2500.0)
    o = oracle.Oracle.from_problem(prob)
    o.step(7500)
    v1 = np.max(np.abs(o.fields()[1]))
    o.step(7500)
    v2 = np.max(np.abs(o.fields()[1]))
    assert v2 > 2 * v1


def test_nusselt_and_residual_definitions():
    """Nu = 1 for pure conduction (u = 0); E_R = 0 for equal snapshots and is scale-free."""
    n = 6
    T = np.random.default_rng(0).uniform(-0.5, 0.5, (n, n))
    z = np.zeros((n, n))
    p = W.default_params(kappa=0.1, wall=(P, P, D, D), T_wall=(0, 0, 0.5, -0.5))
    assert oracle.nusselt(z, z, T, p, 1) == 1.0
    u = np.random.default_rng(1).normal(size=(n, n))
    assert oracle.residual((u, u, T), (u, u, T), 0.0, 0.0) == 0.0
    r1 = oracle.residual((u, u, T), (1.1 * u, 1.1 * u, 1.1 * T), 0.0, 0.0)
    r2 = oracle.residual((5 * u, 5 * u, 5 * T), (5.5 * u, 5.5 * u, 5.5 * T), 0.0, 0.0)
    assert r1 == pytest.approx(r2, rel=1e-12)
    assert r1 == pytest.approx(0.1 / 1.1, rel=1e-12)


def test_residual_floor_branch_by_hand():
    """The floor N (1e-3 X_ref)^2 of the residual's denominator, worked by hand on a 2 x 2 lattice
    (N = 4) with u_ref = 0.1 and dT_ref = 1, so that a wrong factor, exponent or node count fails.
    Velocities of 1e-6 (sum |u|^2 = 8e-12) sit below the velocity floor 4 (1e-4)^2 = 4e-8; one u_x
    changing by 1e-6 gives sqrt(1e-12 / 4e-8) = 5e-3. T = 1e-4 everywhere (sum T^2 = 4e-8) sits
    below the temperature floor 4 (1e-3)^2 = 4e-6; one T changing by 2e-4 gives
    sqrt(4e-8 / 4e-6) = 0.1. With T = 1 (sum 4, above its floor) the same change gives
    sqrt(4e-8 / 4) = 1e-4 and the velocity's 5e-3 is the larger."""
    u = np.full((2, 2), 1e-6)
    u2 = u.copy()
    u2[0, 1] += 1e-6
    for T_level, expect in ((1e-4, 0.1), (1.0, 5e-3)):
        T = np.full((2, 2), T_level)
        T2 = T.copy()
        T2[1, 0] += 2e-4
        got = oracle.residual((u, u, T), (u2, u, T2), 0.1, 1.0)
        assert got == pytest.approx(expect, rel=1e-9)
    # the floor does not apply when X_ref = 0: the ratio is then relative to the fields alone
    T = np.full((2, 2), 1e-4)
    T2 = T.copy()
    T2[1, 0] += 2e-4
    got = oracle.residual((u, u, T), (u, u, T2), 0.0, 0.0)
    assert got == pytest.approx(math.sqrt(4e-8 / (3 * 1e-8 + 9e-8)), rel=1e-9)


# ----------------------------------------------------------------------------- thermal-only mode


def test_thermal_only_collision_equals_coupled_d2q5_part():
    """With the velocity the coupled step would compute, the thermal-only D2Q5 collision gives the
    same post-collision g (the two modes share Eqs. 16-21)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        p = rand_params(rng)
        f, g = rand_pops(rng)
        rho, ux, uy, T, Fx, Fy = macro(f, g, p)
        _, go = oracle.collide_node(p, f, g)
        got = oracle.collide_thermal_node(p, g, ux, uy)
        np.testing.assert_allclose(got, go, atol=1e-15)


def test_thermal_only_moving_frame_diffusivity():
    """Sec. 3.1 exactly as the paper runs it: only the D2Q5 equation, velocity (0, A) given, Ma = 0.3;
    the measured diffusivity equals alpha = 0.05 within 0.1%."""
    L, alpha, B = 100, 0.05, 0.01
    nx, ny = 2, L
    A_ = 0.3 * W.CS
    phi = 2 * math.pi / L
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    p = W.default_params(nu=0.05, kappa=alpha, T0=1.0)
    p["thermal_only"] = 1
    o = oracle.Oracle(nx, ny, p)
    o.init(np.ones((ny, nx)), np.zeros((ny, nx)), A_ * np.ones((ny, nx)), 1.0 + B * np.sin(phi * y))

    def amp():
        c = o.fields()[3][:, 0] - 1.0
        return abs(np.sum(c * np.exp(-1j * phi * np.arange(ny)))) * 2 / ny

    o.step(500)
    a1 = amp()
    o.step(2000)
    a2 = amp()
    assert -math.log(a2 / a1) / (phi * phi * 2000) == pytest.approx(alpha, rel=1e-3)
    np.testing.assert_allclose(o.fields()[2], A_)


def test_thermal_only_conserves_heat_in_a_closed_box():
    """Adiabatic walls and a divergence-free cellular flow: sum g is conserved exactly."""
    n = 24
    p = W.default_params(kappa=0.03, wall=(A, A, A, A))
    p["thermal_only"] = 1
    x, y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    k = math.pi / n
    ux = 0.05 * np.sin(k * x) * np.cos(k * y)
    uy = -0.05 * np.cos(k * x) * np.sin(k * y)
    T = np.random.default_rng(3).uniform(-0.5, 0.5, (n, n))
    o = oracle.Oracle(n, n, p)
    o.init(np.ones((n, n)), ux, uy, T)
    _, g0 = o.populations()
    o.step(400)
    _, g1 = o.populations()
    assert g1.sum() == pytest.approx(g0.sum(), rel=1e-13)


# ----------------------------------------------------------------------------- moving walls (Sec. 3.2)


def test_couette_flow_between_moving_walls_is_linear():
    """Top wall moving at u0, bottom at rest, no force: the steady profile is the straight line
    through the wall velocities, u = u0 (y + 1/2)/ny, to rounding."""
    ny, u0 = 16, 0.05
    p = W.default_params(nu=0.1, kappa=0.1, wall=(P, P, A, A), u_wall=((0, 0), (0, 0), (0, 0), (u0, 0)))
    z = np.zeros((ny, 2))
    o = _run(2, ny, p, np.ones((ny, 2)), z, z, z, 30000)
    _, ux, uy, _ = o.fields()
    np.testing.assert_allclose(ux[:, 0], u0 * (np.arange(ny) + 0.5) / ny, atol=1e-12)
    assert np.max(np.abs(uy)) < 1e-13


def _plate_errors(L, Re=10.0, Pr=0.71):
    prob = W.normal_plate_channel(L=L, Re=Re, Pr=Pr)
    o = oracle.Oracle.from_problem(prob)
    oracle.run_to_steady(o, 1e-11, 400000, 500)
    _, ux, uy, T = o.fields()
    ua, Ta = W.normal_plate_analytic(prob)
    Eu = np.sqrt(np.sum((ux[:, 0] - ua) ** 2) / np.sum(ua ** 2))
    ET = np.sqrt(np.sum((T[:, 0] - Ta) ** 2) / np.sum(Ta ** 2))
    return Eu, ET, np.max(np.abs(uy - prob.meta["v0"])) / prob.meta["v0"]


def test_normal_plate_channel_second_order():
    """Sec. 3.2: moving upper plate with normal injection/withdrawal and a temperature difference.
    The steady u and T profiles match the analytic exponential profiles (E_u, E_T < 1% at L = 30)
    and the errors fall with the second power of the grid spacing from L = 30 to 60 (the paper
    reports slopes of about 2); the normal velocity stays at v0."""
    e30 = _plate_errors(30)
    e60 = _plate_errors(60)
    assert e30[0] < 1e-2 and e30[1] < 1e-2
    assert e30[2] < 1e-4 and e60[2] < 1e-4
    for k in (0, 1):
        order = math.log(e30[k] / e60[k]) / math.log(2)
        assert 1.9 < order < 2.1


# ----------------------------------------------------------------------------- wet walls (the paper's own)


WET = W.WALL_WET


def test_wet_walls_reproduce_couette_poiseuille_and_conduction_exactly():
    """Walls on the end rows of nodes (H = ny - 1) with non-equilibrium bounce-back and
    non-equilibrium extrapolation: Couette flow and conduction are straight lines through the wall
    values and body-force Poiseuille flow is the parabola F/(2 nu) y (H - y), to rounding."""
    ny, u0 = 17, 0.05
    y = np.arange(ny)
    z = np.zeros((ny, 2))
    p = W.default_params(nu=0.1, kappa=0.1, wall=(P, P, WET, WET), T_wall=(0, 0, 0.3, -0.2),
                         u_wall=((0, 0), (0, 0), (0, 0), (u0, 0)))
    o = _run(2, ny, p, np.ones((ny, 2)), z, z, z, 40000)
    _, ux, uy, T = o.fields()
    np.testing.assert_allclose(ux[:, 0], u0 * y / (ny - 1), atol=1e-13)
    np.testing.assert_allclose(T[:, 0], 0.3 - 0.5 * y / (ny - 1), atol=1e-13)
    assert np.max(np.abs(uy)) < 1e-13
    F, nu = 1e-6, 0.1
    p = W.default_params(nu=nu, kappa=0.1, Fv=(F, 0), wall=(P, P, WET, WET))
    o = _run(2, ny, p, np.ones((ny, 2)), z, z, z, 40000)
    ux = o.fields()[1][:, 0]
    ua = F / (2 * nu) * y * (ny - 1 - y)
    assert np.max(np.abs(ux - ua)) / ua.max() < 1e-8


def _rb_wet_nusselt(Ra):
    prob = W.rayleigh_benard_table1(Ra, wet=True)
    o = oracle.Oracle.from_problem(prob)
    hist = []
    while o.steps < 200000:
        o.step(1000)
        hist.append(o.nusselt(1))
        if len(hist) > 3 and hist[-1] > 1.01 and abs(hist[-1] - hist[-2]) < 1e-6 \
                and abs(hist[-2] - hist[-3]) < 1e-6:
            break
    return hist[-1]


@pytest.mark.parametrize("row", [r for r in _table1() if r[0] in (5000.0, 10000.0)], ids=lambda r: f"Ra{r[0]:g}")
def test_table1_nusselt_with_the_papers_walls(row):
    """Table 1 with the paper's own wall conditions (walls on the 31 end-row nodes of a 60 x 30
    box): Nu within 0.2% of the analytic values and 0.4% of the paper's own numbers."""
    Ra, analytic, paper = row
    nu = _rb_wet_nusselt(Ra)
    assert nu == pytest.approx(analytic, rel=2e-3)
    assert nu == pytest.approx(paper, rel=4e-3)


@pytest.mark.slow
@pytest.mark.parametrize("row", [r for r in _table1() if r[0] in (2500.0, 3000.0)], ids=lambda r: f"Ra{r[0]:g}")
def test_table1_nusselt_with_the_papers_walls_rest(row):
    Ra, analytic, paper = row
    assert _rb_wet_nusselt(Ra) == pytest.approx(analytic, rel=2e-3)


def test_normal_plate_channel_with_the_papers_walls():
    """Sec. 3.2 with the paper's own walls (wet walls, L + 1 rows): E_u < 2e-3 and E_T < 5e-3 at
    L = 30, and the errors fall at order > 1.7 from L = 30 to 60."""
    out = []
    for L in (30, 60):
        prob = W.normal_plate_channel(L=L, Re=10.0, Pr=0.71, wet=True)
        o = oracle.Oracle.from_problem(prob)
        oracle.run_to_steady(o, 1e-11, 400000, 500)
        _, ux, _, T = o.fields()
        ua, Ta = W.normal_plate_analytic(prob)
        out.append((np.sqrt(np.sum((ux[:, 0] - ua) ** 2) / np.sum(ua ** 2)),
                    np.sqrt(np.sum((T[:, 0] - Ta) ** 2) / np.sum(Ta ** 2))))
    assert out[0][0] < 2e-3 and out[0][1] < 5e-3
    for k in (0, 1):
        assert math.log(out[0][k] / out[1][k]) / math.log(2) > 1.7


def test_hydrostatic_start_of_rayleigh_benard_is_at_rest():
    """The Rayleigh-Benard workloads start with the density in hydrostatic balance with the
    buoyancy of the conduction profile (c_s^2 d(rho)/dy = rho0 g beta (T - T0)). Under the oracle
    that state stays at rest to within discretisation error (no perturbation, Ra = 1e5 on 4 x 128,
    1,200 steps: max |u_y| < 3e-4 u_c), while a uniform initial density drives a vertical acoustic
    oscillation of the layer at least ten times stronger. A wrong sign or factor in the balance
    leaves an imbalance as large as the uniform start's."""
    peak = {}
    for hyd in (True, False):
        prob = W.rayleigh_benard(4, 128, Ra=1e5, perturb=0.0, hydrostatic=hyd)
        o = oracle.Oracle.from_problem(prob)
        m = 0.0
        for _ in range(6):
            o.step(200)
            m = max(m, float(np.max(np.abs(o.fields()[2]))))
        peak[hyd] = m / prob.meta["u_c"]
    assert peak[True] < 3e-4
    assert peak[False] > 10 * peak[True]
    # the balance itself: c_s^2 d(rho)/dy equals g beta (T - T0) of the conduction line
    prob = W.rayleigh_benard(4, 128, Ra=1e5, perturb=0.0)
    rho, T, gb = prob.rho[:, 0], prob.T[:, 0], prob.params["g_beta"]
    np.testing.assert_allclose(np.diff(rho) / 3.0, gb * 0.5 * (T[1:] + T[:-1]), rtol=1e-9, atol=1e-15)
    assert rho.mean() == pytest.approx(1.0, abs=1e-6)  # the continuous mean; nodes sample it at mid-cells


# ----------------------------------------------------------------------------- wet walls on x sides, corners

WET = W.WALL_WET


def _wet_problem(nx, ny, walls, seed, T_wall=(0.3, -0.2, 0.4, -0.1), u_wall=((0, 0),) * 4, g_beta=0.0,
                 Fv=(0.0, 0.0), thermal_only=0):
    rng = np.random.default_rng(seed)
    p = W.default_params(nu=0.05, kappa=0.04, g_beta=g_beta, Fv=Fv, wall=walls, T_wall=T_wall,
                         u_wall=u_wall, lambda2=1.1, s_b=1.2)
    if thermal_only:
        p = dict(p, thermal_only=1)
    rho = 1.0 + rng.uniform(-1e-3, 1e-3, (ny, nx))
    ux = rng.uniform(-0.02, 0.02, (ny, nx))
    uy = rng.uniform(-0.02, 0.02, (ny, nx))
    T = rng.uniform(-0.3, 0.3, (ny, nx))
    return p, rho, ux, uy, T


def test_wet_x_walls_are_the_transpose_of_wet_y_walls():
    """Wet walls on the x sides (reading r26) give exactly the transpose of the same problem with
    wet walls on the y sides (reading r19, pinned by the exact profiles and Table 1): the moment
    set, the relaxation matrix and the wall rules are symmetric under exchanging x and y, moving
    walls (tangential motion and normal injection) and a body force included (no buoyancy, which
    has a direction)."""
    nx, ny = 5, 9
    uw = ((0, 0), (0, 0), (0.03, 0.01), (-0.02, -0.01))
    p1, rho, ux, uy, T = _wet_problem(nx, ny, (P, P, WET, WET), 1, u_wall=uw, Fv=(2e-5, -1e-5))
    o1 = oracle.Oracle(nx, ny, p1)
    o1.init(rho, ux, uy, T)
    p2 = dict(p1, wall=(WET, WET, P, P), T_wall=(p1["T_wall"][2], p1["T_wall"][3], 0.0, 0.0),
              u_wall=((uw[2][1], uw[2][0]), (uw[3][1], uw[3][0]), (0, 0), (0, 0)), Fv=(-1e-5, 2e-5))
    o2 = oracle.Oracle(ny, nx, p2)
    o2.init(rho.T.copy(), uy.T.copy(), ux.T.copy(), T.T.copy())
    o1.step(60)
    o2.step(60)
    r1, x1, y1, t1 = o1.fields()
    r2, x2, y2, t2 = o2.fields()
    for a, b in ((r2, r1.T), (x2, y1.T), (y2, x1.T), (t2, t1.T)):
        np.testing.assert_allclose(a, b, atol=1e-14, rtol=0)


def test_wet_x_walls_exact_couette_and_conduction():
    """Between wet x walls (periodic y) the steady states are exact: Couette flow u_y linear
    between a resting wall and one moving along the wall, and T linear between the wall
    temperatures, the walls on the end columns (L = nx - 1)."""
    nx, ny = 9, 4
    p = W.default_params(nu=0.1, kappa=0.1, wall=(WET, WET, P, P), T_wall=(0.3, -0.2, 0, 0),
                         u_wall=((0, 0), (0, 0.02), (0, 0), (0, 0)))
    o = oracle.Oracle(nx, ny, p)
    o.init(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    o.step(6000)
    _, ux, uy, T = o.fields()
    s = np.arange(nx) / (nx - 1)
    np.testing.assert_allclose(uy, np.broadcast_to(0.02 * s, (ny, nx)), atol=1e-12)
    np.testing.assert_allclose(ux, 0.0, atol=1e-12)
    np.testing.assert_allclose(T, np.broadcast_to(0.3 - 0.5 * s, (ny, nx)), atol=1e-12)


def test_wet_box_rest_state_is_a_fixed_point():
    """A closed box of wet walls (all four sides, corners included) at rest with every wall at the
    fluid's temperature and no force stays exactly at rest."""
    nx, ny = 7, 6
    p = W.default_params(nu=0.05, kappa=0.04, wall=(WET,) * 4, T_wall=(0.25,) * 4)
    o = oracle.Oracle(nx, ny, p)
    o.init(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), 0.25))
    o.step(200)
    rho, ux, uy, T = o.fields()
    np.testing.assert_allclose(rho, 1.0, atol=1e-14)
    np.testing.assert_allclose(ux, 0.0, atol=1e-15)
    np.testing.assert_allclose(uy, 0.0, atol=1e-15)
    np.testing.assert_allclose(T, 0.25, atol=1e-14)


def test_wet_box_symmetries_through_the_corners():
    """A square closed box of wet walls: (a) without buoyancy, with the left and bottom walls hot
    and the others cold and transpose-symmetric initial fields, the state stays symmetric under
    exchanging x and y (each corner's rule, mean wall temperature and diagonal neighbour map onto
    its transposed corner's); (b) with buoyancy (hot bottom, cold top, side walls at T0) and
    mirror-symmetric initial fields, the state stays mirror-symmetric in x."""
    n = 10
    rng = np.random.default_rng(3)
    A_, B_, C_ = rng.uniform(-0.2, 0.2, (3, n, n))
    p = W.default_params(nu=0.05, kappa=0.04, wall=(WET,) * 4, T_wall=(0.5, -0.5, 0.5, -0.5))
    o = oracle.Oracle(n, n, p)
    o.init(1.0 + 1e-3 * (C_ + C_.T), 0.02 * B_, 0.02 * B_.T, A_ + A_.T)
    o.step(80)
    rho, ux, uy, T = o.fields()
    np.testing.assert_allclose(T, T.T, atol=1e-13)
    np.testing.assert_allclose(rho, rho.T, atol=1e-14)
    np.testing.assert_allclose(ux, uy.T, atol=1e-14)
    p = W.default_params(nu=0.05, kappa=0.04, g_beta=1e-3, wall=(WET,) * 4, T_wall=(0.0, 0.0, 0.5, -0.5))
    o = oracle.Oracle(n, n, p)
    Ts = A_ + A_[:, ::-1]
    o.init(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), Ts)
    o.step(300)
    rho, ux, uy, T = o.fields()
    assert np.max(np.abs(uy)) > 1e-4  # buoyancy has set the fluid moving
    np.testing.assert_allclose(T, T[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(uy, uy[:, ::-1], atol=1e-14)
    np.testing.assert_allclose(ux, -ux[:, ::-1], atol=1e-14)


@pytest.mark.parametrize("U", [0.0, 0.05])
def test_thermal_only_wet_walls_exact_conduction(U):
    """Thermal-only mode with wet y walls: with no velocity, or a uniform velocity along the walls
    (which does not advect an x-uniform field), T is linear between the wall temperatures."""
    nx, ny = 4, 11
    p = dict(W.default_params(kappa=0.1, wall=(P, P, WET, WET), T_wall=(0, 0, 0.4, -0.1)), thermal_only=1)
    o = oracle.Oracle(nx, ny, p)
    o.init(np.ones((ny, nx)), np.full((ny, nx), U), np.zeros((ny, nx)), np.zeros((ny, nx)))
    o.step(5000)
    T = o.fields()[3]
    np.testing.assert_allclose(T, np.broadcast_to((0.4 - 0.5 * np.arange(ny) / (ny - 1))[:, None], (ny, nx)),
                               atol=1e-12)
