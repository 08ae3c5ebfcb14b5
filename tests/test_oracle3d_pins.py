"""Pins of the three-dimensional FP64 oracle (D3Q27 flow + D3Q7 temperature).

The paper states the method in two dimensions and says it extends to three directly; the 3-D oracle
applies the same definitions on the 3-D lattices. These tests check it by routes other than its own
formulas: brute-force moment sums of the central-moment definition (Eq. 5), inverses, conservation
and fixed points, the two-dimensional oracle (itself pinned in test_oracle_pins.py) reproduced step
for step by fields uniform along any one axis, invariance under a permutation of the axes, decay
rates of shear and temperature waves in a moving frame (Secs. 2.1, 3.1), body-force Poiseuille flow
and steady conduction.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1710_10569_gb300 import workloads as W

P, D, A = W.WALL_PERIODIC, W.WALL_DIRICHLET, W.WALL_ADIABATIC
CS2 = 1.0 / 3.0
ORDERS27 = [(a, b, c) for c in range(3) for b in range(3) for a in range(3)]


def _sets():
    m = oracle.matrices3(W.default_params3(), 0.0, 0.0, 0.0)
    return m["e27"].astype(np.float64), m["e7"].astype(np.float64)


E27, E7 = _sets()


def central27(f, u, orders=ORDERS27):
    """Eq. (5b) by brute force on D3Q27: sum_i f_i prod_d (e_id - u_d)^a_d."""
    return np.array([np.sum(f * (E27[:, 0] - u[0]) ** a * (E27[:, 1] - u[1]) ** b *
                            (E27[:, 2] - u[2]) ** c) for a, b, c in orders])


def central7(g, u):
    orders = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2)]
    return np.array([np.sum(g * (E7[:, 0] - u[0]) ** a * (E7[:, 1] - u[1]) ** b *
                            (E7[:, 2] - u[2]) ** c) for a, b, c in orders])


def rand_params3(rng, **kw):
    p = W.default_params3(nu=float(rng.uniform(0.005, 0.2)), kappa=float(rng.uniform(0.005, 0.2)),
                          s_b=float(rng.uniform(0.5, 1.9)), s_3=float(rng.uniform(0.5, 1.9)),
                          s_4=float(rng.uniform(0.5, 1.9)), s_5=float(rng.uniform(0.5, 1.9)),
                          s_6=float(rng.uniform(0.5, 1.9)), lambda2=float(rng.uniform(0.5, 1.9)),
                          g_beta=float(rng.uniform(0, 1e-2)), T0=float(rng.uniform(-0.2, 0.2)),
                          g_axis=int(rng.integers(0, 3)),
                          Fv=tuple(float(v) for v in rng.uniform(-1e-3, 1e-3, 3)))
    p.update(kw)
    return p


def macro3(f, g, p):
    rho, T = f.sum(), g.sum()
    F = np.array(p["Fv"], dtype=np.float64)
    F[p["g_axis"]] += p["rho0"] * p["g_beta"] * (T - p["T0"])
    u = (f @ E27 + 0.5 * F) / rho
    return rho, u, T, F


# ----------------------------------------------------------------------------- transforms


def test_velocity_sets_are_the_full_3d_lattices():
    assert sorted(map(tuple, E27.astype(int))) == sorted(itertools.product((-1, 0, 1), repeat=3))
    assert sorted(map(tuple, E7.astype(int))) == sorted(
        [(0, 0, 0)] + [tuple(s * np.eye(3, dtype=int)[d]) for d in range(3) for s in (1, -1)])


def test_M_is_the_raw_moment_map_and_invertible():
    m = oracle.matrices3(W.default_params3(), 0.0, 0.0, 0.0)
    brute = np.array([E27[:, 0] ** a * E27[:, 1] ** b * E27[:, 2] ** c for a, b, c in ORDERS27])
    np.testing.assert_array_equal(m["M"], brute)
    np.testing.assert_allclose(m["M"] @ m["Minv"], np.eye(27), atol=1e-14)
    np.testing.assert_allclose(m["MT"] @ m["MTinv"], np.eye(7), atol=1e-15)


def test_N_shifts_raw_to_central_moments():
    rng = np.random.default_rng(1)
    for _ in range(20):
        u = rng.uniform(-0.3, 0.3, 3)
        m = oracle.matrices3(W.default_params3(), *u)
        f = rng.uniform(0.0, 0.2, 27)
        g = rng.uniform(-0.2, 0.5, 7)
        np.testing.assert_allclose(m["N"] @ (m["M"] @ f), central27(f, u), atol=1e-14)
        np.testing.assert_allclose(m["NT"] @ (m["MT"] @ g), central7(g, u), atol=1e-15)
        back = oracle.matrices3(W.default_params3(), *(-u))
        np.testing.assert_allclose(m["N"] @ back["N"], np.eye(27), atol=1e-14)
        np.testing.assert_allclose(m["NT"] @ back["NT"], np.eye(7), atol=1e-15)


def test_d3q7_rest_weights():
    """g^eq at T = 1, u = 0 puts cs2_T / 2 on each moving direction (second moment cs2_T per axis)
    and the rest on the rest population."""
    for c2 in (0.25, 1.0 / 6.0):
        wT = oracle.matrices3(W.default_params3(cs2_T=c2), 0, 0, 0)["wT"]
        np.testing.assert_allclose(wT, [1 - 3 * c2] + [c2 / 2] * 6, atol=1e-16)


def test_equilibrium_central_moments_are_the_lattice_maxwellian():
    """Brute-force central moments of f^eq about u: rho prod_d m(a_d) with m = (1, 0, cs2); of g^eq:
    (T, 0, 0, 0, cs2_T T x3)."""
    rng = np.random.default_rng(2)
    mw = (1.0, 0.0, CS2)
    for _ in range(20):
        p = rand_params3(rng)
        rho, T = rng.uniform(0.9, 1.1), rng.uniform(-0.5, 0.5)
        u = rng.uniform(-0.2, 0.2, 3)
        f, g = oracle.equilibrium3_node(p, rho, *u, T)
        exp = [rho * mw[a] * mw[b] * mw[c] for a, b, c in ORDERS27]
        np.testing.assert_allclose(central27(f, u), exp, atol=1e-15)
        c2 = p["cs2_T"]
        np.testing.assert_allclose(central7(g, u), [T, 0, 0, 0, c2 * T, c2 * T, c2 * T], atol=1e-15)


def test_equilibrium_is_a_fixed_point_without_force():
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = rand_params3(rng, g_beta=0.0, Fv=(0.0, 0.0, 0.0))
        u = rng.uniform(-0.2, 0.2, 3)
        f, g = oracle.equilibrium3_node(p, rng.uniform(0.9, 1.1), *u, rng.uniform(-0.5, 0.5))
        fo, go = oracle.collide3_node(p, f, g)
        np.testing.assert_allclose(fo, f, atol=1e-15)
        np.testing.assert_allclose(go, g, atol=1e-15)


def test_collision_conserves_mass_heat_and_adds_the_force():
    rng = np.random.default_rng(4)
    for _ in range(30):
        p = rand_params3(rng)
        f = rng.uniform(0.005, 0.1, 27)
        g = rng.uniform(-0.1, 0.2, 7)
        rho, u, T, F = macro3(f, g, p)
        fo, go = oracle.collide3_node(p, f, g)
        assert fo.sum() == pytest.approx(f.sum(), abs=1e-15)
        np.testing.assert_allclose(fo @ E27, f @ E27 + F, atol=1e-15)
        assert go.sum() == pytest.approx(g.sum(), abs=1e-15)


def test_second_order_relaxation_splits_trace_and_deviators():
    """Brute-force central moments about the pre-collision u: the trace of the normal second
    moments relaxes with s_b, each deviator and each off-diagonal second moment with s_nu
    (nu = (1/s_nu - 1/2) / 3), the third-, fourth-, fifth- and sixth-order moments with s_3 .. s_6
    towards the lattice Maxwellian, plus (1 - s/2) times the forcing moment wherever exactly one
    index is 1."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        p = rand_params3(rng)
        f = rng.uniform(0.005, 0.1, 27)
        g = rng.uniform(-0.1, 0.2, 7)
        rho, u, T, F = macro3(f, g, p)
        fo, _ = oracle.collide3_node(p, f, g)
        s_nu = 1.0 / (3.0 * p["nu"] + 0.5)
        k, ko = central27(f, u), central27(fo, u)
        idx = {o: i for i, o in enumerate(ORDERS27)}
        nrm = [idx[(2, 0, 0)], idx[(0, 2, 0)], idx[(0, 0, 2)]]
        tr, tro = sum(k[i] for i in nrm), sum(ko[i] for i in nrm)
        assert tro - 3 * rho * CS2 == pytest.approx((1 - p["s_b"]) * (tr - 3 * rho * CS2), abs=1e-14)
        dev = k[nrm[0]] - k[nrm[1]]
        assert ko[nrm[0]] - ko[nrm[1]] == pytest.approx((1 - s_nu) * dev, abs=1e-14)
        for o in [(1, 1, 0), (1, 0, 1), (0, 1, 1)]:
            assert ko[idx[o]] == pytest.approx((1 - s_nu) * k[idx[o]], abs=1e-14)
        # third order with one index 1 and one 2: the force of the axis with index 1 enters
        for o in [(2, 1, 0), (0, 2, 1), (1, 0, 2)]:
            d = o.index(1)
            exp = (1 - p["s_3"]) * k[idx[o]] + (1 - p["s_3"] / 2) * CS2 * F[d]
            assert ko[idx[o]] == pytest.approx(exp, abs=1e-14)
        assert ko[idx[(1, 1, 1)]] == pytest.approx((1 - p["s_3"]) * k[idx[(1, 1, 1)]], abs=1e-14)
        # fourth order: (2,2,0)-type relax towards rho cs2^2, (2,1,1)-type towards 0
        for o in [(2, 2, 0), (0, 2, 2), (2, 0, 2)]:
            exp = (1 - p["s_4"]) * k[idx[o]] + p["s_4"] * rho * CS2 ** 2
            assert ko[idx[o]] == pytest.approx(exp, abs=1e-14)
        for o in [(2, 1, 1), (1, 2, 1), (1, 1, 2)]:
            assert ko[idx[o]] == pytest.approx((1 - p["s_4"]) * k[idx[o]], abs=1e-14)
        # fifth order: the axis with index 1 carries (1 - s_5/2) cs2^2 F_d
        for o in [(1, 2, 2), (2, 1, 2), (2, 2, 1)]:
            d = o.index(1)
            exp = (1 - p["s_5"]) * k[idx[o]] + (1 - p["s_5"] / 2) * CS2 ** 2 * F[d]
            assert ko[idx[o]] == pytest.approx(exp, abs=1e-14)
        exp6 = (1 - p["s_6"]) * k[idx[(2, 2, 2)]] + p["s_6"] * rho * CS2 ** 3
        assert ko[idx[(2, 2, 2)]] == pytest.approx(exp6, abs=1e-14)


# ----------------------------------------------------------------------------- lattice


def _embed(axis_uniform):
    """Map of the 2-D axes (x, y) onto 3-D axes, the remaining axis being uniform."""
    return {2: (0, 1), 0: (1, 2), 1: (2, 0)}[axis_uniform]


@pytest.mark.parametrize("uniform", [0, 1, 2])
def test_fields_uniform_along_an_axis_reproduce_the_2d_oracle(uniform):
    """A 3-D lattice whose fields do not vary along one axis (two periodic nodes along it, no
    velocity along it) steps exactly like the two-dimensional D2Q9 + D2Q5 oracle, in every
    orientation: the populations summed along that axis are D2Q9 / D2Q5 populations. Needs
    s_b = s_nu (the 3-D bulk rate acts on the trace of three normal moments, the 2-D one on two)."""
    rng = np.random.default_rng(10 + uniform)
    nx, ny = 6, 5
    nu = 0.06
    s_nu = 1.0 / (3 * nu + 0.5)
    p2 = W.default_params(nu=nu, kappa=0.04, g_beta=4e-3, T0=0.05, s_b=s_nu, s_3=1.3, s_4=0.9,
                          lambda2=1.2, Fv=(1e-4, -5e-5), wall=(P, P, D, A), T_wall=(0, 0, 0.4, -0.3))
    rho = 1.0 + rng.uniform(-1e-3, 1e-3, (ny, nx))
    ux, uy = rng.uniform(-0.05, 0.05, (ny, nx)), rng.uniform(-0.05, 0.05, (ny, nx))
    T = rng.uniform(-0.4, 0.4, (ny, nx))
    o2 = oracle.Oracle(nx, ny, p2)
    o2.init(rho, ux, uy, T)

    ax, ay = _embed(uniform)
    n3 = [0, 0, 0]
    n3[ax], n3[ay], n3[uniform] = nx, ny, 2
    walls, twall = [P] * 6, [0.0] * 6
    walls[2 * ay], walls[2 * ay + 1] = D, A
    twall[2 * ay], twall[2 * ay + 1] = 0.4, -0.3
    Fv = [0.0, 0.0, 0.0]
    Fv[ax], Fv[ay] = 1e-4, -5e-5
    p3 = W.default_params3(nu=nu, kappa=0.04, g_beta=4e-3, T0=0.05, s_b=s_nu, s_3=1.3, s_4=0.9,
                           s_5=1.7, s_6=0.6, lambda2=1.2, Fv=tuple(Fv), g_axis=ay, wall=tuple(walls),
                           T_wall=tuple(twall))

    def lift(a2):
        """(ny, nx) array on axes (ay, ax) -> (nz, ny, nx) array uniform along `uniform`."""
        full = np.empty(n3[::-1])
        for idx in itertools.product(*[range(n) for n in n3[::-1]]):
            c = idx[::-1]  # (x, y, z)
            full[idx] = a2[c[ay], c[ax]]
        return full

    vel = [None, None, None]
    vel[ax], vel[ay], vel[uniform] = ux, uy, np.zeros_like(ux)
    o3 = oracle.Oracle3D(*n3, p3)
    o3.init(lift(rho), *[lift(v) for v in vel], lift(T))
    for _ in range(3):
        o2.step(10)
        o3.step(10)
        r2, ux2, uy2, T2 = o2.fields()
        r3, *u3, T3 = o3.fields()
        np.testing.assert_allclose(r3, lift(r2), atol=1e-13)
        np.testing.assert_allclose(u3[ax], lift(ux2), atol=1e-13)
        np.testing.assert_allclose(u3[ay], lift(uy2), atol=1e-13)
        np.testing.assert_allclose(u3[uniform], 0.0, atol=1e-15)
        np.testing.assert_allclose(T3, lift(T2), atol=1e-13)


def test_stepping_commutes_with_a_permutation_of_the_axes():
    """Relabelling the axes (x, y, z) -> (y, z, x) of the fields, velocities, faces, force and
    buoyancy axis, stepping, and relabelling back gives the original run: no axis is special."""
    prob = W.random_problem3d(4, 5, 3, seed=7, walls=(P, P, D, A, A, D))
    prob.params["g_axis"] = 1
    o = oracle.Oracle3D.from_problem(prob)
    o.step(12)
    r, ux, uy, uz, T = o.fields()

    def perm(a):  # new (x, y, z) = old (y, z, x); arrays are (z, y, x)
        return np.ascontiguousarray(a.transpose(2, 0, 1))

    p = dict(prob.params)
    w, tw, F = p["wall"], p["T_wall"], p["Fv"]
    p["wall"] = (w[2], w[3], w[4], w[5], w[0], w[1])
    p["T_wall"] = (tw[2], tw[3], tw[4], tw[5], tw[0], tw[1])
    p["Fv"] = (F[1], F[2], F[0])
    p["g_axis"] = {0: 2, 1: 0, 2: 1}[prob.params["g_axis"]]
    q = oracle.Oracle3D(prob.ny, prob.nz, prob.nx, p)
    q.init(perm(prob.rho), perm(prob.uy), perm(prob.uz), perm(prob.ux), perm(prob.T))
    q.step(12)
    r2, vx, vy, vz, T2 = q.fields()
    np.testing.assert_allclose(r2, perm(r), atol=1e-14)
    np.testing.assert_allclose(vx, perm(uy), atol=1e-14)
    np.testing.assert_allclose(vy, perm(uz), atol=1e-14)
    np.testing.assert_allclose(vz, perm(ux), atol=1e-14)
    np.testing.assert_allclose(T2, perm(T), atol=1e-14)


def _mode(a, k, n):
    return np.sum(a * np.exp(-1j * k * np.arange(n))) * 2 / n


@pytest.mark.parametrize("adv", [(0.0, 0.0, 0.0), (0.1, -0.1, 0.1)])
def test_shear_wave_decays_at_the_prescribed_viscosity_in_a_moving_frame(adv):
    """u_x = U sin(k z) on a 1 x 1 x 64 periodic lattice decays as exp(-nu k^2 t) (nu =
    (1/s_nu - 1/2)/3) and is carried along z at the advection speed; with a uniform advection
    (0.1, -0.1, 0.1) (Ma 0.3 in magnitude) the measured nu stays within 0.2% of the prescribed one
    (Galilean invariance of the central-moment collision)."""
    L, nu, U = 64, 0.05, 1e-3
    p = W.default_params3(nu=nu, kappa=0.05)
    z = np.arange(L, dtype=np.float64).reshape(L, 1, 1)
    k = 2 * math.pi / L
    o = oracle.Oracle3D(1, 1, L, p)
    o.init(1.0, adv[0] + U * np.sin(k * z), adv[1], adv[2], 0.0)
    o.step(200)
    z1 = _mode(o.fields()[1][:, 0, 0] - adv[0], k, L)
    o.step(1000)
    z2 = _mode(o.fields()[1][:, 0, 0] - adv[0], k, L)
    nu_meas = -math.log(abs(z2) / abs(z1)) / (k * k * 1000)
    assert nu_meas == pytest.approx(nu, rel=2e-3)
    dphase = np.angle(z2 / z1)
    assert abs((dphase + k * adv[2] * 1000 + math.pi) % (2 * math.pi) - math.pi) < 2e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_temperature_wave_diffusivity_in_a_moving_frame(axis):
    """Sec. 3.1 in 3-D: a temperature wave along `axis` advected by u = (0.1, 0.12, -0.08) keeps the
    prescribed diffusivity alpha = (1/lambda1 - 1/2) cs2_T within 0.1% and travels at u_axis."""
    L, alpha, B = 60, 0.05, 0.01
    n3 = [1, 1, 1]
    n3[axis] = L
    adv = (0.1, 0.12, -0.08)
    p = W.default_params3(nu=0.05, kappa=alpha, T0=1.0)
    c = np.arange(L, dtype=np.float64)
    shape = n3[::-1]
    Tline = 1.0 + B * np.sin(2 * math.pi * c / L)
    T = Tline.reshape([L if (2 - i) == axis else 1 for i in range(3)])
    o = oracle.Oracle3D(*n3, p)
    o.init(1.0, adv[0], adv[1], adv[2], np.broadcast_to(T, shape))
    k = 2 * math.pi / L
    o.step(300)
    z1 = _mode(o.fields()[4].reshape(-1) - 1.0, k, L)
    o.step(1500)
    z2 = _mode(o.fields()[4].reshape(-1) - 1.0, k, L)
    a_meas = -math.log(abs(z2) / abs(z1)) / (k * k * 1500)
    assert a_meas == pytest.approx(alpha, rel=1e-3)
    dphase = np.angle(z2 / z1)
    assert abs((dphase + k * adv[axis] * 1500 + math.pi) % (2 * math.pi) - math.pi) < 2e-3


def _poiseuille3_error(nz, s3):
    nu, F = 0.1, 1e-6
    p = W.default_params3(nu=nu, kappa=0.05, Fv=(F, 0.0, 0.0), s_3=s3,
                          wall=(P, P, P, P, A, A))
    o = oracle.Oracle3D(1, 1, nz, p)
    o.init(1.0, 0.0, 0.0, 0.0, 0.0)
    o.step(int(3 * nz * nz / nu))
    _, ux, uy, uz, _ = o.fields()
    zc = np.arange(nz)
    ua = F / (2 * nu) * (zc + 0.5) * (nz - 0.5 - zc)
    assert np.max(np.abs(uz)) < 1e-14 and np.max(np.abs(uy)) < 1e-14
    return np.max(np.abs(ux[:, 0, 0] - ua)) / np.max(ua)


def test_body_force_poiseuille_between_z_walls():
    """u_x(z) = F/(2 rho0 nu) (z+1/2)(nz-1/2-z) between halfway bounce-back walls: relative error
    below 1e-3 at nz = 32 and second-order convergence from nz = 16."""
    for s3 in (1.0, 1.3):
        e16, e32 = _poiseuille3_error(16, s3), _poiseuille3_error(32, s3)
        assert e32 < 1e-3
        assert 3.5 < e16 / e32 < 4.5


def test_conduction_between_dirichlet_faces_is_linear():
    nz = 16
    p = W.default_params3(nu=0.1, kappa=0.1, wall=(P, P, P, P, D, D), T_wall=(0, 0, 0, 0, 0.7, -0.3))
    o = oracle.Oracle3D(1, 1, nz, p)
    o.init(1.0, 0.0, 0.0, 0.0, 0.0)
    o.step(12000)
    T = o.fields()[4][:, 0, 0]
    zc = np.arange(nz)
    np.testing.assert_allclose(T, 0.7 - (zc + 0.5) / nz, atol=1e-12)


def test_closed_box_conserves_mass_and_heat():
    """Bounce-back on all six faces (edges and corners included) conserves sum f exactly, and with
    every face adiabatic sum g too."""
    prob = W.random_problem3d(4, 3, 5, seed=11, walls=(A,) * 6)
    o = oracle.Oracle3D.from_problem(prob)
    f0, g0 = o.populations()
    o.step(25)
    f1, g1 = o.populations()
    assert f1.sum() == pytest.approx(f0.sum(), rel=1e-13)
    assert g1.sum() == pytest.approx(g0.sum(), rel=1e-12, abs=1e-12)


# ----------------------------------------------------------------------------- moving wall faces


@pytest.mark.parametrize("lid_face,axis", [(5, 2), (3, 1), (1, 0)])
def test_couette_flow_between_a_moving_and_a_resting_face_is_linear(lid_face, axis):
    """A channel with walls on the faces of one axis, the upper one moving tangentially with
    (U, V) in the two other directions: the steady velocity is linear from 0 at the resting wall
    to the lid velocity at the moving one, both walls halfway between nodes, exact to 1e-12
    (as in 2-D, halfway bounce-back with the wall's equilibrium is exact for Couette flow)."""
    n = 12
    shape = [1, 1, 1]
    shape[axis] = n
    walls = [P] * 6
    walls[2 * axis], walls[2 * axis + 1] = A, A
    uw = [[0.0, 0.0, 0.0] for _ in range(6)]
    tang = [d for d in range(3) if d != axis]
    uw[lid_face][tang[0]], uw[lid_face][tang[1]] = 0.02, -0.013
    p = W.default_params3(nu=0.1, kappa=0.1, wall=tuple(walls), u_wall=tuple(map(tuple, uw)))
    o = oracle.Oracle3D(*shape, p)
    o.init(1.0, 0.0, 0.0, 0.0, 0.0)
    o.step(int(12 * n * n / 0.1))
    u = o.fields()[1:4]
    c = np.arange(n)
    line = (c + 0.5) / n
    for d, U in ((tang[0], 0.02), (tang[1], -0.013)):
        np.testing.assert_allclose(u[d].reshape(-1), U * line, atol=1e-12 * abs(U) + 1e-15)
    np.testing.assert_allclose(u[axis], 0.0, atol=1e-14)


def test_moving_faces_uniform_along_an_axis_reproduce_the_2d_oracle():
    """Moving walls with tangential motion and normal injection, fields uniform along z: the 3-D
    oracle steps like the 2-D one with the same moving y walls (pinned in test_oracle_pins.py)."""
    rng = np.random.default_rng(21)
    nx, ny = 6, 5
    nu = 0.06
    s_nu = 1.0 / (3 * nu + 0.5)
    uw2 = ((0.0, 0.0), (0.0, 0.0), (0.02, 0.01), (-0.015, -0.005))
    p2 = W.default_params(nu=nu, kappa=0.04, g_beta=4e-3, T0=0.05, s_b=s_nu, s_3=1.3, s_4=0.9,
                          lambda2=1.2, Fv=(1e-4, -5e-5), wall=(P, P, D, A), T_wall=(0, 0, 0.4, -0.3),
                          u_wall=uw2)
    rho = 1.0 + rng.uniform(-1e-3, 1e-3, (ny, nx))
    ux, uy = rng.uniform(-0.05, 0.05, (ny, nx)), rng.uniform(-0.05, 0.05, (ny, nx))
    T = rng.uniform(-0.4, 0.4, (ny, nx))
    o2 = oracle.Oracle(nx, ny, p2)
    o2.init(rho, ux, uy, T)
    uw3 = tuple((u[0], u[1], 0.0) for u in uw2) + ((0.0, 0.0, 0.0),) * 2
    p3 = W.default_params3(nu=nu, kappa=0.04, g_beta=4e-3, T0=0.05, s_b=s_nu, s_3=1.3, s_4=0.9,
                           s_5=1.7, s_6=0.6, lambda2=1.2, Fv=(1e-4, -5e-5, 0.0), g_axis=1,
                           wall=(P, P, D, A, P, P), T_wall=(0, 0, 0.4, -0.3, 0, 0), u_wall=uw3)
    o3 = oracle.Oracle3D(nx, ny, 2, p3)
    lift = lambda a: np.broadcast_to(a, (2, ny, nx))
    o3.init(lift(rho), lift(ux), lift(uy), 0.0, lift(T))
    o2.step(25)
    o3.step(25)
    r2, ux2, uy2, T2 = o2.fields()
    r3, ux3, uy3, uz3, T3 = o3.fields()
    for a3, a2 in ((r3, r2), (ux3, ux2), (uy3, uy2), (T3, T2)):
        np.testing.assert_allclose(a3, lift(a2), atol=1e-13)
    np.testing.assert_allclose(uz3, 0.0, atol=1e-15)


def test_residual3_reduces_to_the_2d_residual():
    """With no z velocity the 3-D residual is the 2-D one of the same (ux, uy, T) fields."""
    rng = np.random.default_rng(31)
    prev = [rng.normal(size=(4, 5, 6)) * s for s in (0.01, 0.02, 0.0, 0.3)]
    cur = [p + rng.normal(size=p.shape) * 1e-4 for p in prev]
    cur[2] = np.zeros_like(cur[2])
    e3 = oracle.residual3(prev, cur, 0.05, 1.0)
    e2 = oracle.residual((prev[0], prev[1], prev[3]), (cur[0], cur[1], cur[3]), 0.05, 1.0)
    assert e3 == pytest.approx(e2, rel=1e-14)


# ----------------------------------------------------------------------------- thermal-only mode


def test_thermal_only_collision_equals_the_coupled_d3q7_part():
    """The D3Q7 collision with a prescribed velocity equals the coupled step's D3Q7 part when the
    prescribed velocity is the flow's (no force, so u = sum f e / rho)."""
    rng = np.random.default_rng(41)
    for _ in range(20):
        p = rand_params3(rng, g_beta=0.0, Fv=(0.0, 0.0, 0.0))
        f = rng.uniform(0.005, 0.1, 27)
        g = rng.uniform(-0.1, 0.2, 7)
        u = (f @ E27) / f.sum()
        _, go = oracle.collide3_node(p, f, g)
        np.testing.assert_allclose(oracle.collide3_thermal_node(p, g, *u), go, atol=1e-16)


@pytest.mark.parametrize("axis", [0, 2])
def test_thermal_only_moving_frame_diffusivity(axis):
    """Sec. 3.1 in 3-D with the D3Q7 equation alone: a temperature wave along `axis` in a prescribed
    uniform flow (0.1, 0.12, -0.08) keeps alpha within 0.1% and travels at u_axis."""
    L, alpha, B = 60, 0.05, 0.01
    n3 = [1, 1, 1]
    n3[axis] = L
    adv = (0.1, 0.12, -0.08)
    p = W.default_params3(nu=0.05, kappa=alpha, T0=1.0, thermal_only=1)
    c = np.arange(L, dtype=np.float64)
    T = (1.0 + B * np.sin(2 * math.pi * c / L)).reshape([L if (2 - i) == axis else 1 for i in range(3)])
    o = oracle.Oracle3D(*n3, p)
    o.init(1.0, adv[0], adv[1], adv[2], np.broadcast_to(T, n3[::-1]))
    k = 2 * math.pi / L
    o.step(300)
    z1 = _mode(o.fields()[4].reshape(-1) - 1.0, k, L)
    o.step(1500)
    z2 = _mode(o.fields()[4].reshape(-1) - 1.0, k, L)
    assert -math.log(abs(z2) / abs(z1)) / (k * k * 1500) == pytest.approx(alpha, rel=1e-3)
    dphase = np.angle(z2 / z1)
    assert abs((dphase + k * adv[axis] * 1500 + math.pi) % (2 * math.pi) - math.pi) < 2e-3
    np.testing.assert_allclose(o.fields()[1], adv[0], atol=0)


def test_thermal_only_closed_box_conserves_heat():
    """Adiabatic faces all round and a divergence-free cellular velocity: sum g is conserved."""
    n = 8
    z, y, x = np.meshgrid(*(np.arange(n) + 0.5,) * 3, indexing="ij")
    k = math.pi / n
    ux = 0.05 * np.sin(k * x) * np.cos(k * y)
    uy = -0.05 * np.cos(k * x) * np.sin(k * y)
    p = W.default_params3(kappa=0.03, wall=(A,) * 6, thermal_only=1)
    o = oracle.Oracle3D(n, n, n, p)
    rng = np.random.default_rng(3)
    o.init(1.0, ux, uy, 0.0, rng.uniform(-0.5, 0.5, (n, n, n)))
    g0 = o.populations()[1].sum()
    o.step(40)
    assert o.populations()[1].sum() == pytest.approx(g0, rel=1e-13, abs=1e-13)
