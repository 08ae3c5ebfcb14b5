"""The 3-D CUDA path (D3Q27 + D3Q7 through include/clb3d.h) against the 3-D FP64 oracle.

Tolerances, normwise per field as in test_gpu_parity.py (rho against max|rho|, velocity against the
larger of max|u| and u_ref, T against the larger of max|T| and dT_ref):
  FP64: 1e-12 (rounding order only).
  FP32 deviation storage: 3 n u32 (floor 2e-6) after n steps, u32 = 2^-24. Each step rounds every
    stored deviation once and sums 27 of them for the density and momentum; relative to the field
    scales these are a few u32 per step, adding up at worst linearly.
  FP16 deviation storage (FP32 arithmetic): 3 sqrt(n) u16, u16 = 2^-11. The half-precision store of
    every deviation each step dominates; the roundings of successive stores are independent and add
    like a random walk; 27 of them enter each density and momentum sum.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1710_10569_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64, F32, F16 = W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV
P, D, A = W.WALL_PERIODIC, W.WALL_DIRICHLET, W.WALL_ADIABATIC
NAMES = ("rho", "ux", "uy", "uz", "T")
U32, U16 = 2.0 ** -24, 2.0 ** -11


def tol3(storage, steps):
    if storage == F64:
        return 1e-12
    if storage == F32:
        return max(2e-6, 3 * steps * U32)
    return 3 * max(steps, 1) ** 0.5 * U16


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def report(tag, errs):
    path = os.environ.get("CLB_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": tag, **errs}) + "\n")


def compare3(tag, got, exp, tol, params):
    u_ref, dT_ref = params.get("u_ref", 0.0), params.get("dT_ref", 0.0)
    us = max(max(float(np.max(np.abs(exp[i]))) for i in (1, 2, 3)), u_ref, 1e-300)
    errs = {}
    for k, (name, a, b) in enumerate(zip(NAMES, got, exp)):
        if name == "rho":
            s = float(np.max(np.abs(b)))
        elif name == "T":
            s = max(float(np.max(np.abs(b))), dT_ref, 1e-300)
        else:
            s = us
        errs[name] = float(np.max(np.abs(a - b))) / s
    report(tag, errs)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{tag}: normwise errors above {tol:g}: {bad} (all: {errs})"
    return errs


CASES = {
    "taylor_green_12": (lambda st: W.taylor_green3d(12, storage=st), 40),
    "random_walls_37x5x6": (lambda st: W.random_problem3d(37, 5, 6, seed=1, storage=st), 30),
    "closed_box_9x7x8": (lambda st: W.random_problem3d(9, 7, 8, seed=2, storage=st,
                                                     walls=(D, A, A, D, D, D)), 30),
    "two_blocks_ragged_150x3x3": (lambda st: W.random_problem3d(150, 3, 3, seed=3, storage=st), 20),
    "column_1x1x40": (lambda st: W.random_problem3d(1, 1, 40, seed=4, storage=st,
                                                  walls=(P, P, P, P, D, D)), 40),
    "slab_6x5x1": (lambda st: W.random_problem3d(6, 5, 1, seed=5, storage=st,
                                               walls=(A, D, P, P, P, P)), 30),
    "moving_faces_33x6x7": (lambda st: W.random_problem3d(33, 6, 7, seed=6, storage=st, moving=True,
                                                        walls=(D, A, P, P, A, D)), 35),
    "moving_box_9x8x7": (lambda st: W.random_problem3d(9, 8, 7, seed=7, storage=st, moving=True,
                                                     walls=(D, A, A, D, A, D)), 35),
}


@pytest.mark.parametrize("storage", [F64, F32, F16], ids=["f64", "f32", "f16dev"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_fields_match_the_oracle(clb, case, storage):
    """Fields after 1 step and after the case's step count (which includes a 32-step graph where
    it is at least 32); in FP64 also every population."""
    make, steps = CASES[case]
    prob = make(storage)
    o = oracle.Oracle3D.from_problem(prob)
    lat = clb.Lattice3D.from_problem(prob)
    done = 0
    for k in (1, steps):
        o.step(k - done)
        lat.step(k - done)
        done = k
        compare3(f"3d_{case}_{W.STORAGE_NAMES[storage]}_{k}", lat.fields(), o.fields(), tol3(storage, k),
                 prob.params)
    if storage == F64:
        fg, gg = lat.populations()
        fo, go = o.populations()
        assert float(np.max(np.abs(fg - fo))) <= 1e-12 * float(np.max(np.abs(fo)))
        assert float(np.max(np.abs(gg - go))) <= 1e-12 * max(float(np.max(np.abs(go))), 1e-3)
    lat.close()


@pytest.mark.parametrize("storage", [F64, F32, F16], ids=["f64", "f32", "f16dev"])
def test_launch_shapes_are_bitwise_equal(clb, storage):
    prob = W.random_problem3d(70, 6, 5, seed=9, storage=storage)
    out = []
    for shape in ((128, 1), (32, 4), (64, 2), (32, 1)):
        lat = clb.Lattice3D.from_problem(prob)
        lat.set_launch(*shape)
        lat.step(45)  # one graph of 32 steps and 13 single launches
        out.append(lat.populations())
        lat.close()
    for f, g in out[1:]:
        assert np.array_equal(f, out[0][0]) and np.array_equal(g, out[0][1])


@pytest.mark.parametrize("storage", [F64, F32], ids=["f64", "f32"])
def test_nusselt_matches_the_oracle(clb, storage):
    prob = W.rayleigh_benard3d(16, 6, 10, Ra=5e4, storage=storage, perturb=1e-2)
    o = oracle.Oracle3D.from_problem(prob)
    lat = clb.Lattice3D.from_problem(prob)
    o.step(80)
    lat.step(80)
    nu_o = o.nusselt(2)
    nu_g = lat.nusselt(2)
    assert nu_g == pytest.approx(nu_o, rel=1e-10 if storage == F64 else 1e-4, abs=1e-12)
    assert lat.nusselt(0) == pytest.approx(o.nusselt(0), rel=1e-9 if storage == F64 else 1e-3, abs=1e-9)


def _pull_sample(f_post, g_post, prob, x, y, z):
    """Pre-collision populations of node (x, y, z) at t+1 from post-collision populations at t
    (Eqs. 12, 22 with the face rules): f_i from x - e_i, across a wall the node's own opposite;
    g likewise, with -g*_opp + cs2_T T_w on Dirichlet faces."""
    p = prob.params
    e27 = oracle.matrices3(p, 0, 0, 0)["e27"]
    e7 = oracle.matrices3(p, 0, 0, 0)["e7"]
    n = (prob.nx, prob.ny, prob.nz)
    c = (x, y, z)

    def opp(e, es):
        return int(np.where((es == -e).all(axis=1))[0][0])

    f = np.empty(27)
    for i in range(27):
        s, ok = [c[d] - e27[i][d] for d in range(3)], True
        for d in range(3):
            if not 0 <= s[d] < n[d]:
                if p["wall"][2 * d] == P:
                    s[d] %= n[d]
                else:
                    ok = False
        f[i] = f_post[(x, y, z)][opp(e27[i], e27)] if not ok else f_post[tuple(s)][i]
    g = np.empty(7)
    for j in range(7):
        s, face = [c[d] - e7[j][d] for d in range(3)], -1
        for d in range(3):
            if s[d] < 0:
                if p["wall"][2 * d] == P:
                    s[d] += n[d]
                else:
                    face = 2 * d
            elif s[d] >= n[d]:
                if p["wall"][2 * d + 1] == P:
                    s[d] -= n[d]
                else:
                    face = 2 * d + 1
        if face < 0:
            g[j] = g_post[tuple(s)][j]
        else:
            bb = g_post[(x, y, z)][opp(e7[j], e7)]
            g[j] = -bb + p["cs2_T"] * p["T_wall"][face] if p["wall"][face] == D else bb
    return f, g


@pytest.mark.parametrize("storage", [F64, F32], ids=["f64", "f32"])
def test_bench_lattice_one_step_on_sampled_nodes(clb, storage):
    """On the 3-D bench lattice (Rayleigh-Benard 256 x 256 x 128, Ra = 1e7), in the default launch
    shape: the populations after one more step at 48 seeded nodes (a third of them on the wall
    layers) equal the oracle's collision of their neighbours' populations, pulled with the face
    rules (FP64: 1e-13 of the population scale; FP32: 2e-6, one step of rounding)."""
    prob = W.rayleigh_benard3d(256, 256, 128, Ra=1e7, storage=storage)
    lat = clb.Lattice3D.from_problem(prob)
    lat.step(20)
    f0, g0 = lat.populations()
    lat.step(1)
    f1, g1 = lat.populations()
    lat.close()
    rng = np.random.default_rng(12)
    pts = [(int(rng.integers(0, 256)), int(rng.integers(0, 256)), int(z))
           for z in list(rng.integers(1, 127, 32)) + [0] * 8 + [127] * 8]
    p = prob.params
    cache = {}

    def post(x, y, z):
        key = (x, y, z)
        if key not in cache:
            cache[key] = oracle.collide3_node(p, f0[:, z, y, x], g0[:, z, y, x])
        return cache[key]

    class _F(dict):
        def __init__(self, which):
            super().__init__()
            self.which = which

        def __getitem__(self, k):
            return post(*k)[self.which]

    scale_f = float(np.max(np.abs(f0)))
    tol = 1e-13 if storage == F64 else 2e-6
    for x, y, z in pts:
        fe, ge = _pull_sample(_F(0), _F(1), prob, x, y, z)
        assert np.max(np.abs(f1[:, z, y, x] - fe)) <= tol * scale_f, (x, y, z)
        assert np.max(np.abs(g1[:, z, y, x] - ge)) <= tol * 1.0, (x, y, z)


def test_largest_lattice_steps_and_conserves_mass(clb):
    """The largest 3-D lattice the 32-bit buffer offsets allow (384 x 384 x 428 in FP32, 63.1 M
    nodes, Rayleigh-Benard with Dirichlet z walls): after 3 steps the fields are finite and the total
    mass, which bounce-back and periodic faces conserve exactly, is unchanged to FP32 rounding."""
    prob = W.rayleigh_benard3d(384, 384, 428, Ra=1e6, storage=F32)
    lat = clb.Lattice3D.from_problem(prob)
    m0 = float(np.sum(lat.fields()[0]))
    lat.step(3)
    rho, ux, uy, uz, T = lat.fields()
    lat.close()
    assert all(np.isfinite(a).all() for a in (rho, ux, uy, uz, T))
    assert float(np.sum(rho)) == pytest.approx(m0, rel=1e-6)
    assert float(np.max(np.abs(T))) <= 0.5 + 1e-2


@pytest.mark.parametrize("storage", [F64, F32], ids=["f64", "f32"])
def test_residual_and_run_match_the_oracle(clb, storage):
    """clb3d_residual against the residual of the oracle's fields at the same two times (FP64 to
    1e-9 relative, FP32 to 1e-3), twice in a row so the snapshot is replaced; clb3d_run stops a
    conduction problem at the residual tolerance with the linear temperature profile."""
    prob = W.rayleigh_benard3d(10, 8, 9, Ra=5e4, perturb=1e-2, storage=storage)
    o = oracle.Oracle3D.from_problem(prob)
    lat = clb.Lattice3D.from_problem(prob)
    p = prob.params
    prev = o.fields()[1:]
    for k in (40, 25):
        o.step(k)
        lat.step(k)
        cur = o.fields()[1:]
        exp = oracle.residual3(prev, cur, p["u_ref"], p["dT_ref"])
        assert lat.residual() == pytest.approx(exp, rel=1e-9 if storage == F64 else 1e-3)
        prev = cur
    lat.close()
    cond = W.default_params3(nu=0.1, kappa=0.1, wall=(P, P, P, P, D, D), T_wall=(0, 0, 0, 0, 0.7, -0.3),
                             storage=storage, dT_ref=1.0)
    lat = clb.Lattice3D(2, 2, 12, cond)
    lat.init_fields(1.0, 0.0, 0.0, 0.0, 0.0)
    steps, er = lat.run(1e-9 if storage == F64 else 1e-6, 40000, 100)
    assert er < (1e-9 if storage == F64 else 1e-6) and steps < 40000
    T = lat.fields()[4][:, 0, 0]
    zc = np.arange(12)
    np.testing.assert_allclose(T, 0.7 - (zc + 0.5) / 12, atol=1e-7 if storage == F64 else 1e-4)
    lat.close()


@pytest.mark.parametrize("storage", [F64, F16], ids=["f64", "f16dev"])
def test_checkpoint_restores_the_run_bit_for_bit(clb, storage):
    """clb3d_save after 37 steps, 20 more steps, clb3d_load, the same 20 steps again: the same
    populations bit for bit; a checkpoint of another lattice is refused."""
    prob = W.random_problem3d(13, 7, 6, seed=15, storage=storage, moving=True, walls=(P, P, D, A, A, D))
    lat = clb.Lattice3D.from_problem(prob)
    lat.step(37)
    ck = lat.save()
    lat.step(20)
    a = lat.populations()
    lat.load(ck)
    lat.step(20)
    b = lat.populations()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    other = clb.Lattice3D(13, 7, 5, prob.params)
    with pytest.raises(clb.CLBError):
        other.load(ck)
    other.close()
    lat.close()


def test_non_finite_fields_are_reported(clb):
    """A NaN in the initial temperature reaches CLB_ENAN in the Nusselt number and the residual."""
    prob = W.rayleigh_benard3d(8, 6, 5, Ra=1e4)
    prob.T[2, 3, 4] = float("nan")
    lat = clb.Lattice3D(prob.nx, prob.ny, prob.nz, prob.params)
    with pytest.raises(clb.CLBError) as e:
        lat.init_fields(*prob.fields())
    assert e.value.status == clb.CLB_ENAN
    lat.step(3)
    for call in (lambda: lat.nusselt(2), lat.residual):
        with pytest.raises(clb.CLBError) as e:
            call()
        assert e.value.status == clb.CLB_ENAN
    lat.close()


@pytest.mark.parametrize("storage", [F64, F32], ids=["f64", "f32"])
def test_high_order_rates_one_form_matches_the_oracle(clb, storage):
    """With s_3 = s_4 = s_5 = s_6 = 1 (the paper's setting) the step takes the form that does not
    form the high-order moments; walls, moving faces, buoyancy and a body force included, it stays
    within the parity bar of the oracle, whose general collision is the same map."""
    prob = W.random_problem3d(23, 6, 7, seed=19, storage=storage, moving=True, walls=(P, P, D, A, A, D))
    prob.params.update(s_3=1.0, s_4=1.0, s_5=1.0, s_6=1.0)
    o = oracle.Oracle3D.from_problem(prob)
    lat = clb.Lattice3D.from_problem(prob)
    o.step(40)
    lat.step(40)
    compare3(f"3d_high1_{W.STORAGE_NAMES[storage]}", lat.fields(), o.fields(), tol3(storage, 40), prob.params)
    lat.close()
