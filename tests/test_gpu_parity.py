"""CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances (normwise per field, see compare()):
  FP64 storage + FP64 arithmetic: 1e-12 (the two sides differ only in rounding order).
  FP32 deviation storage + FP32 arithmetic: 2 n u32 (floor 1e-6) after n steps, u32 = 2^-24: each
    step adds at most a few roundings of size u32 relative to the velocity and temperature scales,
    and they can add up coherently (linear growth).
  FP16 deviation storage + FP32 arithmetic: 2 sqrt(n) u16, u16 = 2^-11: the half-precision store
    of every population each step dominates; the roundings are independent, so they add like a
    random walk.
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
NAMES = ("rho", "ux", "uy", "T")
U32, U16 = 2.0 ** -24, 2.0 ** -11


def tol(storage, steps):
    if storage == F64:
        return 1e-12
    if storage == F32:
        return max(1e-6, 2 * steps * U32)
    return 2 * max(steps, 1) ** 0.5 * U16


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def normwise(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (scale if scale > 0 else 1.0)


def report(tag, errs):
    path = os.environ.get("CLB_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": tag, **errs}) + "\n")


def compare(tag, got, exp, tol, params=None):
    """Normwise errors per field. rho is measured against max|rho|; u against the larger of max|u|
    and the problem's characteristic velocity u_ref (u is a small difference of O(1) populations,
    so its rounding error scales with them, not with |u|); T against the larger of max|T| and the
    problem's temperature difference dT_ref."""
    u_ref = params.get("u_ref", 0.0) if params else 0.0
    dT_ref = params.get("dT_ref", 0.0) if params else 0.0
    errs = {}
    for name, a, b in zip(NAMES, got, exp):
        if name == "rho":
            errs[name] = float(np.max(np.abs(a - b))) / float(np.max(np.abs(b)))
        elif name in ("ux", "uy"):
            s = max(float(np.max(np.abs(exp[1]))), float(np.max(np.abs(exp[2]))), u_ref, 1e-300)
            errs[name] = float(np.max(np.abs(a - b))) / s
        else:
            s = max(float(np.max(np.abs(b))), dT_ref, 1e-300)
            errs[name] = float(np.max(np.abs(a - b))) / s
    report(tag, errs)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{tag}: normwise errors above {tol:g}: {bad} (all: {errs})"
    return errs


def run_both(clb, prob, steps):
    lat = clb.Lattice.from_problem(prob)
    lat.step(steps)
    got = lat.fields()
    o = oracle.Oracle.from_problem(prob)
    o.step(steps)
    return lat, o, got, o.fields()


# ------------------------------------------------------------------ config #1: periodic TG, FP64


def test_taylor_green_64_fp64_1000_steps(clb):
    prob = W.taylor_green(64, storage=F64)
    lat, o, got, exp = run_both(clb, prob, 1000)
    compare("tg64_f64_1000", got, exp, 1e-12, prob.params)
    f, g = lat.populations()
    fo, go = o.populations()
    assert normwise(f, fo) <= 1e-12 and normwise(g, go) <= 1e-12


@pytest.mark.parametrize("storage", [F32, F16])
def test_taylor_green_64_reduced_precision(clb, storage):
    prob = W.taylor_green(64, storage=storage)
    _, _, got, exp = run_both(clb, prob, 1000)
    compare(f"tg64_{W.STORAGE_NAMES[storage]}_1000", got, exp, tol(storage, 1000), prob.params)


# ------------------------------------------------------------------ walls, ragged sizes, all storages

SHAPES = [(67, 45), (130, 7), (2, 2), (3, 257), (257, 3), (33, 33)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_problems_fp64(clb, shape, seed):
    prob = W.random_problem(*shape, seed=seed, storage=F64)
    _, _, got, exp = run_both(clb, prob, 60)
    compare(f"rand{shape}_s{seed}_f64", got, exp, 1e-12, prob.params)


@pytest.mark.parametrize("storage", [F32, F16])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_problems_reduced_precision(clb, storage, seed):
    prob = W.random_problem(67, 45, seed=seed, storage=storage)
    _, _, got, exp = run_both(clb, prob, 60)
    compare(f"rand67x45_s{seed}_{W.STORAGE_NAMES[storage]}", got, exp, tol(storage, 60), prob.params)


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_moving_walls(clb, storage, seed):
    """Random wall velocities on every wall layout: moving-wall bounce-back and the anti-bounce-back
    with the wall velocity, including corners, on the scalar wall path."""
    prob = W.random_problem(45, 38, seed=seed, storage=storage, moving=True)
    _, _, got, exp = run_both(clb, prob, 60)
    compare(f"moving45x38_s{seed}_{W.STORAGE_NAMES[storage]}", got, exp, tol(storage, 60), prob.params)
    if storage == F64:
        lat = clb.Lattice.from_problem(prob)
        o = oracle.Oracle.from_problem(prob)
        f, g = lat.populations()
        fo, go = o.populations()
        assert normwise(f, fo) <= 1e-14 and normwise(g, go) <= 1e-14


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("seed", [0, 1])
def test_wet_walls(clb, storage, seed):
    """The paper's own wall conditions (walls on the end rows, y sides): moving/injecting walls,
    body force and buoyancy, against the oracle."""
    prob = W.random_problem(70, 23, seed=seed, storage=storage, walls=(P, P, W.WALL_WET, W.WALL_WET),
                            moving=True)
    _, _, got, exp = run_both(clb, prob, 60)
    compare(f"wet70x23_s{seed}_{W.STORAGE_NAMES[storage]}", got, exp, tol(storage, 60), prob.params)
    if storage == F64:
        lat = clb.Lattice.from_problem(prob)
        o = oracle.Oracle.from_problem(prob)
        assert lat.nusselt(1) == pytest.approx(o.nusselt(1), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("walls", [(W.WALL_WET, W.WALL_WET, P, P), (W.WALL_WET,) * 4], ids=["wet_x", "wet_box"])
@pytest.mark.parametrize("shape", [(23, 70), (333, 9), (3, 3)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_wet_walls_on_x_sides_and_in_corners(clb, storage, walls, shape):
    """The paper's own wall conditions on the x sides (walls on the end columns), and on all four
    sides of a closed box (the corner rule), with moving/injecting walls, body force and buoyancy,
    against the oracle; rows wide enough for interior warps on the vector path, the smallest box
    (one fluid node), and the Nusselt number along both axes (trapezoid weights in every wet
    direction)."""
    nx, ny = shape
    prob = W.random_problem(nx, ny, seed=nx, storage=storage, walls=walls, moving=True)
    _, _, got, exp = run_both(clb, prob, 40)
    compare(f"wet_{'box' if walls[2] == W.WALL_WET else 'x'}{nx}x{ny}_{W.STORAGE_NAMES[storage]}", got, exp,
            tol(storage, 40), prob.params)
    if storage == F64:
        lat = clb.Lattice.from_problem(prob)
        lat.step(40)
        o = oracle.Oracle.from_problem(prob)
        o.step(40)
        for axis in (0, 1):
            assert lat.nusselt(axis) == pytest.approx(o.nusselt(axis), rel=1e-12, abs=1e-12)


def test_initial_fields_match_oracle(clb):
    """Step 0: the inverse-stream initialisation reproduces the oracle's f(x,0) = f^eq exactly,
    walls included."""
    for seed in range(4):
        prob = W.random_problem(19, 23, seed=seed, storage=F64)
        lat = clb.Lattice.from_problem(prob)
        o = oracle.Oracle.from_problem(prob)
        f, g = lat.populations()
        fo, go = o.populations()
        assert normwise(f, fo) <= 1e-14 and normwise(g, go) <= 1e-14
        compare(f"init_s{seed}", lat.fields(), o.fields(), 1e-14, prob.params)


# ------------------------------------------------------------------ config #2 cavity, config #3 RB


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_cavity_256_short(clb, storage):
    prob = W.cavity(256, storage=storage)
    # the fluid starts at rest with 1e-4 noise: give the buoyant flow time to develop
    _, o, got, exp = run_both(clb, prob, 400)
    compare(f"cavity256_{W.STORAGE_NAMES[storage]}_400", got, exp, tol(storage, 400), prob.params)


RB_FULL_STEPS = 200


@pytest.fixture(scope="module")
def rb_full_oracle():
    """The oracle's fields of the bench workload (Rayleigh-Benard 2048 x 1024, Ra = 1e7) after
    RB_FULL_STEPS steps; computed once for the three storage forms (FP64 arithmetic)."""
    o = oracle.Oracle.from_problem(W.rayleigh_benard(2048, 1024, storage=F64))
    o.step(RB_FULL_STEPS)
    return o.fields()


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_rayleigh_benard_2048x1024_full_size(clb, storage, rb_full_oracle):
    """The bench workload at full size in the launch configuration bench.py times (graph chunks of
    the fused kernel plus single launches), 200 steps, every node compared."""
    prob = W.rayleigh_benard(2048, 1024, storage=storage)
    lat = clb.Lattice.from_problem(prob)
    lat.step(RB_FULL_STEPS)
    got = lat.fields()
    lat.close()
    compare(f"rb2048_{W.STORAGE_NAMES[storage]}_{RB_FULL_STEPS}", got, rb_full_oracle,
            tol(storage, RB_FULL_STEPS), prob.params)


def test_graph_chunks_equal_single_launches(clb):
    """clb_step(n) replays captured 32-step graphs plus single launches; the result does not depend
    on how the steps are grouped."""
    prob = W.random_problem(70, 40, seed=2, storage=F64)
    a = clb.Lattice.from_problem(prob)
    a.step(75)
    b = clb.Lattice.from_problem(prob)
    for _ in range(75):
        b.step(1)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("walls", [(P, P, P, P), (D, D, A, A), (P, P, D, D), (P, P, W.WALL_WET, W.WALL_WET),
                                   (W.WALL_WET, W.WALL_WET, P, P), (W.WALL_WET,) * 4],
                         ids=["periodic", "cavity", "rb", "wet", "wet_x", "wet_box"])
def test_launch_shapes_are_bitwise_equal(clb, storage, walls):
    """Vector interior path, scalar wall/ragged path and every launch shape give the same bits."""
    prob = W.random_problem(333, 37, seed=3, storage=storage, walls=walls)
    ref = None
    for shape in ((128, 1, 1, 0, 0), (64, 4, 2, 0, 0), (128, 2, 4, 0, 0), (32, 8, 1, 0, 0),
                  (256, 1, 2, 0, 0), (32, 1, 4, 0, 0), (128, 1, 2, 2, 4), (128, 1, 2, 3, 7),
                  (128, 1, 4, 4, 16), (128, 1, 4, 3, 1)):
        if storage == F64 and shape[2] == 4 and shape[3] == 4:
            continue  # exceeds shared memory
        lat = clb.Lattice.from_problem(prob)
        lat.set_launch(*shape[:3])
        lat.set_pipeline(shape[3], shape[4])
        lat.step(40)
        got = lat.fields()
        if ref is None:
            ref = got
        for x, y in zip(got, ref):
            assert np.array_equal(x, y), shape


EDGE_SHAPES = [(2, 2), (3, 257), (257, 3), (129, 2), (128, 5), (256, 4), (131, 9)]
EDGE_WALLS = {"periodic": (P, P, P, P), "cavity": (D, D, A, A), "rb": (P, P, D, D), "wet_x": (W.WALL_WET, W.WALL_WET, P, P),
              "wet_y": (P, P, W.WALL_WET, W.WALL_WET)}


@pytest.mark.parametrize("rates", ["general", "one"])
@pytest.mark.parametrize("storage", [F32, F16])
@pytest.mark.parametrize("walls", sorted(EDGE_WALLS))
@pytest.mark.parametrize("shape", EDGE_SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_small_and_edge_shapes_reduced_precision(clb, storage, walls, shape, rates):
    """Lattices where the FP16 step's split into interior warps and edge warps degenerates (no
    interior row or column, one warp per row, a ragged last warp, two rows) and where the FP32
    vector path covers few or no warps, with random rates and with the high-order rates at 1 (the
    forms the host picks between): within the parity bar of the oracle at every node."""
    w = EDGE_WALLS[walls]
    nx, ny = shape
    if (w[0] == W.WALL_WET and nx < 3) or (w[2] == W.WALL_WET and ny < 3):
        pytest.skip("a wet wall pair needs at least 3 nodes across")
    prob = W.random_problem(nx, ny, seed=11, storage=storage, walls=w)
    if rates == "one":
        prob.params.update(s_3=1.0, s_4=1.0, lambda2=1.0)
    _, _, got, exp = run_both(clb, prob, 40)
    compare(f"edge{shape}_{walls}_{rates}_{W.STORAGE_NAMES[storage]}", got, exp, tol(storage, 40), prob.params)


# ------------------------------------------------------------------ diagnostics


def test_nusselt_and_residual_match_oracle(clb):
    for prob in (W.random_problem(41, 33, seed=1, storage=F64), W.cavity(48, Ra=1e4, storage=F64)):
        lat = clb.Lattice.from_problem(prob)
        o = oracle.Oracle.from_problem(prob)
        prev = o.fields()[1:]
        lat.step(100)
        o.step(100)
        cur = o.fields()
        nu_gpu = lat.nusselt(prob.nu_axis)
        nu_ref = oracle.nusselt(cur[1], cur[2], cur[3], prob.params, prob.nu_axis)
        assert nu_gpu == pytest.approx(nu_ref, rel=1e-11, abs=1e-12)
        er_gpu = lat.residual()
        er_ref = oracle.residual(prev, cur[1:], prob.params["u_ref"], prob.params["dT_ref"])
        assert er_gpu == pytest.approx(er_ref, rel=1e-9)


@pytest.mark.parametrize("storage", [F32, F16])
def test_reduced_precision_diagnostics_match_oracle(clb, storage):
    """FP32 and FP16 storage: the node terms of the diagnostics are formed in FP32 (FP64 sums). E_R
    of a random problem's first 100 steps and Nu of a Rayleigh-Benard cell agree with the FP64
    oracle to the fields' precision, and a second pass gives the same Nu."""
    prob = W.random_problem(300, 37, seed=5, storage=storage)
    lat = clb.Lattice.from_problem(prob)
    o = oracle.Oracle.from_problem(prob.with_storage(F64))
    prev = o.fields()[1:]
    lat.step(100)
    o.step(100)
    er_ref = oracle.residual(prev, o.fields()[1:], prob.params["u_ref"], prob.params["dT_ref"])
    assert lat.residual() == pytest.approx(er_ref, rel=1e-2 if storage == F16 else 1e-4)

    prob = W.rayleigh_benard(256, 128, Ra=1e5, storage=storage)
    lat = clb.Lattice.from_problem(prob)
    o = oracle.Oracle.from_problem(prob.with_storage(F64))
    lat.step(100)
    o.step(100)
    cur = o.fields()
    nu_ref = oracle.nusselt(cur[1], cur[2], cur[3], prob.params, prob.nu_axis)
    nu_gpu = lat.nusselt(prob.nu_axis)
    assert nu_gpu == pytest.approx(nu_ref, rel=2e-3 if storage == F16 else 1e-4)
    assert lat.nusselt(prob.nu_axis) == nu_gpu


def test_run_to_steady_conduction(clb):
    """clb_run stops at the residual tolerance; the steady state is the conduction line."""
    ny = 16
    p = W.default_params(nu=0.1, kappa=0.1, wall=(P, P, D, D), T_wall=(0, 0, 0.5, -0.5), dT_ref=1.0,
                         u_ref=0.0)
    lat = clb.Lattice(4, ny, p)
    lat.init_fields()
    steps, er = lat.run(1e-10, 200000, 100)
    assert er < 1e-10 and steps < 200000
    T = lat.fields()[3][:, 0]
    np.testing.assert_allclose(T, 0.5 - (np.arange(ny) + 0.5) / ny, atol=1e-9)


def test_nan_is_reported(clb):
    prob = W.random_problem(16, 16, seed=0, storage=F64)
    lat = clb.Lattice.from_problem(prob)
    blob = bytearray(lat.save())
    # poison the first population value after the checkpoint header
    hdr = 40
    blob[hdr:hdr + 8] = np.array([np.nan]).tobytes()
    lat.load(bytes(blob))
    with pytest.raises(clb.CLBError) as e:
        lat.nusselt(1)
    assert e.value.status == clb.CLB_ENAN


# ------------------------------------------------------------------ checkpoints


def test_checkpoint_roundtrip_bitwise(clb):
    prob = W.random_problem(50, 30, seed=2, storage=F32)
    a = clb.Lattice.from_problem(prob)
    a.step(25)
    blob = a.save()
    a.step(30)
    ref = a.fields()
    b = clb.Lattice(prob.nx, prob.ny, prob.params)
    b.load(blob)
    assert b.steps == 25
    b.step(30)
    for x, y in zip(b.fields(), ref):
        assert np.array_equal(x, y)


def test_pipeline_rejects_bad_shapes(clb):
    prob = W.random_problem(64, 64, seed=1, storage=F64)
    a = clb.Lattice.from_problem(prob)
    a.set_launch(128, 1, 4)
    for stages, rows in ((4, 8), (5, 8), (1, 8), (3, 300)):
        with pytest.raises(clb.CLBError):
            a.set_pipeline(stages, rows)
    a.set_launch(128, 1, 1)
    with pytest.raises(clb.CLBError):
        a.set_pipeline(2, 8)


def test_autotune_keeps_state(clb):
    prob = W.random_problem(300, 200, seed=1, storage=F32)
    a = clb.Lattice.from_problem(prob)
    before = a.fields()
    shape = a.autotune()
    assert a.launch() == shape
    for x, y in zip(a.fields(), before):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_check_equals_nusselt_and_residual(clb, storage):
    """clb_check gives, from one pass, what clb_nusselt and clb_residual give (bitwise), and its
    snapshot serves the next residual the same way."""
    prob = W.rayleigh_benard(96, 48, Ra=2e4, storage=storage)
    a, b = clb.Lattice.from_problem(prob), clb.Lattice.from_problem(prob)
    for n in (150, 150):
        a.step(n)
        b.step(n)
        nu, er = a.check(1)
        assert nu == b.nusselt(1)
        assert er == b.residual()
    a.close()
    b.close()


@pytest.mark.parametrize("storage", [F64, F32])
def test_pinned_and_pageable_host_fields_agree(clb, storage):
    """clb_init_fields reads pinned host arrays directly and stages pageable ones; clb_fields
    writes pinned arrays directly and pageable ones through staging. Both routes give the same
    bits, also when the two kinds are mixed in one call."""
    import torch
    prob = W.random_problem(130, 41, seed=5, storage=storage)
    n = prob.nodes
    pin = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(8)]
    for t, a in zip(pin[:4], prob.fields()):
        t.numpy()[:] = a.ravel()
    a = clb.Lattice(prob.nx, prob.ny, prob.params)
    a.init_fields(*[t.numpy() for t in pin[:4]])
    b = clb.Lattice(prob.nx, prob.ny, prob.params)
    b.init_fields(prob.rho, pin[1].numpy(), prob.uy, pin[3].numpy())  # mixed kinds
    for lat in (a, b):
        lat.step(37)
    ref = a.fields()  # pageable outputs
    a.fields_into(*[t.numpy() for t in pin[4:]])
    for t, r in zip(pin[4:], ref):
        assert np.array_equal(t.numpy().reshape(prob.ny, prob.nx), r)
    for x, y in zip(b.fields(), ref):
        assert np.array_equal(x, y)
    a.close()
    b.close()
