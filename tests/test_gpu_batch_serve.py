"""Batched and served stepping: every instance evolves exactly as it does alone, and matches the
oracle like a single lattice does."""
import numpy as np
import pytest

import oracle
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


def mixed_problems(storage, count=6):
    probs = [W.random_problem(17 + 13 * k, 11 + 7 * k, seed=k, storage=storage) for k in range(count - 2)]
    if count >= 6:
        # the paper's own walls on the x sides, and on all four sides (corners)
        probs[2] = W.random_problem(43, 25, seed=2, storage=storage, walls=(W.WALL_WET, W.WALL_WET, W.WALL_PERIODIC,
                                                                             W.WALL_PERIODIC), moving=True)
        probs[3] = W.random_problem(56, 32, seed=3, storage=storage, walls=(W.WALL_WET,) * 4, moving=True)
    probs.append(W.cavity(40, Ra=1e4, storage=storage))
    probs.append(W.taylor_green(24, ny=48, storage=storage))
    return probs


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_instance_alone_equals_instance_in_mix(clb, storage):
    probs = mixed_problems(storage)
    mix = clb.Batch(probs)
    mix.step(70)
    for k, prob in enumerate(probs):
        alone = clb.Batch([prob])
        alone.step(70)
        for a, b in zip(mix.fields(k), alone.fields(0)):
            assert np.array_equal(a, b), (k, prob.name)


@pytest.mark.parametrize("tile", [(128, 1, 1), (64, 2, 2), (32, 4, 4), (256, 1, 2), (64, 1, 4)])
def test_tile_shape_does_not_change_results(clb, tile):
    probs = mixed_problems(F32)
    ref = clb.Batch(probs)
    ref.step(40)
    b = clb.Batch(probs)
    b.set_tile(*tile)
    b.step(40)
    for k in range(len(probs)):
        for x, y in zip(b.fields(k), ref.fields(k)):
            assert np.array_equal(x, y)


# Rows one to four tiles long, ending at every residue modulo V = 1, 2, 4 and modulo the tile width;
# short lattices, and tall ones that take several tiles (of several groups of rows) along y.
WIDE = [(nx, 5 + k % 3) for k, nx in enumerate([63, 64, 65, 66, 67, 97, 127, 128, 129, 130, 131, 133,
                                                191, 193, 258])] + [(97, 70), (133, 33), (64, 129)]


@pytest.mark.parametrize("storage", [F32, F16, F64])
@pytest.mark.parametrize("tile", [(32, 4, 2), (32, 4, 4), (64, 2, 2), (32, 1, 1)])
def test_rows_wider_than_a_tile_equal_single_lattice(clb, storage, tile):
    """The last tile of a row that runs past the row's end is moved left to end on the last
    multiple of V below nx, and the nx % V nodes after it are updated one by one; every node must
    come out exactly as the single-lattice step computes it (walls on x, some of them moving)."""
    probs = [W.random_problem(nx, ny, seed=1 + k % 3, storage=storage, moving=k % 2 == 1)
             for k, (nx, ny) in enumerate(WIDE)]
    b = clb.Batch(probs)
    b.set_tile(*tile)
    b.step(12)
    for k, prob in enumerate(probs):
        single = clb.Lattice.from_problem(prob)
        single.step(12)
        for x, y in zip(b.fields(k), single.fields()):
            assert np.array_equal(x, y), (prob.name, tile)


def test_row_groups_per_block_equal_single_lattice(clb):
    """A batch large enough (3.7 M nodes) that each block steps several groups of rows, with odd and
    even widths and walls on x: sampled instances equal the single-lattice step bitwise. A small
    batch keeps one group per block (the launch keeps enough blocks to fill the device)."""
    sizes = [(256 + 3 * (k % 5), 200 + 17 * (k % 7)) for k in range(56)]
    probs = [W.random_problem(nx, ny, seed=1 + k % 3, storage=F32, moving=k % 2 == 1)
             for k, (nx, ny) in enumerate(sizes)]
    b = clb.Batch(probs)
    launch = b.launch()
    assert launch["tile"] == (32, 4, 2) and launch["groups"] >= 2, launch
    b.step(6)
    for k in (0, 1, 2, 3, 4, 9, 27, 55):
        single = clb.Lattice.from_problem(probs[k])
        single.step(6)
        for x, y in zip(b.fields(k), single.fields()):
            assert np.array_equal(x, y), probs[k].name
    assert clb.Batch(probs[:2]).launch()["groups"] == 1


def test_batch_autotune_keeps_state_and_results(clb):
    probs = mixed_problems(F32)
    ref = clb.Batch(probs)
    ref.step(20)
    b = clb.Batch(probs)
    b.step(10)
    tile = b.autotune()
    assert tile[0] % 32 == 0 and tile[2] in (1, 2, 4)
    b.step(10)
    for k in range(len(probs)):
        for x, y in zip(b.fields(k), ref.fields(k)):
            assert np.array_equal(x, y)


def test_batch_matches_oracle_and_single_lattice(clb):
    probs = mixed_problems(F64)
    b = clb.Batch(probs)
    b.step(50)
    nu, er = b.diagnostics()
    for k, prob in enumerate(probs):
        o = oracle.Oracle.from_problem(prob)
        o.step(50)
        exp = o.fields()
        got = b.fields(k)
        for a, e in zip(got, exp):
            assert np.max(np.abs(a - e)) <= 1e-12 * max(np.max(np.abs(e)), 1e-300)
        single = clb.Lattice.from_problem(prob)
        single.step(50)
        assert nu[k] == pytest.approx(single.nusselt(prob.nu_axis), rel=1e-12, abs=1e-14)


def test_batch_run_retires_converged_instances(clb):
    """Conduction problems of different heights converge at different times; each instance stops
    at its own residual crossing and keeps its state after retirement."""
    probs = []
    for ny in (8, 16, 24):
        p = W.default_params(nu=0.1, kappa=0.1, wall=(W.WALL_PERIODIC,) * 2 + (W.WALL_DIRICHLET,) * 2,
                             T_wall=(0, 0, 0.5, -0.5), dT_ref=1.0, storage=F64)
        z = np.zeros((ny, 4))
        probs.append(W.Problem(f"cond{ny}", 4, ny, p, np.ones((ny, 4)), z, z, z.copy(), nu_axis=1))
    b = clb.Batch(probs)
    steps, er, status = b.run(1e-9, 100000, 100)
    assert (status == 0).all() and (er < 1e-9).all()
    assert steps[0] < steps[1] < steps[2]
    for k, prob in enumerate(probs):
        T = b.fields(k)[3][:, 0]
        np.testing.assert_allclose(T, 0.5 - (np.arange(prob.ny) + 0.5) / prob.ny, atol=1e-7)


def test_served_results_equal_alone(clb):
    """Requests submitted while others run are admitted as memory frees up; each result equals the
    same problem stepped alone for the same number of steps."""
    probs = mixed_problems(F32, count=5)
    srv = clb.Server(hbm_budget_bytes=64 << 20, max_slots=2, storage=F32)
    ids = []
    for k, prob in enumerate(probs):
        ids.append(srv.submit(prob, step_cap=64 * (k + 1), tol=0.0))
        srv.progress(32)  # a request arrives each round
    for _ in range(100):
        active, queued = srv.progress(32)
        if active == 0 and queued == 0:
            break
    for rid, prob in zip(ids, probs):
        done, nu, steps, er = srv.poll(rid)
        assert done and steps == 64 * (probs.index(prob) + 1)
        got = srv.fetch(rid, prob.ny, prob.nx)
        alone = clb.Batch([prob])
        alone.step(steps)
        for a, b in zip(got, alone.fields(0)):
            assert np.array_equal(a, b), prob.name


def test_serve_budget_and_errors(clb):
    srv = clb.Server(hbm_budget_bytes=1 << 20, max_slots=4, storage=F32)
    big = W.cavity(256, storage=F32)
    with pytest.raises(clb.CLBError) as e:
        srv.submit(big, step_cap=10, tol=0.0)
    assert e.value.status == clb.CLB_ENOMEM
    small = W.cavity(16, storage=F32)
    rid = srv.submit(small, step_cap=32, tol=0.0)
    with pytest.raises(clb.CLBError) as e:
        srv.fetch(rid, 16, 16)
    assert e.value.status == clb.CLB_EBUSY
    for _ in range(10):
        active, queued = srv.progress(32)
        if not active and not queued:
            break
    assert srv.poll(rid)[0]


def test_nan_in_one_instance_leaves_the_others_running(clb):
    """A blown-up instance is reported as CLB_ENAN and retired; the others step on unaffected."""
    probs = mixed_problems(F64, count=4)
    b = clb.Batch(probs)
    bad = probs[1]
    T = bad.T.copy()
    T[3, 4] = np.nan
    b.init_fields(1, bad.rho, bad.ux, bad.uy, T)
    steps, er, status = b.run(0.0, 200, 100)
    assert status[1] == clb.CLB_ENAN and steps[1] == 100
    assert all(status[k] == clb.CLB_OK and steps[k] == 200 for k in (0, 2, 3))
    alone = clb.Batch([probs[2]])
    alone.step(200)
    for a, c in zip(b.fields(2), alone.fields(0)):
        assert np.array_equal(a, c)


def test_serve_cancel(clb):
    srv = clb.Server(hbm_budget_bytes=64 << 20, max_slots=1, storage=F32)
    a = srv.submit(W.cavity(32, storage=F32), step_cap=10 ** 6, tol=0.0)
    b = srv.submit(W.cavity(24, storage=F32), step_cap=64, tol=0.0)
    srv.progress(32)           # a runs, b waits for the only slot
    srv.cancel(a)              # frees the slot
    for _ in range(10):
        active, queued = srv.progress(32)
        if not active and not queued:
            break
    assert srv.poll(b)[0]
    with pytest.raises(clb.CLBError):
        srv.poll(a)


@pytest.mark.parametrize("storage", [F64, F32])
def test_widest_lattice(clb, storage):
    """The largest edge the ABI accepts (2^20 nodes) on a 2-row channel, against the oracle."""
    import oracle
    prob = W.random_problem(1 << 20, 2, seed=2, storage=storage, moving=True)
    lat = clb.Lattice.from_problem(prob)
    lat.step(3)
    got = lat.fields()
    o = oracle.Oracle.from_problem(prob)
    o.step(3)
    exp = o.fields()
    for a, e in zip(got[1:], exp[1:]):
        assert np.max(np.abs(a - e)) <= (1e-12 if storage == F64 else 1e-5) * max(np.max(np.abs(e)), 0.05)


def test_serve_pool_reuses_memory_one_at_a_time(clb):
    """A budget that holds one of these lattices but not two: requests are admitted one after
    another into the same pool memory, and each result still equals the problem alone (nothing of
    a retired request leaks into the next one's state)."""
    # 128 x 96 in FP32: two population buffers of 14 planes x 96 rows x 512 bytes (1.38 MB) and a
    # 0.3 MB snapshot, about 1.7 MB in all; the 2.5 MB budget holds one such lattice
    probs = [W.cavity(128, Ra=1e4, ny=96, seed=k, storage=F32) for k in range(4)]
    srv = clb.Server(hbm_budget_bytes=5 << 19, max_slots=4, storage=F32)
    ids = [srv.submit(p, step_cap=96, tol=0.0) for p in probs]
    most = 0
    for _ in range(40):
        active, queued = srv.progress(32)
        most = max(most, active)
        if not active and not queued:
            break
    assert most == 1
    for rid, prob in zip(ids, probs):
        done, nu, steps, er = srv.poll(rid)
        assert done and steps == 96
        alone = clb.Batch([prob])
        alone.step(96)
        for a, b in zip(srv.fetch(rid, prob.ny, prob.nx), alone.fields(0)):
            assert np.array_equal(a, b), prob.name


def test_batch_status_reports_the_last_check(clb):
    probs = mixed_problems(F64, count=3)
    b = clb.Batch(probs)
    steps, er, status = b.run(0.0, 300, 100)
    st, er2, steps2, nu2 = b.status()
    assert (st == status).all() and (steps2 == steps).all()
    np.testing.assert_array_equal(er2, er)
    for k, prob in enumerate(probs):
        single = clb.Lattice.from_problem(prob)
        single.step(300)
        assert nu2[k] == pytest.approx(single.nusselt(prob.nu_axis), rel=1e-12, abs=1e-14)
