"""3-D batches (clb3d_batch_*): every lattice of a batch evolves bitwise as it does alone through the
single-lattice step, whatever the batch's tile shape, groups of rows per block and the times its
lattices are (re)initialised; the batch's first lattice also matches the FP64 oracle."""
import dataclasses

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


def mixed3(storage):
    """Uneven extents (odd and even, below and above one block), random faces (some moving) and
    rates (the general collision), plus a Rayleigh-Benard box with the paper's rates (the form that
    skips the high-order moments)."""
    shapes = [(5, 7, 3), (33, 4, 6), (40, 9, 5), (130, 3, 4), (17, 17, 17)]
    probs = [W.random_problem3d(nx, ny, nz, seed=k, storage=storage, moving=k % 2 == 1)
             for k, (nx, ny, nz) in enumerate(shapes)]
    probs.append(W.rayleigh_benard3d(24, 12, 10, Ra=1e5, storage=storage))
    return probs


def alone(clb, prob, steps):
    lat = clb.Lattice3D.from_problem(prob)
    lat.step(steps)
    return lat


def assert_same(a, b, what):
    for x, y in zip(a, b):
        assert np.array_equal(x, y), what


@pytest.mark.parametrize("storage", [F64, F32, F16])
def test_batch_equals_single_lattices(clb, storage):
    probs = mixed3(storage)
    b = clb.Batch3D(probs)
    b.step(37)  # one graph chunk and single launches
    for k, prob in enumerate(probs):
        lat = alone(clb, prob, 37)
        assert_same(b.fields(k), lat.fields(), prob.name)
        fb, gb = b.member(k).populations()
        fl, gl = lat.populations()
        assert np.array_equal(fb, fl) and np.array_equal(gb, gl), prob.name
        assert b.member(k).nusselt(prob.nu_axis) == lat.nusselt(prob.nu_axis)
        assert b.member(k).residual() == lat.residual()
    b.close()


@pytest.mark.parametrize("tile", [(32, 1), (64, 2), (128, 2), (256, 1), (32, 8)])
def test_tile_shape_does_not_change_results(clb, tile):
    probs = mixed3(F32)
    ref = clb.Batch3D(probs)
    ref.step(9)
    b = clb.Batch3D(probs)
    b.set_tile(*tile)
    assert b.launch()["block"] == tile
    b.step(9)
    for k in range(len(probs)):
        assert_same(b.fields(k), ref.fields(k), (tile, k))


def test_row_groups_per_block(clb):
    """A batch large enough that each block steps several groups of rows equals the lattices alone;
    a small batch keeps one group per block."""
    probs = [W.random_problem3d(64 + 3 * k, 48, 40 + k, seed=10 + k, storage=F32) for k in range(12)]
    b = clb.Batch3D(probs)
    launch = b.launch()
    assert launch["groups"] >= 2, launch
    b.step(5)
    for k in (0, 5, 11):
        assert_same(b.fields(k), alone(clb, probs[k], 5).fields(), k)
    assert clb.Batch3D(probs[:1]).launch()["groups"] == 1


def test_reinitialised_lattice_restarts(clb):
    """Lattice 1 re-initialised after an odd number of batch steps (its state then sits in the other
    buffer of the pair than the batch's parity suggests) evolves as a fresh lattice; the others go on."""
    probs = mixed3(F32)[:3]
    b = clb.Batch3D(probs)
    b.step(5)
    new = dataclasses.replace(W.random_problem3d(probs[1].nx, probs[1].ny, probs[1].nz, seed=99, storage=F32),
                              params=probs[1].params)
    b.init_fields(1, *new.fields())
    b.step(40)
    assert_same(b.fields(0), alone(clb, probs[0], 45).fields(), "untouched lattice")
    assert_same(b.fields(1), alone(clb, new, 40).fields(), "re-initialised lattice")
    assert_same(b.fields(2), alone(clb, probs[2], 45).fields(), "untouched lattice")


def test_batch_matches_oracle(clb):
    prob = W.random_problem3d(9, 6, 5, seed=3, storage=F64, moving=True)
    b = clb.Batch3D([prob, W.random_problem3d(12, 5, 7, seed=4, storage=F64)])
    b.step(20)
    o = oracle.Oracle3D.from_problem(prob)
    o.step(20)
    for got, exp in zip(b.fields(0), o.fields()):
        assert np.max(np.abs(got - exp)) <= 1e-12 * max(np.max(np.abs(exp)), 0.05)


def test_member_cannot_be_stepped_alone(clb):
    b = clb.Batch3D(mixed3(F32)[:2])
    with pytest.raises(RuntimeError):
        b.member(0).step(1)
