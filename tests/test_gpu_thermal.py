"""The thermal-only mode (D2Q5 with a prescribed velocity) on the GPU against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_10569_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64, F32, F16 = W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV
P, D, A = W.WALL_PERIODIC, W.WALL_DIRICHLET, W.WALL_ADIABATIC
U32, U16 = 2.0 ** -24, 2.0 ** -11


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def cellular(nx, ny, U, seed):
    x, y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    kx, ky = math.pi / nx, math.pi / ny
    ux = U * np.sin(kx * x) * np.cos(ky * y)
    uy = -U * np.cos(kx * x) * np.sin(ky * y)
    T = np.random.default_rng(seed).uniform(-0.5, 0.5, (ny, nx))
    return ux, uy, T


def tol(storage, n):
    return 1e-12 if storage == F64 else (max(1e-6, 2 * n * U32) if storage == F32 else 2 * n ** 0.5 * U16)


WET = W.WALL_WET


@pytest.mark.parametrize("storage", [F64, F32, F16])
@pytest.mark.parametrize("walls", [(P, P, P, P), (D, D, A, A), (P, P, D, D), (A, D, D, A), (P, P, WET, WET),
                                   (WET, WET, P, P), (WET, WET, WET, WET)],
                         ids=["periodic", "cavity", "rb", "mixed", "wet_y", "wet_x", "wet_box"])
@pytest.mark.parametrize("shape", [(67, 45), (3, 130), (2, 2), (300, 7)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_thermal_parity(clb, storage, walls, shape):
    """Every node's temperature against the oracle's thermal-only mode, on halfway walls, on the
    paper's own (wet) walls on either axis and in a closed wet box (corners), on rows wider than a
    block of the field kernel."""
    nx, ny = shape
    if WET in walls and min(nx, ny) < 3:
        pytest.skip("wet walls need 3 nodes across")
    p = W.default_params(kappa=0.04, wall=walls, T_wall=(0.4, -0.3, 0.2, -0.5), lambda2=1.2,
                         storage=storage, T_ref=0.0)
    ux, uy, T = cellular(nx, ny, 0.08, seed=nx)
    th = clb.Thermal(nx, ny, p)
    th.init(T, ux, uy)
    th.step(90)
    got = th.temperature()
    po = dict(p)
    po["thermal_only"] = 1
    o = oracle.Oracle(nx, ny, po)
    o.init(np.ones((ny, nx)), ux, uy, T)
    o.step(90)
    exp = o.fields()[3]
    err = float(np.max(np.abs(got - exp))) / max(float(np.max(np.abs(exp))), 0.5)
    assert err <= tol(storage, 90), err
    if storage == F64:
        _, go = o.populations()
        assert np.max(np.abs(th.populations() - go)) <= 1e-13


@pytest.mark.parametrize("storage", [F64, F32])
def test_thermal_moving_frame_diffusivity(clb, storage):
    """Sec. 3.1 with the thermal-only kernel: alpha measured within 0.1% at Ma = 0.3."""
    L, alpha, B = 100, 0.05, 0.01
    nx, ny = 2, L
    A_ = 0.3 * W.CS
    phi = 2 * math.pi / L
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    p = W.default_params(kappa=alpha, T0=1.0, T_ref=1.0, storage=storage)
    th = clb.Thermal(nx, ny, p)
    th.init(1.0 + B * np.sin(phi * y), np.zeros((ny, nx)), A_ * np.ones((ny, nx)))

    def amp():
        c = th.temperature()[:, 0] - 1.0
        return abs(np.sum(c * np.exp(-1j * phi * np.arange(ny)))) * 2 / ny

    th.step(500)
    a1 = amp()
    th.step(2000)
    a2 = amp()
    assert -math.log(a2 / a1) / (phi * phi * 2000) == pytest.approx(alpha, rel=1e-3)
