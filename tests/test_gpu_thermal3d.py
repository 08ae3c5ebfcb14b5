"""The 3-D thermal-only mode (D3Q7 with a prescribed velocity, include/clb3d.h clb3d_thermal_*)
against the 3-D oracle's thermal-only mode, with the tolerances of test_gpu_parity3d.py."""
import math

import numpy as np
import pytest

import oracle
from paper_1710_10569_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F64, F32, F16 = W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV
P, D, A = W.WALL_PERIODIC, W.WALL_DIRICHLET, W.WALL_ADIABATIC
U32, U16 = 2.0 ** -24, 2.0 ** -11


def tol(storage, steps):
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


def _case(storage, walls, seed, shape=(19, 6, 7)):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    ux = 0.08 * np.sin(2 * math.pi * x / nx) * np.cos(2 * math.pi * y / ny)
    uy = -0.08 * np.cos(2 * math.pi * x / nx) * np.sin(2 * math.pi * y / ny)
    uz = 0.03 * np.sin(2 * math.pi * z / nz)
    T = rng.uniform(-0.5, 0.5, (nz, ny, nx))
    p = W.default_params3(kappa=float(rng.uniform(0.01, 0.1)), lambda2=float(rng.uniform(0.8, 1.5)),
                          wall=walls, T_wall=tuple(float(v) for v in rng.uniform(-0.5, 0.5, 6)),
                          storage=storage, thermal_only=1, dT_ref=0.5)
    return p, T, ux, uy, uz


@pytest.mark.parametrize("storage", [F64, F32, F16], ids=["f64", "f32", "f16dev"])
@pytest.mark.parametrize("walls", [(P,) * 6, (P, P, D, A, D, D), (A, D, A, A, D, A)], ids=["periodic", "walls", "box"])
def test_thermal_only_matches_the_oracle(clb, storage, walls):
    p, T, ux, uy, uz = _case(storage, walls, seed=len(walls) + walls.count(D))
    nz, ny, nx = T.shape
    o = oracle.Oracle3D(nx, ny, nz, p)
    o.init(1.0, ux, uy, uz, T)
    th = clb.Thermal3D(nx, ny, nz, p)
    th.init(T, ux, uy, uz)
    for k in (1, 40):
        o.step(k - o.steps)
        th.step(k - (1 if k == 40 else 0))
        got, exp = th.temperature(), o.fields()[4]
        err = float(np.max(np.abs(got - exp))) / max(float(np.max(np.abs(exp))), 0.5)
        assert err <= tol(storage, k), (k, err)
    if storage == F64:
        np.testing.assert_allclose(th.populations(), o.populations()[1], atol=1e-13)
    th.close()


def test_thermal_only_moving_frame_diffusivity(clb):
    """Sec. 3.1 in 3-D on the GPU: a temperature wave along z in a uniform prescribed flow
    (0.1, 0.12, -0.08) keeps alpha = 0.05 within 0.1%."""
    L, alpha, B = 60, 0.05, 0.01
    p = W.default_params3(nu=0.05, kappa=alpha, T0=1.0, T_ref=1.0, thermal_only=1, storage=F64)
    zc = np.arange(L, dtype=np.float64).reshape(L, 1, 1)
    th = clb.Thermal3D(1, 1, L, p)
    th.init(1.0 + B * np.sin(2 * math.pi * zc / L), 0.1, 0.12, -0.08)
    k = 2 * math.pi / L

    def amp():
        c = th.temperature().reshape(-1) - 1.0
        return abs(np.sum(c * np.exp(-1j * k * np.arange(L)))) * 2 / L

    th.step(300)
    a1 = amp()
    th.step(1500)
    a2 = amp()
    assert -math.log(a2 / a1) / (k * k * 1500) == pytest.approx(alpha, rel=1e-3)
    th.close()
