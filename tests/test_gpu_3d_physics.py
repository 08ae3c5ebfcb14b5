"""The 3-D path on physics the paper fixes (Sec. 3.3, Table 1): convection rolls in a box that is
thin along y reproduce the two-dimensional Nusselt numbers."""
import numpy as np
import pytest

from paper_1710_10569_gb300 import workloads as W
from conftest import golden_path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def _table1():
    rows = {}
    for line in open(golden_path("table1_nusselt.txt")):
        if line.strip() and not line.startswith("#"):
            ra, an, pap, _ = line.split()
            rows[int(float(ra))] = (float(an), float(pap))
    return rows


@pytest.mark.parametrize("storage", [W.STORAGE_F64, W.STORAGE_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("Ra", [5000, 10000])
def test_rayleigh_benard_rolls_in_3d_match_table1(clb, Ra, storage):
    """60 x 4 x 30 nodes (periodic in x and y, Dirichlet walls on the z faces, H = 30), Pr = 0.71,
    Ma = 0.3, a seeded 1e-3 temperature disturbance: after 150,000 steps the rolls (axes along y)
    carry the Nusselt number of Table 1 within 2.5% of the analytic value, as the two-dimensional
    path does with the same walls."""
    prob = W.rayleigh_benard3d(60, 4, 30, Ra=float(Ra), u_c=0.3 / 3 ** 0.5, perturb=1e-3, storage=storage)
    lat = clb.Lattice3D.from_problem(prob)
    lat.step(150000)
    nu = lat.nusselt(2)
    _, ux, uy, uz, _ = lat.fields()
    lat.close()
    analytic = _table1()[Ra][0]
    assert nu == pytest.approx(analytic, rel=2.5e-2)
    # rolls with axes along y: the flow does not vary along y and has no y component
    assert float(np.max(np.abs(uy))) < 1e-3 * float(np.max(np.abs(uz)))
