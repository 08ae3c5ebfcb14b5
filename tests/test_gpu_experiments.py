"""The paper's experiments on the CUDA path, against stored oracle values (written by the committed
scripts in tests/golden/ that call only the oracle) and against the paper's printed numbers."""
import json
import math
import os

import numpy as np
import pytest

from paper_1710_10569_gb300 import workloads as W
from conftest import golden_path

pytestmark = pytest.mark.gpu

F64, F32, F16 = W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def clb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10569_gb300 import clb as c
    c.lib()
    return c


def _golden(name):
    path = golden_path(name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    with open(path) as f:
        return json.load(f)


def _table1_paper():
    rows = {}
    for line in open(golden_path("table1_nusselt.txt")):
        if line.strip() and not line.startswith("#"):
            ra, an, pap, _ = line.split()
            rows[int(float(ra))] = (float(an), float(pap))
    return rows


@pytest.mark.parametrize("storage", [F64, F32])
def test_table1_rayleigh_benard_batch(clb, storage):
    """Sec. 3.3, Table 1: the eight Rayleigh numbers stepped together in one batch from the paper's
    initial state. In FP64 the Nusselt numbers at 10k, 20k and 30k steps equal the oracle's to 1e-9,
    and at 200k steps the oracle's to 1e-6 and the analytic values of Table 1 within 2.5% (0.5% for
    Ra <= 1e4). FP32 storage, whose temperature populations are stored against the conduction line
    between the walls, grows the rolls from the paper's 1e-3 density disturbance at every Ra,
    onset included, and meets the oracle's steady values to 1e-4 at 200k steps."""
    gold = _golden("table1_oracle.json")
    paper = _table1_paper()
    ras = sorted(int(k) for k in gold)
    probs = [W.rayleigh_benard_table1(float(ra), storage=storage) for ra in ras]
    b = clb.Batch(probs)
    done = 0
    for n in (10000, 20000, 30000):
        b.step(n - done)
        done = n
        nu, _ = b.diagnostics()
        if storage != F64:
            continue
        for k, ra in enumerate(ras):
            exp = gold[str(ra)]["at"][str(n)]
            assert nu[k] == pytest.approx(exp, rel=1e-9), (ra, n)
    b.step(200000 - done)
    nu, _ = b.diagnostics()
    for k, ra in enumerate(ras):
        steady = gold[str(ra)]["steady"]
        assert nu[k] == pytest.approx(steady, rel=1e-6 if storage == F64 else 1e-4), ra
        analytic = paper[ra][0]
        assert nu[k] == pytest.approx(analytic, rel=5e-3 if ra <= 10000 else 2.5e-2), ra


def test_table1_fp16_stalls_below_its_resolution(clb):
    """FP16 deviation storage keeps about 11 bits: near onset the per-step growth of the roll stays
    below half a unit in the last place of the stored deviations, so from the paper's 1e-3 density
    disturbance the layer stays at conduction (Nu within 1e-3 of 1) for Ra <= 1e4 over 200k steps,
    and the developed rolls at Ra >= 2e4 come out within 6% of the oracle. This bounds the FP16
    form: it is for developed flows, not for onset."""
    from paper_1710_10569_gb300 import experiments as X
    gold = _golden("table1_oracle.json")
    r16 = X.table1(storage=F16)
    for ra, nu in r16.items():
        if ra <= 10000:
            assert nu == pytest.approx(1.0, abs=1e-3), ra
        else:
            assert nu == pytest.approx(gold[str(ra)]["steady"], rel=0.06), ra


def test_table1_fp32_follows_onset_when_seeded(clb):
    """With a temperature disturbance (1e-3, seeded) above the FP32 storage resolution the FP32
    batch develops the same roll states as FP64 from the same disturbance, Nu within 1e-3 at
    200k steps for Ra = 2000 .. 3e4 (at 5e4 the seeded state is not steady)."""
    from paper_1710_10569_gb300 import experiments as X
    ras = (2000, 2500, 3000, 5000, 10000, 20000, 30000)
    r32 = X.table1(storage=F32, ras=ras, seed_T=1e-3)
    r64 = X.table1(storage=F64, ras=ras, seed_T=1e-3)
    for ra in ras:
        assert r64[ra] > 1.1
        assert r32[ra] == pytest.approx(r64[ra], rel=1e-3), ra


@pytest.mark.parametrize("storage", [F64, F32])
def test_cavity_256_ra1e5_steady_state(clb, storage):
    """The side-heated cavity (256^2, Ra = 1e5, Pr = 0.71) run to E_R < 1e-8: the mean Nusselt
    number equals the oracle's steady value (FP64: 1e-6 relative; FP32: 1e-3, with a step cap since
    FP32 rounding puts a floor under E_R)."""
    gold = _golden("cavity256_ra1e5.json")
    prob = W.cavity(256, Ra=1e5, Pr=0.71, u_c=0.1, seed=0, storage=storage)
    lat = clb.Lattice.from_problem(prob)
    cap = gold["steps"] + 20000
    steps, er = lat.run(1e-8, cap, 100)
    nu = lat.nusselt(prob.nu_axis)
    if storage == F64:
        assert er < 1e-8
        assert abs(steps - gold["steps"]) <= 1000
        assert nu == pytest.approx(gold["nusselt"], rel=1e-6)
    else:
        assert nu == pytest.approx(gold["nusselt"], rel=1e-3)


@pytest.mark.parametrize("storage", [F64, F32])
@pytest.mark.parametrize("Ma", [0.0, 0.3])
def test_moving_frame_diffusivity(clb, storage, Ma):
    """Sec. 3.1 on the GPU: the temperature wave's measured diffusivity equals the prescribed
    alpha = 0.05 within 0.1% for Ma = 0 and 0.3."""
    L, alpha, B = 100, 0.05, 0.01
    nx, ny = 2, L
    A_ = Ma * W.CS
    phi = 2 * math.pi / L
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    p = W.default_params(nu=0.05, kappa=alpha, T0=1.0, T_ref=1.0, storage=storage)
    prob = W.Problem("wave", nx, ny, p, np.ones((ny, nx)), np.zeros((ny, nx)),
                     A_ * np.ones((ny, nx)), 1.0 + B * np.sin(phi * y))
    lat = clb.Lattice.from_problem(prob)

    def amp():
        c = lat.fields()[3][:, 0] - 1.0
        return abs(np.sum(c * np.exp(-1j * phi * np.arange(ny)))) * 2 / ny

    lat.step(500)
    a1 = amp()
    lat.step(2000)
    a2 = amp()
    measured = -math.log(a2 / a1) / (phi * phi * 2000)
    assert measured == pytest.approx(alpha, rel=1e-3)


def test_critical_rayleigh_number(clb):
    """Sec. 3.3: the growth rate of the disturbance changes sign at Ra_c; the least-squares zero of
    the growth rates at Ra = 1702..1710 lies within 0.5% of the linear-stability value 1707.76 (the
    paper finds 1706.82)."""
    from paper_1710_10569_gb300 import experiments as X
    theory = None
    for line in open(golden_path("critical_rayleigh.txt")):
        if line.startswith("theory"):
            theory = float(line.split()[1])
    r = X.critical_rayleigh(storage=F64)
    assert r["growth_rate"][0] < 0 < r["growth_rate"][-1]
    assert np.all(np.diff(r["growth_rate"]) > 0)
    assert r["ra_c"] == pytest.approx(theory, rel=5e-3)


def test_ma_sweep_nusselt_is_insensitive(clb):
    """Sec. 3.3: over Ma = 0.1..0.3 the Nusselt number barely changes while the steps to converge
    scale like 1/Ma. The paper's own walls give 0.08% at Ra = 5000; with the walls halfway between
    nodes used here the change is 0.3-0.4% (the oracle gives the same), bounded by 0.5%."""
    from paper_1710_10569_gb300 import experiments as X
    r = X.ma_sweep(5000.0, mas=(0.1, 0.2, 0.3), tol=1e-7)
    assert r["nu_rel_change"] < 5e-3
    ratio = r["steps"][0] / r["steps"][2]
    assert 1.5 < ratio < 5.0


@pytest.mark.parametrize("storage", [F32, F64])
def test_high_rayleigh_stability(clb, storage):
    """Sec. 3.3, last paragraph: the method stays stable at Ra = 1e9 with 220 vertical nodes
    (nu ~ 1e-3, s_nu within 0.3% of 2): 200,000 steps with finite fields and bounded speeds."""
    from paper_1710_10569_gb300 import experiments as X
    r = X.stability(Ra=1e9, ny=220, steps=200000, storage=storage)
    assert r["finite"]
    assert r["max_speed_over_uc"] < 3.0
    assert r["nu"] > 1.0


def test_normal_plate_second_order_convergence(clb):
    """Sec. 3.2 on the GPU: Pr = 0.71, Re = 10, 20, 30, L = 30 .. 150 in one batch; the slopes of
    log E_u and log E_T against log(1/L) lie within 1.9 .. 2.1 (the paper: about 2)."""
    from paper_1710_10569_gb300 import experiments as X
    r = X.normal_plate_convergence()
    for re in ("10.0", "20.0", "30.0"):
        assert 1.9 < r["slope_u"][re] < 2.1, r
        assert 1.9 < r["slope_T"][re] < 2.1, r


@pytest.mark.parametrize("storage", [F64, F32])
def test_table1_with_the_papers_walls(clb, storage):
    """Table 1 with the paper's own walls (60 x 31 nodes, H = 30) for Ra = 2500 .. 1e4 in one batch:
    Nu within 0.2% of the analytic values and 0.4% of the paper's numbers after 100k steps."""
    paper = _table1_paper()
    ras = (2500, 3000, 5000, 10000)
    probs = [W.rayleigh_benard_table1(float(ra), wet=True, storage=storage) for ra in ras]
    if storage == F32:  # FP32 needs a disturbance above its resolution near onset (see DESIGN)
        rng = np.random.default_rng(0)
        for p in probs:
            p.T = p.T + rng.uniform(-1e-3, 1e-3, p.T.shape)
    b = clb.Batch(probs)
    b.step(100000)
    nu, _ = b.diagnostics()
    for k, ra in enumerate(ras):
        assert nu[k] == pytest.approx(paper[ra][0], rel=2e-3), ra
        assert nu[k] == pytest.approx(paper[ra][1], rel=4e-3), ra


def test_normal_plate_convergence_with_the_papers_walls(clb):
    """Sec. 3.2 with the paper's own walls on the GPU (15 channels in one batch): the errors fall
    towards second order; at Re Pr = 21 the thermal layer is steep and the order is still rising
    over L = 30..150 (1.45, 1.67, 1.77, 1.82 pairwise), so the test asks for an overall slope above
    1.5 and an order above 1.75 between the two finest grids, for u and T at every Re."""
    from paper_1710_10569_gb300 import experiments as X
    r = X.normal_plate_convergence(wet=True)
    Ls = r["L"]
    for re in ("10.0", "20.0", "30.0"):
        for key in ("u", "T"):
            assert 1.5 < r[f"slope_{key}"][re] < 2.2, (re, key, r[f"slope_{key}"])
            e = r[f"E_{key}"][re]
            assert math.log(e[-2] / e[-1]) / math.log(Ls[-1] / Ls[-2]) > 1.75, (re, key, e)
