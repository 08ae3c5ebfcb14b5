"""Throughput of the fused coupled D2Q9 + D2Q5 central-moment LBM step on GB300.

Workload (default): Rayleigh-Benard convection in a 2:1 box, 2048 x 1024 nodes, periodic in x,
Dirichlet walls T = +-0.5 at the bottom/top, Ra = 1e7, Pr = 0.71, u_c = 0.1, seeded T perturbation
1e-3, FP32 population storage and FP32 arithmetic. One bench step = one time step of the whole
lattice (every node: pull, macroscopics, D2Q9 and D2Q5 central-moment collision, store).

Metric: MLUPS (million coupled node updates per second), with the fused step kernel's fraction of
the measured HBM copy bandwidth. The timed region runs K steps through clb_run (the fused step every
step, the FP64 Nusselt number and residual every 100 steps and after the last one) on the lattice's
stream; the two population buffers (2 x 117 MB in FP32) exceed the 129 MB L2. The roofline times the
step kernel alone over a fixed window of 2048 graph-replayed launches (both graph parities captured
before the window), and the DRAM bytes per launch measured by ncu are reported beside the
algorithmic bytes.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun) every rank steps its own replica of the lattice (replicas only: the
workload is one lattice per GPU and no data crosses GPUs); value = all ranks' node updates / the
slowest rank's time.

Beside the headline the JSON line carries (rank 0, N = 1): `e2e` (the same run through the C ABI
from pinned host fields), `cpu_baseline` (the FP64 oracle on the host cores), `variants` (FP16
deviation storage on 4096 x 2048, FP64), `thermal_only` (D2Q5 alone, 4096 x 4096), `three_d`
(D3Q27 + D3Q7 on 256 x 256 x 128 in three storage forms, a batch of 48 uneven boxes, the D3Q7
thermal-only step on 256^3), `batched` (256 uneven cavities in one launch per step, a fixed 1,000
steps, and `to_steady_state`: every cavity run to E_R < 1e-6 or the 500k-step cap with retirement,
against the plain FP64 path on a seeded subset), `served` (a Poisson request trace, every request run
to steady state, against the plain FP64 one-at-a-time path) and `rb_long` (Rayleigh-Benard 2048 x
1024 for 200,000 steps in FP64, FP32 and FP16 deviation storage, Nusselt statistics per form).
`--served-large` runs a served trace over edges 64-4096 instead; `--thermal-only`, `--three-d-only`,
`--batched-only`, `--steady-only` and `--rb-long` run one part alone; `--no-long` skips the
steady-state and 200,000-step runs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1710_10569_gb300 import workloads as W  # noqa: E402

BYTES_PER_NODE = {W.STORAGE_F64: 224, W.STORAGE_F32: 112, W.STORAGE_F16DEV: 56}  # 14 in + 14 out
DTYPE = {W.STORAGE_F64: "f64", W.STORAGE_F32: "f32", W.STORAGE_F16DEV: "f16dev storage, f32 arithmetic"}
# Lattice of each storage form when it runs as a variant beside the headline: FP16 storage moves
# 56 B per node, so at 2048 x 1024 a step's 117 MB would fit the 129 MB L2; it runs at 4096 x 2048.
VARIANT_SIZE = {W.STORAGE_F64: (2048, 1024), W.STORAGE_F32: (2048, 1024), W.STORAGE_F16DEV: (4096, 2048)}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_traffic.json")
KERNEL_SOURCES = ["paper_1710_10569_gb300/csrc/clb_core.cuh", "paper_1710_10569_gb300/csrc/clb_kernels.cuh"]
KERNEL3D_SOURCES = ["paper_1710_10569_gb300/csrc/clb_core.cuh", "paper_1710_10569_gb300/csrc/clb3d.cu"]


_CODE_TOKENS = re.compile(r'"(?:\\.|[^"\\\n])*"|//[^\n]*|/\*.*?\*/|\s+', re.S)


def _code_only(text: str) -> str:
    """The source with its comments dropped (string literals kept) and each run of white space
    made one blank, so that an edit of comments or layout leaves the hash alone."""
    def keep(m):
        t = m.group(0)
        return t if t.startswith('"') else " "
    return re.sub(r"\s+", " ", _CODE_TOKENS.sub(keep, text)).strip()


def kernel_hash(sources=KERNEL_SOURCES) -> str:
    """Hash of the code (not the comments) of the kernel sources the committed ncu counts were
    taken on."""
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# GB300 FP64 issue rate: 152 SMs x 2 DP lanes per clock x 2.07 GHz (the 1.26 TFLOP/s FP64 figure
# with an FMA counted as two flops)
FP64_DP_INSTR_PEAK = 152 * 2 * 2.07e9


def profile_counts():
    """The committed ncu counts, if taken on the current kernel source (else {})."""
    if not os.path.exists(TRAFFIC_FILE):
        return {}
    with open(TRAFFIC_FILE) as f:
        d = json.load(f)
    return d if d.get("kernel_source_hash") == kernel_hash() else {}


def flops_per_node():
    """Floating-point operations per node update (an FMA counted as two), from the FP64 step's
    committed ncu instruction counts, if they were taken on the current kernel source (else None).
    The FP32 and FP16 forms evaluate the same expressions except the ten 1-D inverse pairs
    (s + d)/2, (s - d)/2 per node, which their packed pairs form as two sums and two halvings (4
    flops) where FP64 uses one halving and two FMAs (5 flops): 8 flops fewer per node."""
    ops = profile_counts().get("fp64_ops_per_node")
    if not ops:
        return None
    return 2 * ops["dfma"] + ops["dadd"] + ops["dmul"]


def traffic_per_launch(storage: int, nx: int, ny: int):
    """DRAM bytes of one step's kernel launch (for the FP16 form the step's interior and edge
    kernels together) on an nx x ny lattice from the committed ncu summary, if it was taken on the
    current kernel source and that lattice (else None)."""
    e = profile_counts().get("launches", {}).get(W.STORAGE_NAMES[storage])
    if not e or e.get("nx") != nx or e.get("ny") != ny:
        return None
    return float(e["dram_bytes_per_launch"])


def traffic3d_per_launch(storage: int, nx: int, ny: int, nz: int):
    """DRAM bytes per 3-D step-kernel launch from the committed ncu summary, if it was taken on the
    current 3-D kernel source and that lattice (else None)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        d = json.load(f)
    if d.get("kernel3d_source_hash") != kernel_hash(KERNEL3D_SOURCES):
        return None
    e = d.get("launches3d", {}).get(W.STORAGE_NAMES[storage])
    if not e or (e.get("nx"), e.get("ny"), e.get("nz")) != (nx, ny, nz):
        return None
    return float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self):
        if not self.proc:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(units: float, seconds: float, world: int):
    """Whole-job throughput: total units over all ranks / the slowest rank's time."""
    if world == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([units, seconds], dtype=torch.float64, device=dev)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def kernels_per_step(storage: int) -> int:
    """Kernels one step launches on a Rayleigh-Benard lattice: the FP16 form splits the step into
    an interior kernel and an edge kernel (wall rows) that run side by side."""
    return 2 if storage == W.STORAGE_F16DEV else 1


def step_kernel_name(storage: int) -> str:
    if storage == W.STORAGE_F16DEV:
        return "k_step_inner_f16x4_hi1 + k_step_edge<f16dev> (one step)"
    return f"k_step<{W.STORAGE_NAMES[storage]}>"


def workload(storage: int, nx: int = 2048, ny: int = 1024):
    return W.rayleigh_benard(nx, ny, Ra=1e7, Pr=0.71, u_c=0.1, perturb=1e-3, seed=0, storage=storage)


DIAG_INTERVAL = 100  # steps between the FP64 Nusselt / residual reductions of a run


def time_run(lat, steps: int, warmup: int, world: int):
    """Device time of `steps` time steps run the way a user runs to a steady state (clb_run): the
    fused step every step and the FP64 Nusselt number / residual reduction, read back to the host,
    every DIAG_INTERVAL steps (tolerance 0, so the run never stops early)."""
    import torch
    lat.run(0.0, warmup, DIAG_INTERVAL)
    lat.sync()
    stream = torch.cuda.ExternalStream(lat.stream) if lat.stream else torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    lat.run(0.0, steps, DIAG_INTERVAL)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    return e0.elapsed_time(e1) / 1e3


KERNEL_WINDOW = 2048  # launches of the step kernel timed for the roofline (64 graph replays)


def diag_checks(steps: int) -> int:
    """FP64 Nusselt / residual checks that clb_run makes over `steps` steps: one every
    DIAG_INTERVAL steps and one after the last step."""
    return -(-steps // DIAG_INTERVAL)


def time_steps(lat, steps: int, warmup: int, world: int):
    """Device time of `steps` launches of the fused step kernel alone (graph replays). The
    warm-up runs 64 steps first: the library captures the graphs of both buffer parities on its
    first 32-step chunk, so no capture or instantiation falls inside the timed window."""
    import torch
    lat.step(64 + warmup)
    lat.sync()
    stream = torch.cuda.ExternalStream(lat.stream) if lat.stream else torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    return e0.elapsed_time(e1) / 1e3


def cpu_baseline(storage: int, nx: int, ny: int, seconds: float = 10.0):
    """The oracle, as it stands, on the full bench lattice for as many steps as take about
    `seconds` (one step timed first to size the sample)."""
    import oracle
    prob = workload(storage, nx, ny)
    o = oracle.Oracle.from_problem(prob)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    sample_steps = int(min(400, max(3, seconds / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.step(sample_steps)
    dt = time.perf_counter() - t0
    return {"value": prob.nodes * sample_steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.threads(),
            "kind": "oracle",
            "sample": f"{sample_steps} steps of the full {prob.nx}x{prob.ny} lattice (FP64 oracle, "
                      f"{oracle.threads()} OpenMP threads), {dt:.1f} s"}


def e2e_run(storage: int, steps: int, nx: int, ny: int):
    """The same metric through the public C ABI with host buffers: upload the initial fields from
    pinned host memory, step, and read the fields back, all inside the timed region."""
    import torch
    from paper_1710_10569_gb300 import clb
    prob = workload(storage, nx, ny)
    n = prob.nodes
    pin = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(8)]
    for t, a in zip(pin[:4], prob.fields()):
        t.numpy()[:] = a.ravel()
    lat = clb.Lattice(prob.nx, prob.ny, prob.params)
    lat.init_fields(*[t.numpy() for t in pin[:4]])
    lat.step(64)
    lat.sync()
    t0 = time.perf_counter()
    lat.init_fields(*[t.numpy() for t in pin[:4]])
    lat.run(0.0, steps, DIAG_INTERVAL)
    lat.fields_into(*[t.numpy() for t in pin[4:]])
    dt = time.perf_counter() - t0
    lat.close()
    diag_bytes = 8 * 8 * diag_checks(steps)  # Nu, residual and the final sums read per check
    return {"value": n * steps / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": 4 * 8 * n / steps, "d2h_bytes_per_step": (4 * 8 * n + diag_bytes) / steps,
            "steps": steps, "seconds": dt,
            "path": "pinned host fields -> clb_init_fields -> clb_run (diagnostics every "
                    f"{DIAG_INTERVAL} steps) -> clb_fields -> pinned host"}


def thermal_run(storage: int, steps: int, nx: int = 4096, ny: int = 4096):
    """The D2Q5-only step with a prescribed velocity (a cellular flow of amplitude 0.1) on a
    Rayleigh-Benard temperature field: 5 populations in and out plus the node's velocity. The
    lattice is 4096 x 4096 so that a step's working set (two 336 MB FP32 buffers and 134 MB of
    velocities) is several times the 129 MB L2; at 2048 x 1024 it would fit."""
    import torch
    from paper_1710_10569_gb300 import clb
    prob = workload(storage, nx, ny)
    nx, ny = prob.nx, prob.ny
    x, y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    ux = 0.1 * np.sin(kx * x) * np.cos(ky * y)
    uy = -0.1 * np.cos(kx * x) * np.sin(ky * y)
    th = clb.Thermal(nx, ny, prob.params)
    th.init(prob.T, ux, uy)
    th.step(64)
    th.sync()
    stream = torch.cuda.ExternalStream(th.stream) if th.stream else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    th.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    th.close()
    per_node = {W.STORAGE_F64: 96, W.STORAGE_F32: 48, W.STORAGE_F16DEV: 28}[storage]
    peak, _ = measured_peaks()
    gbs = per_node * nx * ny * steps / dt / 1e9
    return {"workload": f"thermal_only_{nx}x{ny}_cellular_flow", "mlups": nx * ny * steps / dt / 1e6,
            "bytes_per_node": per_node, "achieved_gbs": gbs, "hbm_frac": gbs / peak, "steps": steps,
            "storage": W.STORAGE_NAMES[storage]}


def batched_run(storage: int, count: int = 256, steps: int = 1000, seq_subset: int = 32):
    """Many side-heated cavities of uneven sizes (edge log-uniform 64-512, Ra log-uniform 1e3-1e6,
    Pr uniform 0.71-7) stepped in one launch per time step, against the same instances stepped one
    after another through single-lattice handles (a seeded subset of `seq_subset` instances is timed
    both ways)."""
    import torch
    from paper_1710_10569_gb300 import clb
    probs = W.batch_cavities(count, seed=0, storage=storage)
    nodes = sum(p.nodes for p in probs)

    def device_seconds(stream_handle, fn):
        """CUDA-event time of fn's work on the given stream."""
        st = torch.cuda.ExternalStream(stream_handle) if stream_handle else torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def time_batch(ps, k):
        b = clb.Batch(ps)
        b.autotune()
        launch = b.launch()
        b.step(64)
        dt = device_seconds(b.stream, lambda: b.step(k))
        b.close()
        return dt, launch

    dt_all, launch = time_batch(probs, steps)
    peak, _ = measured_peaks()
    sub = probs[:seq_subset]
    sub_nodes = sum(p.nodes for p in sub)
    dt_sub, _ = time_batch(sub, steps)
    lats = [clb.Lattice.from_problem(p) for p in sub]  # all on torch's current stream
    for lat in lats:
        lat.step(64)

    def sequential():
        for lat in lats:
            lat.step(steps)

    dt_seq = device_seconds(lats[0].stream, sequential)
    for lat in lats:
        lat.close()
    return {"instances": count, "nodes": nodes, "steps": steps, "storage": W.STORAGE_NAMES[storage],
            "tile": list(launch["tile"]), "row_groups_per_block": launch["groups"],
            "blocks_per_launch": launch["blocks"], "mlups": nodes * steps / dt_all / 1e6,
            "hbm_frac": nodes * steps * BYTES_PER_NODE[storage] / dt_all / 1e9 / peak,
            "instance_steps_per_s": count * steps / dt_all,
            "subset": {"instances": seq_subset, "batched_mlups": sub_nodes * steps / dt_sub / 1e6,
                       "sequential_mlups": sub_nodes * steps / dt_seq / 1e6,
                       "speedup": dt_seq / dt_sub}}


BYTES_PER_NODE_3D = {W.STORAGE_F64: 544, W.STORAGE_F32: 272, W.STORAGE_F16DEV: 136}  # 34 in + 34 out


def three_d_run(steps: int, nx: int = 256, ny: int = 256, nz: int = 128):
    """The 3-D form (D3Q27 + D3Q7): Rayleigh-Benard on nx x ny x nz, Ra = 1e7, timed with CUDA
    events on the lattice's stream: FP32 deviation storage (HBM roofline at 272 B/node), FP16
    deviation storage (136 B/node) and FP64 (FP64 issue-bound; a shorter window)."""
    import torch
    from paper_1710_10569_gb300 import clb
    peak, _ = measured_peaks()
    out = {}
    for st, k in ((W.STORAGE_F32, steps), (W.STORAGE_F16DEV, steps), (W.STORAGE_F64, max(32, steps // 32))):
        prob = W.rayleigh_benard3d(nx, ny, nz, Ra=1e7, storage=st)
        lat = clb.Lattice3D.from_problem(prob)
        lat.step(64)
        stream = torch.cuda.ExternalStream(lat.stream) if lat.stream else torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        lat.close()
        gbs = BYTES_PER_NODE_3D[st] * prob.nodes * k / dt / 1e9
        out[W.STORAGE_NAMES[st]] = {"mlups": prob.nodes * k / dt / 1e6, "achieved_gbs": gbs,
                                    "hbm_frac": gbs / peak, "steps": k,
                                    "bytes_per_node": BYTES_PER_NODE_3D[st],
                                    "dram_bytes_per_launch": traffic3d_per_launch(st, nx, ny, nz)}
    out["workload"] = f"rayleigh_benard3d_{nx}x{ny}x{nz}_Ra1e7_Pr0.71"
    out["kernel"] = "k_step3"
    out["thermal_only"] = thermal3d_run(steps)
    out["batched"] = batched3d_run(steps)
    return out


def batched3d_run(steps: int, count: int = 48, seq_subset: int = 12):
    """A 3-D batch: 48 Rayleigh-Benard boxes with extents log-uniform in 24-128 (each axis drawn
    separately), FP32, one k_step3_batched launch per step, against a seeded subset stepped one
    lattice after another through single-lattice launches; CUDA events on the batch's stream."""
    import torch
    from paper_1710_10569_gb300 import clb
    peak, _ = measured_peaks()
    st = W.STORAGE_F32
    probs = W.batch_boxes3d(count, seed=0, storage=st)

    def timed(stream_handle, fn):
        s = torch.cuda.ExternalStream(stream_handle) if stream_handle else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def batch_time(ps):
        b = clb.Batch3D(ps)
        b.step(64)
        dt = timed(b.stream, lambda: b.step(steps))
        launch = b.launch()
        b.close()
        return dt, launch

    nodes = sum(p.nodes for p in probs)
    dt, launch = batch_time(probs)
    sub = probs[:seq_subset]
    sub_nodes = sum(p.nodes for p in sub)
    dt_sub, _ = batch_time(sub)
    lats = [clb.Lattice3D.from_problem(p) for p in sub]
    for lat in lats:
        lat.step(64)

    def sequential():
        for lat in lats:
            lat.step(steps)

    dt_seq = timed(lats[0].stream, sequential)
    for lat in lats:
        lat.close()
    gbs = BYTES_PER_NODE_3D[st] * nodes * steps / dt / 1e9
    return {"instances": count, "nodes": nodes, "steps": steps, "storage": W.STORAGE_NAMES[st],
            "block": list(launch["block"]), "row_groups_per_block": launch["groups"],
            "blocks_per_launch": launch["blocks"], "mlups": nodes * steps / dt / 1e6,
            "achieved_gbs": gbs, "hbm_frac": gbs / peak,
            "subset": {"instances": seq_subset, "batched_mlups": sub_nodes * steps / dt_sub / 1e6,
                       "sequential_mlups": sub_nodes * steps / dt_seq / 1e6, "speedup": dt_seq / dt_sub}}


def thermal3d_run(steps: int, n: int = 256):
    """The 3-D thermal-only step (D3Q7 with a prescribed cellular velocity) on n^3 nodes, FP32
    deviation storage: 7 populations in and out plus 3 velocity components in = 68 B/node."""
    import torch
    from paper_1710_10569_gb300 import clb
    p = W.default_params3(kappa=0.02, storage=W.STORAGE_F32, thermal_only=1,
                          wall=(W.WALL_PERIODIC,) * 4 + (W.WALL_DIRICHLET,) * 2, T_wall=(0.0,) * 4 + (0.5, -0.5))
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) + 0.5,) * 3, indexing="ij")
    k = 2 * math.pi / n
    th = clb.Thermal3D(n, n, n, p)
    th.init(0.5 - z / n, 0.1 * np.sin(k * x) * np.cos(k * y), -0.1 * np.cos(k * x) * np.sin(k * y), 0.0)
    th.step(64)
    stream = torch.cuda.ExternalStream(th.stream) if th.stream else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    th.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    th.close()
    peak, _ = measured_peaks()
    nodes = n ** 3
    gbs = 68 * nodes * steps / dt / 1e9
    return {"workload": f"thermal_only3d_{n}^3_cellular_flow", "mlups": nodes * steps / dt / 1e6,
            "bytes_per_node": 68, "achieved_gbs": gbs, "hbm_frac": gbs / peak, "steps": steps, "storage": "f32"}


def served_run(storage: int, count: int = 48, step_cap: int = 500000, tol: float = 1e-6,
               plain_tol: float = 1e-8, lo: int = 32, hi: int = 128, rb_Ra=(2.5e3, 2.5e4),
               hbm_budget_gb: int = 32, plain_same_tol: bool = True):
    """A seeded Poisson request trace (mean 50 requests/s; periodic Taylor-Green, side-heated
    cavity (Ra 1e3-1e6) and Rayleigh-Benard (Ra in rb_Ra, where the rolls are steady); edges
    log-uniform lo-hi, aspect 1 or 2), each request run to steady state: served with continuous
    batching in `storage` to E_R < tol (FP32 rounding keeps E_R above ~1e-7, so tol sits above that
    floor), against the plain FP64 one-at-a-time path to E_R < plain_tol on the same trace (and,
    with plain_same_tol, to the served tolerance as well). The Nusselt numbers of the two paths are
    compared request by request."""
    from paper_1710_10569_gb300 import serve
    trace = W.request_trace(count=count, seed=0, rate_hz=50.0, lo=lo, hi=hi, storage=storage,
                            rb_Ra_range=rb_Ra)
    s_sum, s_rec = serve.serve_trace(trace, storage, hbm_budget_bytes=hbm_budget_gb << 30, max_slots=256,
                                     chunk=100, step_cap=step_cap, tol=tol)
    p_sum, p_rec = serve.plain_trace(trace, step_cap=step_cap, tol=plain_tol)
    out = {"requests": count, "edges": [lo, hi], "rayleigh_benard_Ra": list(rb_Ra), "step_cap": step_cap,
           "tol": tol, "plain_tol": plain_tol,
           "node_updates": float(sum(r["nodes"] * r["steps"] for r in s_rec)),
           "storage": W.STORAGE_NAMES[storage],
           "served": s_sum, "plain_f64": p_sum,
           "speedup_solves_per_s": s_sum["solves_per_s"] / p_sum["solves_per_s"],
           "p99_ratio_plain_over_served": p_sum["p99_s"] / s_sum["p99_s"],
           "nusselt_vs_plain_f64": serve.nusselt_agreement(s_rec, p_rec, tol, plain_tol)}
    if plain_same_tol and plain_tol != tol:
        q_sum, _ = serve.plain_trace(trace, step_cap=step_cap, tol=tol)
        out["plain_f64_same_tol"] = q_sum
        out["speedup_solves_per_s_same_tol"] = s_sum["solves_per_s"] / q_sum["solves_per_s"]
        out["p99_ratio_same_tol"] = q_sum["p99_s"] / s_sum["p99_s"]
    return out


def batched_steady_run(count: int = 256, tol: float = 1e-6, plain_tol: float = 1e-8, cap: int = 500000,
                       subset: int = 8, subset_max_edge: int = 160):
    """The 256 uneven cavities (FP32) run to steady state with retirement (clb_batch_run: every 100
    steps the instances with E_R < tol or at the cap leave the launch), against the plain FP64
    one-at-a-time path to E_R < plain_tol on a seeded subset of `subset` instances drawn from those
    with edges <= subset_max_edge (the cheapest for the plain path, so its solves/s is on the high
    side). The Nusselt numbers of the subset are compared between the two paths."""
    from paper_1710_10569_gb300 import clb
    probs = W.batch_cavities(count, seed=0, storage=W.STORAGE_F32)
    b = clb.Batch(probs)
    t0 = time.perf_counter()
    steps, er, status = b.run(tol, cap, DIAG_INTERVAL)
    wall = time.perf_counter() - t0
    _, _, _, nu = b.status()
    b.close()
    rng = np.random.default_rng(1)
    small = [k for k, p in enumerate(probs) if p.nx <= subset_max_edge]
    pick = sorted(int(k) for k in rng.choice(small, subset, replace=False))
    rows = []
    t1 = time.perf_counter()
    for k in pick:
        lat = clb.Lattice.from_problem(probs[k].with_storage(W.STORAGE_F64))
        s64, e64 = lat.run(plain_tol, cap, DIAG_INTERVAL)
        n64 = lat.nusselt(probs[k].nu_axis)
        lat.close()
        rows.append({"name": probs[k].name, "steps_plain": int(s64), "er_plain": float(e64),
                     "nu_plain": float(n64), "steps": int(steps[k]), "nu": float(nu[k]),
                     "rel": abs(float(nu[k]) - float(n64)) / abs(float(n64))})
    wall_plain = time.perf_counter() - t1
    nodes = sum(p.nodes for p in probs)
    return {"instances": count, "nodes": nodes, "storage": "f32", "tol": tol, "cap": cap,
            "wall_s": wall, "solves_per_s": count / wall,
            "converged": int((er < tol).sum()), "at_cap": int((steps >= cap).sum()),
            "status_nonzero": int((status != 0).sum()),
            "steps_p50": float(np.median(steps)), "steps_max": int(steps.max()),
            "node_updates": float(sum(p.nodes * int(s) for p, s in zip(probs, steps))),
            "plain_f64_subset": {"instances": subset, "edges_max": subset_max_edge, "tol": plain_tol,
                                 "wall_s": wall_plain, "solves_per_s": subset / wall_plain,
                                 "converged": int(sum(r["er_plain"] < plain_tol for r in rows)),
                                 "nusselt_rel_max": max(r["rel"] for r in rows), "rows": rows},
            "speedup_solves_per_s": (count / wall) / (subset / wall_plain)}


def rb_long_run(steps: int = 200000, window: int = 50000, interval: int = DIAG_INTERVAL):
    """Rayleigh-Benard 2048 x 1024 at Ra = 1e7 stepped `steps` steps in each storage form (FP16
    deviation storage, FP32 deviation storage, FP64), with the FP64 Nusselt number (Eq. 29) and
    residual taken every `interval` steps (clb_check). The flow is chaotic, so the forms are
    compared by statistics: the Nusselt number averaged over the last `window` steps (with the
    standard error of that mean from 5 blocks of the window) and the residual's median and maximum
    there, each form against FP64. Wall time and throughput include the checks."""
    from paper_1710_10569_gb300 import clb
    out = {"workload": "rayleigh_benard_2048x1024_Ra1e7_Pr0.71", "steps": steps, "window": window,
           "check_interval": interval, "forms": {}}
    for st in (W.STORAGE_F64, W.STORAGE_F32, W.STORAGE_F16DEV):
        prob = workload(st)
        lat = clb.Lattice.from_problem(prob)
        nus, ers = [], []
        t0 = time.perf_counter()
        for _ in range(steps // interval):
            lat.step(interval)
            nu, er = lat.check(1)
            nus.append(nu)
            ers.append(er)
        wall = time.perf_counter() - t0
        lat.close()
        nus, ers = np.array(nus), np.array(ers)
        tail = window // interval
        blocks = np.array([b.mean() for b in np.array_split(nus[-tail:], 5)])
        onset = next((int((k + 1) * interval) for k, v in enumerate(nus) if v > 1.5), None)
        out["forms"][W.STORAGE_NAMES[st]] = {
            "mlups": prob.nodes * steps / wall / 1e6, "wall_s": wall,
            "nu_mean": float(nus[-tail:].mean()), "nu_std": float(nus[-tail:].std()),
            "nu_mean_stderr": float(blocks.std(ddof=1) / math.sqrt(len(blocks))),
            "nu_final": float(nus[-1]), "residual_median": float(np.median(ers[-tail:])),
            "residual_max": float(ers[-tail:].max()), "steps_to_nu_1.5": onset,
            "nu_every_5000_steps": [round(float(v), 4) for v in nus[5000 // interval - 1::5000 // interval]]}
    ref = out["forms"]["f64"]
    for name, f in out["forms"].items():
        if name != "f64":
            f["nu_mean_rel_vs_f64"] = abs(f["nu_mean"] - ref["nu_mean"]) / ref["nu_mean"]
            f["nu_mean_diff_in_stderr"] = abs(f["nu_mean"] - ref["nu_mean"]) / math.hypot(
                f["nu_mean_stderr"], ref["nu_mean_stderr"])
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1710_10569_gb300 import clb
    storage = {"f64": W.STORAGE_F64, "f32": W.STORAGE_F32, "f16dev": W.STORAGE_F16DEV}[args.storage]

    # CPU baseline first (before the GPU is busy), rank 0 at N = 1 only
    cpu = cpu_baseline(storage, args.nx, args.ny) if (rank == 0 and world == 1 and not args.no_cpu) else None

    prob = workload(storage, args.nx, args.ny)
    lat = clb.Lattice.from_problem(prob)
    if args.autotune:
        lat.autotune()
    with ClockSampler(local) as clocks:
        secs = time_run(lat, args.steps, args.warmup, world)
        # the dominant kernel alone, for the roofline: its average launch duration over a fixed
        # window of graph-replayed launches, whatever --steps is
        k_steps = KERNEL_WINDOW
        secs_kernel = time_steps(lat, k_steps, 3, world)
    nodes = prob.nodes
    units, tmax = aggregate(float(nodes) * args.steps, secs, world)
    mlups = units / tmax / 1e6
    peak, peak_kind = measured_peaks()
    per_launch_s = secs_kernel / k_steps
    alg_bytes = BYTES_PER_NODE[storage] * nodes
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = traffic_per_launch(storage, prob.nx, prob.ny)

    variants = {}
    if rank == 0 and not args.no_variants:
        for st in (W.STORAGE_F64, W.STORAGE_F16DEV, W.STORAGE_F32):
            if st == storage:
                continue
            vx, vy = VARIANT_SIZE[st]
            p2 = workload(st, vx, vy)
            l2 = clb.Lattice.from_problem(p2)
            if args.autotune:
                l2.autotune()
            k = max(200, args.steps // (8 if st == W.STORAGE_F64 else 2))
            s2 = time_steps(l2, k, max(3, args.warmup // 4), 1)
            variants[W.STORAGE_NAMES[st]] = {
                "workload": f"rayleigh_benard_{p2.nx}x{p2.ny}_Ra1e7_Pr0.71",
                "mlups": p2.nodes * k / s2 / 1e6,
                "achieved_gbs": BYTES_PER_NODE[st] * p2.nodes / (s2 / k) / 1e9,
                "hbm_frac": BYTES_PER_NODE[st] * p2.nodes / (s2 / k) / 1e9 / peak,
                "steps": k, "dram_bytes_per_launch": traffic_per_launch(st, p2.nx, p2.ny),
                "working_set_mb": BYTES_PER_NODE[st] * p2.nodes / 1e6,
                "launch": list(l2.launch())}
            ops = profile_counts().get("fp64_ops_per_node")
            if st == W.STORAGE_F64 and ops:
                dp = sum(ops.values())
                rate = dp * p2.nodes * k / s2
                variants["f64"]["roofline"] = {
                    "bound": "alu", "achieved": rate / 1e12, "peak": FP64_DP_INSTR_PEAK / 1e12,
                    "unit": "T DP instructions/s", "frac": rate / FP64_DP_INSTR_PEAK,
                    "dp_instructions_per_node": dp,
                    "peak_kind": "derived: 152 SMs x 2 FP64 lanes/clock x 2.07 GHz"}
            l2.close()
    e2e = e2e_run(storage, args.steps, args.nx, args.ny) if rank == 0 else None
    thermal = thermal_run(storage, max(200, args.steps // 8)) if (rank == 0 and not args.no_variants) else None
    three_d = three_d_run(max(200, args.steps // 20)) if (rank == 0 and not args.no_variants) else None
    rb_long = rb_long_run() if (rank == 0 and not args.no_long) else None
    batched = batched_run(storage) if (rank == 0 and not args.no_serve) else None
    if batched is not None and not args.no_long:
        batched["to_steady_state"] = batched_steady_run()
    served = served_run(storage) if (rank == 0 and not args.no_serve) else None
    if rank == 0:
        line = {
            "metric": "coupled D2Q9+D2Q5 MLUPS & % HBM roofline", "value": mlups, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[storage], "data": "synthetic",
            "config": {"workload": f"rayleigh_benard_{prob.nx}x{prob.ny}_Ra1e7_Pr0.71",
                       "nodes": nodes, "storage": W.STORAGE_NAMES[storage],
                       "step": "fused collide-and-stream every step; FP64 Nusselt number and residual "
                               f"reduced and read back every {DIAG_INTERVAL} steps and after the last "
                               f"step (clb_run): {diag_checks(args.steps)} check(s) inside the timed "
                               f"{args.steps} steps",
                       "diag_checks_timed": diag_checks(args.steps),
                       "launch": list(lat.launch()),
                       "l2": "no flush: each step reads one population buffer and writes the "
                             f"other ({alg_bytes / 2 / 1e6:.0f} MB each, {alg_bytes / 1e6:.0f} MB "
                             "per step against the 129 MB L2); roofline.traffic is the ncu DRAM "
                             "bytes per launch",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel_launches_timed": k_steps,
                         "kernel_us_per_launch": per_launch_s * 1e6,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel": step_kernel_name(storage),
                         "flops_per_node": flops_per_node(),
                         "peak_kind": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            # every step's fused kernel (the FP16 form: the interior and edge kernels), plus the
            # two reduction kernels of each check
            "gpu_launches": args.steps * kernels_per_step(storage) + 2 * diag_checks(args.steps),
            "clocks": clocks.summary(),
            "variants": variants,
            "thermal_only": thermal,
            "three_d": three_d,
            "batched": batched,
            "served": served,
            "rb_long": rb_long,
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The oracle (plain FP64 C, OpenMP over nodes) on the host cores, each step a bounded sample
    of the workload: one time step of a 256 x 128 Rayleigh-Benard lattice with the bench
    parameters."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    storage = W.STORAGE_F32
    full = workload(storage)
    prob = W.rayleigh_benard(256, 128, Ra=1e7, Pr=0.71, u_c=0.1, perturb=1e-3, seed=0, storage=storage)
    prob.params.update({k: full.params[k] for k in ("nu", "kappa", "g_beta")})
    o = oracle.Oracle.from_problem(prob)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = prob.nodes * args.steps / dt / 1e6
    sample = (f"each step: one time step of a {prob.nx}x{prob.ny} lattice with the "
              f"{full.nx}x{full.ny} workload's parameters")
    line = {"impl": "reference", "metric": "coupled D2Q9+D2Q5 MLUPS & % HBM roofline", "value": v,
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rayleigh_benard_{full.nx}x{full.ny}_Ra1e7_Pr0.71",
                       "sample": sample},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "f16dev"])
    ap.add_argument("--nx", type=int, default=2048, help="lattice width of the timed workload")
    ap.add_argument("--ny", type=int, default=1024, help="lattice height of the timed workload")
    ap.add_argument("--autotune", action="store_true", help="time the autotuned launch shape instead of the default")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the batched and served runs")
    ap.add_argument("--no-long", action="store_true",
                    help="skip the 200,000-step Rayleigh-Benard run in three storage forms")
    ap.add_argument("--rb-long", action="store_true",
                    help="run only the 200,000-step Rayleigh-Benard run in three storage forms "
                         "(--steps sets its length) and print its JSON")
    ap.add_argument("--thermal-only", action="store_true",
                    help="run only the D2Q5 thermal-only step (4096 x 4096) and print its JSON")
    ap.add_argument("--three-d-only", action="store_true",
                    help="run only the 3-D workload (D3Q27 + D3Q7, 256 x 256 x 128) and print its JSON")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched workload (256 uneven cavities) and print its JSON")
    ap.add_argument("--steady-only", action="store_true",
                    help="run only the steady-state runs (256 batched cavities with retirement; the "
                         "served trace) and print their JSON")
    ap.add_argument("--served-large", action="store_true",
                    help="run only a served trace over the full edge range (32 requests, edges "
                         "64-4096, cap 4,000 steps, tol 1e-8) against plain FP64, and print its JSON")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.thermal_only:
        st = {"f64": W.STORAGE_F64, "f32": W.STORAGE_F32, "f16dev": W.STORAGE_F16DEV}[args.storage]
        print(json.dumps(thermal_run(st, args.steps)), flush=True)
    elif args.rb_long:
        print(json.dumps(rb_long_run(args.steps, min(50000, args.steps // 4 // DIAG_INTERVAL * DIAG_INTERVAL))),
              flush=True)
    elif args.three_d_only:
        print(json.dumps(three_d_run(args.steps)), flush=True)
    elif args.served_large:
        st = {"f64": W.STORAGE_F64, "f32": W.STORAGE_F32, "f16dev": W.STORAGE_F16DEV}[args.storage]
        print(json.dumps(served_run(st, count=32, step_cap=4000, tol=1e-8, plain_tol=1e-8, lo=64, hi=4096,
                                    rb_Ra=(1e3, 1e6), hbm_budget_gb=96)), flush=True)
    elif args.steady_only:
        st = {"f64": W.STORAGE_F64, "f32": W.STORAGE_F32, "f16dev": W.STORAGE_F16DEV}[args.storage]
        print(json.dumps({"batched_to_steady_state": batched_steady_run(), "served": served_run(st)}), flush=True)
    elif args.batched_only:
        print(json.dumps(batched_run({"f64": W.STORAGE_F64, "f32": W.STORAGE_F32,
                                      "f16dev": W.STORAGE_F16DEV}[args.storage], steps=args.steps)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
