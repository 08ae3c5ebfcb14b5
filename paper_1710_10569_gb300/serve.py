"""Request loops over the library: continuous batching (clb_serve_*) and the plain one-at-a-time
FP64 path it is compared with.

A trace is a list of (arrival_seconds, Problem). `serve_trace` replays it in real time: each request
is submitted when its arrival time has passed, admitted by the library as soon as a slot and enough
of the HBM budget are free, stepped together with the other resident requests (one batched launch
per time step), and retired when its residual drops below `tol` or its step cap is reached.
`plain_trace` runs the same requests one after another through a single-lattice handle in FP64.
Both report per-request latency (completion - arrival), steps, Nusselt number, and the summary
solves/s, p50 and p99 latency.
"""
from __future__ import annotations

import time

import numpy as np

from . import clb
from . import workloads as W


def _summary(records, wall, tol):
    lat = np.array([r["latency_s"] for r in records])
    return {"requests": len(records), "wall_s": wall, "solves_per_s": len(records) / wall,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_steps": float(np.mean([r["steps"] for r in records])), "tol": tol,
            "converged": int(sum(r["residual"] < tol for r in records))}


def serve_trace(trace, storage: int, hbm_budget_bytes: int, max_slots: int = 256, chunk: int = 100,
                step_cap: int = 20000, tol: float = 1e-6, stream=None, keep_fields: bool = False):
    """Replay `trace` through a clb_serve server. Returns (summary, records)."""
    srv = clb.Server(hbm_budget_bytes, max_slots, storage, stream=stream)
    pending = sorted(trace, key=lambda a: a[0])
    live = {}
    records = []
    t0 = time.perf_counter()
    i = 0
    while i < len(pending) or live:
        now = time.perf_counter() - t0
        while i < len(pending) and pending[i][0] <= now:
            arrival, prob = pending[i]
            prob = prob.with_storage(storage)
            rid = srv.submit(prob, step_cap=step_cap, tol=tol)
            live[rid] = (arrival, prob)
            i += 1
        if not live:
            time.sleep(max(0.0, pending[i][0] - (time.perf_counter() - t0)))
            continue
        srv.progress(chunk)
        done_now = time.perf_counter() - t0
        for rid in list(live):
            done, nu, steps, er = srv.poll(rid)
            if done:
                arrival, prob = live.pop(rid)
                rec = {"name": prob.name, "arrival_s": arrival, "latency_s": done_now - arrival,
                       "steps": steps, "nu": nu, "residual": er, "nodes": prob.nodes}
                fields = srv.fetch(rid, prob.ny, prob.nx)
                if keep_fields:
                    rec["fields"] = fields
                records.append(rec)
    wall = time.perf_counter() - t0
    srv.close()
    return _summary(records, wall, tol), records


def plain_trace(trace, step_cap: int = 20000, tol: float = 1e-6, interval: int = 100, stream=None):
    """The same requests in arrival order, one at a time, FP64 storage, single-lattice handles."""
    pending = sorted(trace, key=lambda a: a[0])
    records = []
    t0 = time.perf_counter()
    for arrival, prob in pending:
        wait = arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        p64 = prob.with_storage(W.STORAGE_F64)
        lat = clb.Lattice.from_problem(p64, stream=stream)
        steps, er = lat.run(tol, step_cap, interval)
        nu = lat.nusselt(prob.nu_axis)
        lat.close()
        records.append({"name": prob.name, "arrival_s": arrival,
                        "latency_s": time.perf_counter() - t0 - arrival, "steps": steps, "nu": nu,
                        "residual": er, "nodes": prob.nodes})
    wall = time.perf_counter() - t0
    return _summary(records, wall, tol), records


def nusselt_agreement(served, plain, tol: float, plain_tol: float | None = None):
    """Relative differences of the served Nusselt numbers from the plain FP64 ones, per request:
    overall and over the requests that reached their residual tolerance in both paths (steady
    states; `plain_tol` is the plain path's, `tol` by default), with the worst requests listed."""
    plain_tol = tol if plain_tol is None else plain_tol
    by = {r["name"]: r for r in plain}
    rows = []
    for r in served:
        q = by.get(r["name"])
        if q is None:
            continue
        rel = abs(r["nu"] - q["nu"]) / max(abs(q["nu"]), 1e-300)
        rows.append({"name": r["name"], "rel": rel, "steps": r["steps"], "steps_plain": q["steps"],
                     "nu": r["nu"], "nu_plain": q["nu"],
                     "converged": r["residual"] < tol and q["residual"] < plain_tol})
    rels = np.array([x["rel"] for x in rows])
    conv = np.array([x["rel"] for x in rows if x["converged"]])
    return {"requests": len(rows), "max": float(rels.max()) if rels.size else None,
            "median": float(np.median(rels)) if rels.size else None,
            "fraction_within_1e-3": float(np.mean(rels <= 1e-3)) if rels.size else None,
            "converged_requests": int(conv.size),
            "max_over_converged": float(conv.max()) if conv.size else None,
            "worst": sorted(rows, key=lambda x: -x["rel"])[:3]}
