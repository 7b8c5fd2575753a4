"""Trace replay for the serving loop (pe_server_*): arrivals in real time, continuous batching on
the GPU, per-request latency (arrival -> result on the host) and throughput.

The work itself runs in the CUDA library through ``sssp.Server``; this module only turns trace
entries (``inputs.serving_trace``) into requests and keeps the clock.
"""
from __future__ import annotations

import math
import time
from typing import Dict, List

import numpy as np

from . import inputs
from . import sssp


def build_solve(req: Dict, range_scale: float = 1.0, node_spacing: float = 5000.0) -> inputs.Solve:
    """The march of one trace entry: isovelocity (V ignored), Munk, or Munk + Gaussian eddy with
    a profile node every ``node_spacing`` metres (evaluated at the node's centre)."""
    steps = max(1, int(math.ceil(req["range_m"] * range_scale / req["dr"])))
    if req["env"] == "isovelocity":
        s = inputs.isovelocity(N=req["N"], H=req["H"], freq=req["freq"], dr=req["dr"], steps=steps,
                               pade_order=req["pade_order"], zs=req["zs"])
        return s
    s = inputs.munk(N=req["N"], H=req["H"], freq=req["freq"], dr=req["dr"], steps=steps,
                    pade_order=req["pade_order"], zs=req["zs"])
    if req["env"] == "munk_eddy":
        z = s.z
        cm = inputs.munk_c(z)
        rng_total = steps * req["dr"]
        nodes = []
        r = 0.0
        while r < rng_total or not nodes:
            rc = r + 0.5 * node_spacing
            nodes.append((r, inputs.n2_from_c(cm + inputs.gaussian_eddy_dc(rc, z, req["eddy_dc"], r0=req["eddy_r0"]),
                                              s.c0)))
            r += node_spacing
        s.profiles = nodes
    return s


def _depth_summary(depth, points: int = 24) -> Dict:
    """Admitted concurrency and queue depth over time: maxima, time averages and an evenly
    decimated trace of (seconds, live, queued)."""
    if not depth:
        return {"max_live": 0, "max_queued": 0, "mean_live": 0.0, "mean_queued": 0.0, "trace": []}
    t = np.array([d[0] for d in depth])
    live = np.array([d[1] for d in depth], dtype=np.float64)
    q = np.array([d[2] for d in depth], dtype=np.float64)
    w = np.diff(np.concatenate([[0.0], t]))  # time each sample stood for
    idx = np.unique(np.linspace(0, len(depth) - 1, min(points, len(depth))).astype(int))
    return {"max_live": int(live.max()), "max_queued": int(q.max()),
            "mean_live": float((live * w).sum() / max(w.sum(), 1e-12)),
            "mean_queued": float((q * w).sum() / max(w.sum(), 1e-12)),
            "trace": [[round(float(t[i]), 3), int(live[i]), int(q[i])] for i in idx]}


def replay(trace: List[Dict], hbm_budget: float, chunk_steps: int = 50, tl_every: int = 10,
           range_scale: float = 1.0, max_live: int = 1024, stream=None, keep_results: bool = False,
           admit: int = sssp.ADMIT_MINIMAX_C0 | sssp.ADMIT_CONVERGENT_ORDER, keep_ids=None,
           record_params: bool = False, pacing: int = 64):
    """Replay ``trace`` against a fresh server; returns latency / throughput figures.  ``admit``
    are the server's admission adaptations (default: minimax reference sound speed and a Pade
    order at which the Neumann series converges); ``keep_results`` also returns, per request,
    (field, TL rows, solve, (k0, n2 scale, Pade order) it was marched with); ``keep_ids`` keeps
    those only for the given trace ids; ``record_params`` returns every completed request's
    (k0, n2 scale, Pade order) under "params"; ``pacing``: the server's pacing limit (a cheaper
    request marches up to that many chunks per step; 1 = lockstep)."""
    keep = None if keep_ids is None else set(keep_ids)
    keep_results = keep_results or keep is not None
    srv = sssp.Server(int(hbm_budget), max_live=max_live, chunk_steps=chunk_steps, stream=stream)
    srv.set_pacing(pacing)
    order = sorted(range(len(trace)), key=lambda i: trace[i]["t_arrival"])
    pending = list(order)
    running = {}     # id -> (trace index, arrival wall time)
    lat = {}
    units = 0
    results = {}
    failed = {}
    adapted = {}
    params = {}
    t0 = time.perf_counter()
    nsteps = 0
    depth = []  # (seconds since start, live solves, queued requests) after every server step
    while pending or running:
        now = time.perf_counter() - t0
        while pending and trace[pending[0]]["t_arrival"] <= now:
            i = pending.pop(0)
            s = build_solve(trace[i], range_scale)
            rid = srv.submit(s, tl_every=tl_every, admit=admit)
            running[rid] = (i, t0 + trace[i]["t_arrival"], s.N * s.steps, s)
        if not running:
            time.sleep(max(0.0, trace[pending[0]]["t_arrival"] - (time.perf_counter() - t0)))
            continue
        live, queued, _ = srv.step()
        nsteps += 1
        tnow = time.perf_counter()
        depth.append((tnow - t0, live, queued))
        for rid in list(running):
            state = srv.state(rid)
            if state == 3:  # the march failed on the device (e.g. a diverging Neumann series)
                i, ta, u, s = running.pop(rid)
                failed[i] = "failed"
                try:
                    srv.take(rid)
                except sssp.PEError as e:
                    failed[i] = str(e)
                continue
            if state == 2:
                i, ta, u, s = running.pop(rid)
                lat[i] = tnow - ta
                units += u
                prm = srv.params(rid)
                if prm[2] != s.pade_order or prm[1] != 1.0:
                    adapted[i] = prm
                if record_params:
                    params[i] = prm
                f, tl = srv.take(rid)
                if keep_results and (keep is None or trace[i]["id"] in keep):
                    results[i] = (f, tl, s, prm)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    L = np.array([lat[i] for i in sorted(lat)])
    pct = (lambda q: float(np.percentile(L, q))) if L.size else (lambda q: None)
    out = {"requests": len(trace), "completed": len(lat), "failed": len(failed),
           "failed_ids": sorted(failed), "failures": {str(k): v for k, v in sorted(failed.items())},
           "order_lowered": sum(1 for i, p in adapted.items() if p[2] != trace[i]["pade_order"]),
           "wall_s": wall, "server_steps": nsteps,
           "throughput": units / wall, "p50_s": pct(50), "p99_s": pct(99),
           "mean_s": float(L.mean()) if L.size else None, "peak_live": st["peak_live"], "peak_bytes": st["peak_bytes"],
           "queue_depth": _depth_summary(depth)}
    if keep_results:
        out["results"] = results
    if record_params:
        out["params"] = params
    return out
