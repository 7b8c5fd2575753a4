"""Benchmark of the GB300 SSSP marcher.

Default workload (the headline): the batched precision sweep's FFT form, 256 range-independent
Munk solves (H = 5000 m, source at 1000 m, N = 1023 interior DST-I points each, f ~ U[50, 500] Hz
from default_rng(4), dr = 25 m, 2000 range steps, [6/6] Pade, Neumann series to 1e-10 or 12
terms, TL every 10 steps), all marched together by one batched launch (one CTA per solve).  One
bench step = set the 256 starters + one 2000-range-step batched march (TL rows land in HBM).

Besides the device-timed value the JSON line carries: the roofline of the march kernel, the
end-to-end figure through the public API with host buffers, the same solves marched one at a
time on the plain marcher (``vs_plain``), the serving mix (``served``: Poisson trace of 1000
requests under a 120 GB budget, p50/p99 latency and throughput), parity of each against stored
FP64 oracle runs or the plain path, and the FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload (the
reference arm of this comparison).  Under torchrun (N > 1) every rank marches its own copy of
the batch (independent replicas, weak scaling, no collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "depth-pt·range-steps/s at ≤0.1 dB TL error vs plain path; served p50/p99 latency"
UNIT = "depth-pt·range-steps/s"
WORKLOAD_MUNK = "munk_n4095_f50_dr50_s2000_p6_neumann12"
WORKLOAD = "munk_batch256_n1023_f50-500_dr25_s2000_p6_neumann12"
BATCH_TL_EVERY = 10


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of the GB300s, else the stated fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def _config(extra=None):
    c = {"workload": WORKLOAD_MUNK, "N": 4095, "H_m": 5000.0, "freq_hz": 50.0, "dr_m": 50.0, "range_steps": 2000,
         "pade_order": 6, "neumann_terms": 12, "neumann_tol": 1e-10, "tl_every": 1, "solves_per_gpu": 1,
         "l2": "flushed between timed iterations (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            a = [x.strip() for x in ln.split(",")]
            if len(a) < 9:
                continue
            try:
                sm.append(float(a[1]))
                mx.append(float(a[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if a[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_over_ranks(local_ms: float, local_units: float, device=None):
    """Whole-job figures of a replica run: the slowest rank's time (max over ranks, after a
    barrier) and the units all ranks processed.  Works with any torch.distributed backend
    (NCCL on GPUs, gloo on CPU); without a process group it returns the local figures."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local_ms, local_units
    dist.barrier()
    t = torch.tensor([local_ms, local_units], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0].item()), float(sm[1].item())


def _dst_flops(N):
    L = N + 1
    return 5.0 * L * math.log2(L)


def run_cpu_oracle_sample(seconds=15.0, workload="batch"):
    """Time the FP64 oracle (as it stands: Algorithm 1's sum form, explicit O(N^2) sine sums
    through BLAS) on the host cores, on a bounded sample of the workload, as depth-pt*steps per
    second.  Batch: the first range steps of successive members of the 256-solve batch; Munk:
    the first range steps of the N = 4095 march."""
    from oracle import sssp_oracle as O
    from paper_2511_03343_gb300 import inputs
    solves = inputs.munk_batch(steps=2000) if workload == "batch" else [inputs.munk()]
    units, el, done = 0, 0.0, []
    per = 20 if workload == "batch" else None
    for s in solves:
        g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr)
        plan = O.pade_plan(g.sigma, s.pade_order)
        O.march(s.u0, s.profiles, g, s.pade_order, 1, s.neumann_terms, s.neumann_tol, tl_every=1, plan=plan)
        if per is None:  # one solve: as many steps as fit in the time
            t0 = time.perf_counter()
            O.march(s.u0, s.profiles, g, s.pade_order, 1, s.neumann_terms, s.neumann_tol, tl_every=1, plan=plan)
            one = time.perf_counter() - t0
            n = max(1, min(s.steps, int(seconds / max(one, 1e-6))))
        else:
            n = per
        t0 = time.perf_counter()
        O.march(s.u0, s.profiles, g, s.pade_order, n, s.neumann_terms, s.neumann_tol, tl_every=1, plan=plan)
        el += time.perf_counter() - t0
        units += s.N * n
        done.append(n)
        if el >= seconds:
            break
    what = (f"first {per} range steps of each of the first {len(done)} of the 256 batch members (N=1023)"
            if workload == "batch" else f"first {done[0]} of 2000 range steps of the N=4095 Munk march")
    return {"value": units / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{what} (FP64 oracle, sum form, direct O(N^2) DST-I via BLAS), {el:.1f} s"}


def bench_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores; each bench step is a
    bounded sample of the workload (``--ref-sample-steps`` range steps of one solve: for the
    batch, members in turn)."""
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    from oracle import sssp_oracle as O
    from paper_2511_03343_gb300 import inputs
    batch = args.workload == "batch"
    solves = inputs.munk_batch(steps=2000) if batch else [inputs.munk()]
    sample_steps = args.ref_sample_steps
    times, units = [], 0
    for i in range(args.warmup + args.steps):
        s = solves[i % len(solves)]
        g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr)
        plan = O.pade_plan(g.sigma, s.pade_order)
        t0 = time.perf_counter()
        O.march(s.u0, s.profiles, g, s.pade_order, sample_steps, s.neumann_terms, s.neumann_tol, tl_every=1, plan=plan)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
            units += s.N * sample_steps
    tot = sum(times)
    value = units / tot
    what = (f"each step: {sample_steps} of the 2000 range steps of one batch member (N=1023; members in turn)"
            if batch else f"each step: {sample_steps} of the 2000 range steps of the N=4095 Munk march")
    cfg = _batch_config() if batch else _config()
    cfg["reference_sample_range_steps"] = sample_steps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": what + " (FP64 oracle, sum form, direct O(N^2) DST-I)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _batch_config(extra=None):
    c = {"workload": WORKLOAD, "solves": 256, "N": 1023, "H_m": 5000.0, "freq_hz": "U[50, 500] default_rng(4)",
         "dr_m": 25.0, "range_steps": 2000, "pade_order": 6, "neumann_terms": 12, "neumann_tol": 1e-10,
         "zs_m": 1000.0, "c0_mps": 1500.0, "tl_every": BATCH_TL_EVERY, "solves_per_gpu": 256,
         "l2": "flushed between timed iterations (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


def _load_make_golden():
    import importlib.util
    here = os.path.join(ROOT, "tests", "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def _batch_parity(fields, tls, tl_every):
    """Field / TL error of the bench's own output for the batch members stored from the FP64
    oracle's product form (tests/golden/batch_n1023_s2000.txt): worst member and per member."""
    import numpy as np
    mg = _load_make_golden()
    path = os.path.join(ROOT, "tests", "golden", "batch_n1023_s2000.txt")
    if not os.path.exists(path):
        return None
    runs = mg.load_batch(path)
    per = {}
    step = mg.BATCH_TL_EVERY // tl_every
    for i, (freq, fidx, fref, tl_r, tl_ref) in runs.items():
        if i not in fields:
            continue
        u, tl = fields[i], tls[i]
        rows = tl[step - 1::step][:, ::mg.BATCH_TL_STRIDE].astype(np.float64)
        mask = tl_ref < 100
        per[str(i)] = {"freq_hz": round(freq, 3),
                       "field_rel_l2_sampled": float(np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)),
                       "max_tl_err_db": float(np.max(np.abs(rows - tl_ref)[mask]))}
    if not per:
        return None
    return {"against": "stored FP64 oracle runs, product form (tests/golden/batch_n1023_s2000.txt)",
            "members": per,
            "worst_field_rel_l2": max(v["field_rel_l2_sampled"] for v in per.values()),
            "worst_tl_err_db": max(v["max_tl_err_db"] for v in per.values())}


def _tl_vs(tl_a, tl_b):
    import numpy as np
    a = tl_a.astype(np.float64)
    b = tl_b.astype(np.float64)
    mask = b < 100
    return float(np.max(np.abs(a - b)[mask])) if mask.any() else 0.0


def bench_batch(args):
    """The headline line: the 256-solve Munk batch (see the module docstring)."""
    import numpy as np
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from paper_2511_03343_gb300 import inputs, sssp
    steps = args.range_steps
    solves = inputs.munk_batch(steps=steps)
    stream = torch.cuda.current_stream()
    plans = [sssp.plan_for(s, stream=stream, tl_every=BATCH_TL_EVERY) for s in solves]
    for pl in plans:
        pl.set_kernel(args.kernel)
    # the batch shape (points per thread of the one-CTA kernel) chosen by the library's autotuner
    tune = None if args.no_autotune else sssp.autotune_batch(plans, steps=8)
    u0s = [torch.from_numpy(s.u0.astype(np.complex64)).cuda() for s in solves]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step(ev=None):
        for pl, u0 in zip(plans, u0s):
            pl.set_field(u0, 0.0)
        if ev is not None:
            ev[0].record(stream)
        sssp.march_batch(plans, steps)
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    nd0 = sum(pl.transform_count() for pl in plans)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[2].record(stream)
        one_step(e)
        e[3].record(stream)
        torch.cuda.synchronize()
        step_ms.append(e[2].elapsed_time(e[3]))
        kern_ms.append(e[0].elapsed_time(e[1]))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    nd1 = sum(pl.transform_count() for pl in plans)
    units_local = float(sum(s.N for s in solves) * steps * args.steps)
    tot_ms, units = aggregate_over_ranks(sum(step_ms), units_local, device="cuda")
    value = units / (tot_ms * 1e-3)
    mg = _load_make_golden()
    members = sorted(mg.load_batch().keys()) if steps == 2000 else []
    fields = {i: plans[i].read_field() for i in members}
    tls = {i: plans[i].read_tl()[0] for i in members}
    parity = _batch_parity(fields, tls, BATCH_TL_EVERY) if members else None

    # end to end through the public API with host (pinned) buffers: starters H2D, march, TL rows
    # and fields D2H, every step
    rows = steps // BATCH_TL_EVERY
    u0_host = [torch.from_numpy(s.u0.astype(np.complex64)).pin_memory() for s in solves]
    tl_host = torch.empty(len(solves) * rows * solves[0].N, dtype=torch.float32).pin_memory()
    field_host = torch.empty(len(solves) * solves[0].N, dtype=torch.complex64).pin_memory()
    tl_views = [tl_host[i * rows * s.N:(i + 1) * rows * s.N] for i, s in enumerate(solves)]
    f_views = [field_host[i * s.N:(i + 1) * s.N] for i, s in enumerate(solves)]
    e2e_ms = []
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for pl, u0 in zip(plans, u0_host):
            pl.set_field(u0, 0.0)
        sssp.march_batch(plans, steps)
        for pl, tv, fv in zip(plans, tl_views, f_views):
            pl.read_tl(out=tv)
            pl.read_field(out=fv)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_ms.append(el * 1e3)
    e2e_tot = sum(e2e_ms) if e2e_ms else float("nan")
    e2e_tot, _ = aggregate_over_ranks(e2e_tot, 0.0, device="cuda")

    # roofline of the dominant kernel (the batched march kernel, FP32 ALU bound)
    kern_avg = sum(kern_ms) / len(kern_ms)
    dst_per_launch = (nd1 - nd0) / args.steps
    L = solves[0].N + 1
    flops = dst_per_launch * (_dst_flops(solves[0].N) + 10.0 * L)
    achieved = flops / (kern_avg * 1e-3) / 1e12
    sm_max = float(clk.get("sm_max_mhz") or 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * 128 * 2 * sm_max * 1e6 / 1e12

    line = None
    if rank == 0:
        plain = None if (args.no_plain or world > 1) else _vs_plain(args, sssp, inputs, solves, members, fields, tls,
                                                                     stream, flush, f"cta{plans[0].shape}")
        served = None if (args.no_served or world > 1) else _served_block(args, sssp, stream)
        cpu = run_cpu_oracle_sample(args.cpu_seconds, "batch") if (world == 1 and not args.no_cpu) else None
        bytes_in = sum(s.N for s in solves) * 8
        bytes_out = sum(s.N for s in solves) * (rows * 4 + 8)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": _batch_config({"kernel": plans[0].kernel, "points_per_thread": plans[0].shape,
                                         "range_steps": steps, "autotune": tune}),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None,
                             "kernel": f"{plans[0].kernel} march kernel, one launch of 256 solves",
                             "flops_per_launch": flops, "dst_per_launch": dst_per_launch, "kernel_ms": kern_avg,
                             "flop_convention": "per DST-I of length N: 5(N+1)log2(N+1) + 10(N+1)",
                             "peak_note": f"FP32 FMA peak of all {sms} SMs at the sampled max SM clock "
                                          "(128 lanes x 2 flop per SM per cycle; derived, not measured)"},
                "e2e": {"value": units / (e2e_tot * 1e-3) if e2e_ms else None, "unit": UNIT,
                        "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": bytes_out},
                "gpu_launches": (len(solves) + 1) * args.steps,
                "clocks": clk, "parity": parity, "vs_plain": plain, "served": served, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    for pl in plans:
        pl.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _vs_plain(args, sssp, inputs, solves, members, fields, tls, stream, flush, batch_shape):
    """The same solves marched one plan at a time on the plain marcher (pe_march, one solve on
    the GPU at a time, the kernel the library picks for one solve): the stored members (lowest,
    second lowest, then evenly up to the highest frequency), each timed alone with CUDA events;
    their results against the batched run (bitwise) and their throughput."""
    import numpy as np
    import torch
    out, tot_ms, units, same = {}, 0.0, 0, True
    worst_tl = 0.0
    for i in members:
        s = solves[i]
        pl = sssp.plan_for(s, stream=stream, tl_every=BATCH_TL_EVERY)
        tune = sssp.autotune_batch([pl], steps=8)  # the plain path at its own best shape
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pl.march(s.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        u = pl.read_field()
        tl, _ = pl.read_tl()
        kernel = pl.kernel if pl.kernel == "cluster" else f"cta{pl.shape}"
        pl.close()
        tot_ms += ms
        units += s.N * s.steps
        if kernel == batch_shape:
            same = same and np.array_equal(u, fields[i]) and np.array_equal(tl, tls[i])
        worst_tl = max(worst_tl, _tl_vs(tls[i], tl))
        out[str(i)] = {"freq_hz": round(s.freq, 3), "ms": ms, "shape": kernel, "autotune_ms": tune["ms"]}
    if not members:
        return None
    return {"value": units / (tot_ms * 1e-3), "unit": UNIT, "solves_timed": len(members),
            "what": "the stored batch members, each marched alone (pe_march) at the shape the autotuner picks "
                    "for one solve, CUDA events per solve",
            "batched_results_bitwise_equal_where_same_shape": bool(same), "max_tl_diff_db_batched_vs_plain": worst_tl,
            "members": out}


def _served_block(args, sssp, stream):
    """The serving mix: the Poisson trace (default_rng(5), 200 req/s, 1000 requests) replayed in
    real time through the continuous-batching server with a 120 GB budget, ranges scaled by
    ``--served-range-scale``; p50/p99 latency (arrival -> result on the host) and throughput.
    Parity: a few completed requests marched again alone on the plain marcher with the values
    admission chose (TL difference, bitwise equality)."""
    import numpy as np
    from paper_2511_03343_gb300 import inputs, serving
    trace = inputs.serving_trace(count=args.serve_requests)
    check = [t["id"] for t in trace if t["N"] <= 1023][:6]
    res = serving.replay(trace, hbm_budget=120e9, chunk_steps=args.chunk_steps, tl_every=10,
                         range_scale=args.served_range_scale, stream=stream, keep_ids=check, pacing=args.pacing)
    worst, same = 0.0, True
    for i, (field, tl, s, prm) in res.pop("results").items():
        k0, sc, p = prm
        pl = sssp.Plan(s.N, s.H, k0, s.dr, p, s.neumann_terms, s.neumann_tol, stream=stream)
        pl.set_output(10)
        if s.neumann_terms > 1:
            pl.set_profile_nodes([(r, sc * np.asarray(n2)) for r, n2 in s.profiles])
        pl.set_field(s.u0, s.r0)
        pl.march(s.steps)
        u = pl.read_field()
        tl2, _ = pl.read_tl()
        pl.close()
        same = same and np.array_equal(u, field) and np.array_equal(tl2, tl)
        if tl.size:
            worst = max(worst, _tl_vs(tl, tl2))
    res["parity_vs_plain"] = {"requests": len(check), "bitwise_equal": bool(same), "max_tl_diff_db": worst}
    res["config"] = {"requests": len(trace), "rate_per_s": 200, "range_scale": args.served_range_scale,
                     "budget_bytes": 120e9, "chunk_steps": args.chunk_steps, "tl_every": 10,
                     "pacing": args.pacing, "admission": "minimax c0 + convergent Pade order"}
    res.pop("queue_depth", None)
    return res


def _golden_check(tl, u):
    """TL / field error of the bench's own output against the stored FP64 oracle runs: the
    product form the GPU marches (identical rules) and Algorithm 1's sum form (the 12-term
    series is not converged to 1e-10 here, so the two forms themselves differ by ~8.5e-5)."""
    import importlib.util
    import numpy as np
    here = os.path.join(ROOT, "tests", "golden")
    p = os.path.join(here, "make_golden.py")
    files = {"product": "munk_n4095_s2000_product.txt", "sum": "munk_n4095_s2000.txt"}
    if not all(os.path.exists(os.path.join(here, f)) for f in files.values()):
        return None
    spec = importlib.util.spec_from_file_location("make_golden", p)
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    out = {}
    for form, name in files.items():
        meta, fidx, fref, tl_r, tl_ref = mg.load(os.path.join(here, name))
        every = int(meta["tl_every"])
        rows = tl[every - 1::every][:, ::int(meta["tl_stride"])].astype(np.float64)
        mask = tl_ref < 100
        out[form] = {"max_tl_err_db": float(np.max(np.abs(rows - tl_ref)[mask])),
                     "field_rel_l2_sampled": float(np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref)),
                     "against": "stored FP64 oracle run (tests/golden/%s)" % name}
    return out


def bench_other(args):
    """Secondary workloads (not the headline line): 'batch' = 256 Munk solves N = 1023,
    f ~ U[50, 500] Hz (default_rng(4)), dr = 25 m, 2000 steps, [6/6], Neumann 12 terms, marched
    together by pe_march_batch (one launch, one CTA per solve); 'eddy' = Munk + Gaussian eddy,
    N = 16383, 250 Hz, dr = 25 m, [8/8], a profile node per step; 'iso' = isovelocity N = 255."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from paper_2511_03343_gb300 import inputs, sssp
    stream = torch.cuda.current_stream()
    steps = args.range_steps
    if args.workload == "batch":
        solves = inputs.munk_batch(count=args.batch_count, steps=steps)
    elif args.workload == "eddy":
        solves = [inputs.munk_eddy(steps=steps)]
    elif args.workload == "large":
        # grids of 65536 points, a batch whose footprint is several times the L2: the HBM-bound case
        solves = inputs.munk_batch(count=args.large_count, N=65535, steps=steps, seed=6, fmin=100.0, fmax=1000.0)
    else:
        solves = [inputs.isovelocity(steps=steps)]
    plans = []
    for s in solves:
        pl = sssp.Plan(s.N, s.H, s.k0, s.dr, s.pade_order, s.neumann_terms, s.neumann_tol, stream=stream)
        pl.set_kernel(args.kernel)
        pl.set_output(1)
        if s.neumann_terms > 1:
            pl.set_profile_nodes(s.profiles)
        plans.append(pl)
    u0s = [torch.from_numpy(s.u0.astype(np.complex64)).cuda() for s in solves]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tune = None
    if args.tune:  # the library's shape autotuner over every shape these solves can take
        for pl, u0 in zip(plans, u0s):
            pl.set_field(u0, 0.0)
        tune = sssp.autotune_batch(plans, steps=4)

    def one():
        for pl, u0 in zip(plans, u0s):
            pl.set_field(u0, 0.0)
        if len(plans) == 1:
            plans[0].march(steps)
        else:
            sssp.march_batch(plans, steps)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    nd0 = sum(pl.transform_count() for pl in plans)
    clocks = ClockSampler(0)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    nd1 = sum(pl.transform_count() for pl in plans)
    units = sum(s.N * steps for s in solves) * args.steps
    tot = sum(ms)
    line = {"metric": METRIC, "value": units / (tot * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": args.workload, "solves": len(solves), "N": [s.N for s in solves][:1],
                       "kernel": plans[0].kernel, "cluster_shape": plans[0].cluster_shape,
                       "range_steps": steps, "autotune": tune},
            "dst_per_step": (nd1 - nd0) / args.steps, "clocks": clk}
    if args.workload == "large":
        # algorithmic bytes of a transform of length L = N + 1: two global passes of 16 B per point
        L = solves[0].N + 1
        gbs = 32.0 * L * (nd1 - nd0) / (tot * 1e-3) / 1e9
        peak = _hbm_peak()
        line["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                            "traffic": None, "bytes_per_transform": 32.0 * L,
                            "peak_note": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}
    print(json.dumps(line), flush=True)
    for pl in plans:
        pl.close()


def bench_serve(args):
    """Serving mix: Poisson arrivals (200 req/s, default_rng(5)) of solves with N in
    {255, 1023, 4095, 16383, 65535}, f in [25, 1000] Hz, environment in {isovelocity, Munk,
    Munk + eddy}, Pade order 4..8, under a 120 GB budget, continuous batching (pe_server_*).
    Ranges are scaled by --range-scale (10-200 km x scale).  Compared with the one-at-a-time
    plain marcher: the same requests marched alone, FIFO in arrival order."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from paper_2511_03343_gb300 import inputs, serving, sssp
    trace = inputs.serving_trace(count=args.serve_requests)
    stream = torch.cuda.current_stream()
    # warm the kernels of every size
    for N in (255, 1023, 4095, 16383, 65535):
        pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4, stream=stream)
        pl.set_field(np.ones(N, dtype=np.complex64))
        pl.march(1)
        pl.read_field()
        pl.close()
    clocks = ClockSampler(0)
    clocks.start()
    res = serving.replay(trace, hbm_budget=120e9, chunk_steps=args.chunk_steps, tl_every=10,
                         range_scale=args.range_scale, stream=stream, record_params=True, pacing=args.pacing)
    clk = clocks.stop()
    prm = res.pop("params")
    line = {"metric": METRIC, "value": res["throughput"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * res["wall_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": "serving_mix", "requests": len(trace), "rate_per_s": 200,
                       "range_scale": args.range_scale, "budget_bytes": 120e9, "chunk_steps": args.chunk_steps,
                       "pacing": args.pacing},
            "served": {k: v for k, v in res.items() if k != "results"}, "clocks": clk}
    if args.serve_baseline:
        # one-at-a-time: every request marched alone on the plain marcher with the values admission
        # gave it, FIFO in arrival order.  Marching each whole request alone would take hours at full
        # ranges, so its service time is extrapolated from `--baseline-steps` timed steps (after one
        # untimed step), linearly in the step count.
        import numpy as np
        svc, units = [], 0
        k = args.baseline_steps
        for i, t in enumerate(trace):
            s = serving.build_solve(t, args.range_scale)
            k0, sc, p = prm.get(i, (s.k0, 1.0, s.pade_order))
            pl = sssp.Plan(s.N, s.H, k0, s.dr, p, s.neumann_terms, s.neumann_tol, stream=stream)
            pl.set_output(10)
            if s.neumann_terms > 1:
                pl.set_profile_nodes([(r, sc * np.asarray(n2)) for r, n2 in s.profiles])
            pl.set_field(s.u0, s.r0)
            pl.march(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n = min(k, max(1, s.steps - 1))
            e0.record(stream)
            pl.march(n)
            e1.record(stream)
            torch.cuda.synchronize()
            svc.append(e0.elapsed_time(e1) * 1e-3 * s.steps / n)
            units += s.N * s.steps
            pl.close()
        free_at, lat = 0.0, []
        for t, sv in sorted(zip(trace, svc), key=lambda x: x[0]["t_arrival"]):
            start = max(free_at, t["t_arrival"])
            free_at = start + sv
            lat.append(free_at - t["t_arrival"])
        line["one_at_a_time"] = {"throughput": units / sum(svc), "busy_s": sum(svc),
                                 "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                                 "how": f"each request alone on the plain marcher (pe_march) with its admitted "
                                        f"values; service time extrapolated from {k} timed steps; FIFO queue"}
    print(json.dumps(line), flush=True)


def bench_gemm(args):
    """The 256-solve Munk batch (N = 1023, [6/6], 12 terms) with the DST-I as the library's own
    tensor-core GEMM (tcgen05.mma, TMA-fed, fused epilogues), per precision: throughput of the
    lockstep march (one captured graph per range step), the tensor work rate, and the sampled final
    field of the stored members against the FP64 oracle runs (the fixed-12-term rule the lockstep
    batch uses).  FP32 (CUDA cores, the reference) may run fewer steps (``--gemm-fp32-steps``)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from oracle import sssp_oracle as O
    from paper_2511_03343_gb300 import inputs, sssp
    stream = torch.cuda.current_stream()
    steps = args.range_steps
    solves = inputs.munk_batch(count=args.batch_count, steps=steps)
    mg = _load_make_golden()
    runs = (mg.load_batch(os.path.join(ROOT, "tests", "golden", "batch_n1023_s2000_fixed12.txt"))
            if (steps == 2000 and args.batch_count == 256) else {})
    L = solves[0].N + 1
    C = 2 * len(solves)
    out = {}
    for mode in ["bf16x3", "3xtf32", "tf32", "fp32"]:
        n_steps = steps if mode != "fp32" else min(steps, args.gemm_fp32_steps)
        plans = [sssp.plan_for(s, stream=stream) for s in solves]
        gb = sssp.GemmBatch(plans, mode)
        gb.march(2)
        torch.cuda.synchronize()
        gb.close()
        gb = sssp.GemmBatch(plans, mode)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gb.march(n_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        gemms = solves[0].pade_order * (2 * solves[0].neumann_terms - 2) * n_steps
        products = 3 if mode in ("bf16x3", "3xtf32") else 1
        tflops = 2.0 * L * L * C * products * gemms / (ms * 1e-3) / 1e12
        rec = {"ms": ms, "range_steps": n_steps, "throughput": sum(s.N for s in solves) * n_steps / (ms * 1e-3),
               "gemms": gemms, "us_per_gemm": 1e3 * ms / gemms, "tensor_tflops": tflops if mode != "fp32" else None,
               "fp32_tflops": tflops if mode == "fp32" else None}
        if runs and n_steps == 2000:
            worst = (0.0, 0.0)
            for i, (freq, fidx, fref, tl_r, tl_ref) in runs.items():
                u = gb.read_field(i).astype(np.complex128)
                rel = float(np.linalg.norm(u[fidx] - fref) / np.linalg.norm(fref))
                tl = O.transmission_loss(u, tl_r[-1])[::mg.BATCH_TL_STRIDE]
                mask = tl_ref[-1] < 100
                worst = (max(worst[0], rel), max(worst[1], float(np.max(np.abs(tl - tl_ref[-1])[mask]))))
            rec["parity"] = {"worst_field_rel_l2_sampled": worst[0], "worst_final_tl_err_db": worst[1],
                             "against": "stored FP64 oracle runs of 8 members, fixed 12 terms "
                                        "(tests/golden/batch_n1023_s2000_fixed12.txt)"}
        out[mode] = rec
        gb.close()
        for pl in plans:
            pl.close()
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        peak = 1900.0
    for mode in ("bf16x3",):
        if out[mode]["tensor_tflops"]:
            out[mode]["frac_of_bf16_peak"] = out[mode]["tensor_tflops"] / peak
    print(json.dumps({"metric": METRIC, "unit": UNIT, "config": {"workload": "batch_gemm_dst", "solves": len(solves),
                      "N": solves[0].N, "range_steps": steps, "gemm": f"{L} x {C} x {L} per transform, "
                      "128 x 64 output tiles, K split over 2-CTA clusters (partials summed in distributed shared memory), "
                      "tcgen05.mma kind::f16 / kind::tf32"}, "bf16_peak_tflops": peak,
                      "modes": out}), flush=True)


def bench_fdssp(args):
    """The coarse-grid comparison of Section 4.3 (FD-SSP, the 3-point stencil, against SSSP):
    Munk with H = 4 km, 20 Hz, a smooth beam exp(-((z - 1000 m)/200 m)^2), [4/4], 400 steps of
    50 m; a reference SSSP march on 2047 points, then SSSP and FD-SSP on 127, 255 and 511 points:
    the field error at the common depths and the device time of each march."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from paper_2511_03343_gb300 import inputs, sssp
    stream = torch.cuda.current_stream()
    H, f, dr, steps, zs = 4000.0, 20.0, 50.0, args.range_steps if args.range_steps != 2000 else 400, 1000.0

    def run(N, op):
        s = inputs.munk(N=N, H=H, freq=f, dr=dr, steps=steps, pade_order=4, zs=zs)
        s.u0 = np.exp(-((s.z - zs) / 200.0) ** 2).astype(np.complex128)
        pl = sssp.plan_for(s, stream=stream, op=op)
        pl.march(2)
        pl.set_field(s.u0, 0.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pl.march(steps)
        e1.record(stream)
        u = pl.read_field()
        pl.close()
        return u, e0.elapsed_time(e1)

    ref, _ = run(2047, "spectral")
    rows = []
    for N in (127, 255, 511):
        stride = 2048 // (N + 1)
        r = ref[stride - 1::stride]
        for op in ("spectral", "fd3"):
            u, ms = run(N, op)
            rows.append({"N": N, "dz_m": H / (N + 1), "operator": "SSSP" if op == "spectral" else "FD-SSP",
                         "field_rel_l2_vs_sssp_2047": float(np.linalg.norm(u - r) / np.linalg.norm(r)),
                         "ms_per_march": ms, "throughput": N * steps / (ms * 1e-3)})
    print(json.dumps({"metric": "coarse-grid field error (Section 4.3)", "unit": "relative L2",
                      "config": {"workload": "fdssp_coarse_grid", "H_m": H, "freq_hz": f, "dr_m": dr,
                                 "range_steps": steps, "pade_order": 4, "reference": "SSSP, N = 2047"},
                      "rows": rows}), flush=True)


def bench_dst(args):
    """Transform-level comparison: the library's batched DST-I kernels against a cuFFT DST-I
    (odd extension to length 2(N+1), complex64 C2C through torch.fft; comparison baseline only).
    Inputs larger than L2 where the batch allows; per-transform device time with CUDA events."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from paper_2511_03343_gb300 import sssp
    stream = torch.cuda.current_stream()
    rows = []
    for N, count in [(1023, 256), (1023, 16384), (4095, 1), (4095, 4096), (16383, 512), (65535, 128)]:
        L = N + 1
        x = torch.randn(count, N, dtype=torch.complex64, device="cuda")
        out = torch.empty_like(x)
        pl = sssp.Plan(N, 100.0, 0.4, 5.0, 4, stream=stream)

        def ours():
            pl.dst1_batch(x, out)

        ext = torch.zeros(count, 2 * L, dtype=torch.complex64, device="cuda")

        def cufft():
            ext[:, 1:L] = x
            ext[:, L + 1:] = -torch.flip(x, dims=[1])
            return 0.5j * torch.fft.fft(ext, dim=1)[:, 1:L]

        res = {}
        for name, fn in [("ours", ours), ("cufft", cufft)]:
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / reps / count * 1e3  # us per transform
        ref = cufft()
        ours()
        err = float((out - ref).abs().max() / ref.abs().max())
        io = 16.0 * N  # read + write one complex64 vector
        rows.append({"N": N, "batch": count, "us_per_dst_ours": res["ours"], "us_per_dst_cufft": res["cufft"],
                     "speedup_vs_cufft": res["cufft"] / res["ours"],
                     "io_GBps_ours": io / (res["ours"] * 1e-6) / 1e9, "max_rel_diff": err})
        pl.close()
        del x, out, ext
    print(json.dumps({"metric": "DST-I time per transform", "unit": "us", "rows": rows}), flush=True)


def bench_munk(args):
    import numpy as np
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2511_03343_gb300 import build as B
    B.build()
    from paper_2511_03343_gb300 import inputs, sssp
    s = inputs.munk(steps=args.range_steps)
    stream = torch.cuda.current_stream()
    pl = sssp.Plan(s.N, s.H, s.k0, s.dr, s.pade_order, s.neumann_terms, s.neumann_tol, stream=stream)
    pl.set_kernel(args.kernel)
    pl.set_output(1)
    pl.set_profile_nodes(s.profiles)
    u0_dev = torch.from_numpy(s.u0.astype(np.complex64)).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    per_launch_dst = []

    def one_step(ev=None):
        pl.set_field(u0_dev, 0.0)
        c0 = None
        if ev is not None:
            ev[0].record(stream)
        pl.march(s.steps)
        if ev is not None:
            ev[1].record(stream)
        return c0

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    nd0 = pl.transform_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[2].record(stream)
        one_step(e)
        e[3].record(stream)
        torch.cuda.synchronize()
        step_ms.append(e[2].elapsed_time(e[3]))
        kern_ms.append(e[0].elapsed_time(e[1]))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    nd1 = pl.transform_count()
    dst_per_launch = (nd1 - nd0) / args.steps
    tot_ms, units = aggregate_over_ranks(sum(step_ms), float(s.N * s.steps * args.steps), device="cuda")
    value = units / (tot_ms * 1e-3)
    # parity of the bench's own output
    tl, _ = pl.read_tl()
    u = pl.read_field()
    parity = _golden_check(tl, u) if s.steps == 2000 else None

    # end to end through the public API with host (pinned) buffers
    u0_host = torch.from_numpy(s.u0.astype(np.complex64)).pin_memory()
    tl_host = torch.empty(s.steps * s.N, dtype=torch.float32).pin_memory()
    field_host = torch.empty(s.N, dtype=torch.complex64).pin_memory()
    e2e_ms = []
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl.set_field(u0_host, 0.0)
        pl.march(s.steps)
        pl.read_tl(out=tl_host)
        pl.read_field(out=field_host)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_ms.append(el * 1e3)
    e2e_tot = sum(e2e_ms) if e2e_ms else float("nan")
    e2e_tot, _ = aggregate_over_ranks(e2e_tot, 0.0, device="cuda")

    # roofline of the dominant kernel (the fused march kernel, FP32 ALU bound)
    kern_avg = sum(kern_ms) / len(kern_ms)
    N = s.N
    diag = 10.0 * (N + 1)  # per transform: the diagonal multiplies around it
    flops = dst_per_launch * (_dst_flops(N) + diag)
    achieved = flops / (kern_avg * 1e-3) / 1e12
    sm_max = float(clk.get("sm_max_mhz") or 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flop x max SM clock
    line = None
    if rank == 0:
        cpu = run_cpu_oracle_sample(args.cpu_seconds, "munk") if (world == 1 and not args.no_cpu) else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": _config({"kernel": pl.kernel}),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None,
                             "kernel": ("sssp_march_cluster_kernel<12, 8> (one solve over an 8-CTA cluster, 8 SMs)"
                                        if pl.kernel == "cluster" else "sssp_march_kernel<12> (one CTA, one SM)"),
                             "flops_per_launch": flops, "dst_per_launch": dst_per_launch,
                             "kernel_ms": kern_avg,
                             "peak_note": f"FP32 FMA peak of all {sms} SMs at the sampled max SM clock (derived, not measured)"},
                "e2e": {"value": s.N * s.steps * args.steps * world / (e2e_tot * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": s.N * 8, "d2h_bytes_per_step": s.N * s.steps * 4 + s.N * 8},
                "gpu_launches": 2 * args.steps,
                "clocks": clk, "parity": parity, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    pl.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-sample-steps", type=int, default=10)
    ap.add_argument("--range-steps", type=int, default=2000,
                    help="range steps per march (2000 = the workload; fewer only for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="batch",
                    choices=["munk", "batch", "eddy", "iso", "serve", "gemm", "dst", "large", "fdssp"])
    ap.add_argument("--large-count", type=int, default=64, help="solves in the N = 65535 batch ('large')")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--range-scale", type=float, default=1.0)
    ap.add_argument("--served-range-scale", type=float, default=0.2,
                    help="range scale of the serving trace replayed inside the default bench line")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune", action="store_true",
                    help="eddy / large / iso workloads: run the shape autotuner before timing")
    ap.add_argument("--gemm-fp32-steps", type=int, default=2000)
    ap.add_argument("--chunk-steps", type=int, default=50)
    ap.add_argument("--pacing", type=int, default=64,
                    help="serving: a cheaper request marches up to this many chunks per server step (1: lockstep)")
    ap.add_argument("--serve-baseline", action="store_true")
    ap.add_argument("--baseline-steps", type=int, default=4)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--kernel", default="auto", choices=["auto", "cta", "cluster"],
                    help="march kernel: one CTA per solve, one solve per thread-block cluster, or automatic")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "serve":
        bench_serve(args)
    elif args.workload == "gemm":
        bench_gemm(args)
    elif args.workload == "dst":
        bench_dst(args)
    elif args.workload == "fdssp":
        bench_fdssp(args)
    elif args.workload == "munk":
        bench_munk(args)
    elif args.workload == "batch":
        bench_batch(args)
    else:
        bench_other(args)


if __name__ == "__main__":
    main()
