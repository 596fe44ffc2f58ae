#!/usr/bin/env python
"""Benchmark of the area-hint refinement initializer on GB300.

One step = the whole hot path on one synthetic netlist resident in HBM:
pl_build_graph (static graph, rebuilt in place) + pl_filter_init (GSP
initialization and T_hint rounds of area hints + refinement filter) +
pl_hpwl.  Metric: movable cells initialized per second (whole job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config large]
  python bench.py --impl reference ...   (the FP64 CPU oracle, host cores)

Under torchrun each rank runs its own replica netlist (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "area-hint init cells/s"
WORKLOADS = {
    # name: (netgen config, params)
    "large": ("large", dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                            tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))),
    "half": ("half", dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                          tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))),
    "medium": ("medium", dict(nbx=32, nby=32, wdtype=1)),
    "tiny": ("tiny", dict(nbx=16, nby=16, wdtype=1)),
}
DESCR = {
    "large": "2.2M std cells, 8k macros, 2.25M nets (degree cap 10k), 8k I/O; BF16 weights, "
             "FP32 coordinates; taps {2,4,8}; 32x32 bins; T_hint 3",
    "half": "1.1M std cells, 4k macros, 1.125M nets (cap 5k), 4k I/O; large's parameters "
            "(profiling case: matrix larger than L2, a few GB on the device)",
    "medium": "210k std cells, 550 macros, 220k nets (cap 2k), 1k I/O; FP32 weights; order 8",
    "tiny": "2k std cells, 20 macros, 2.2k nets; FP32; order 8",
}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", self.gpu], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_params(config):
    """The oracle's parameters for a bench workload (same names as the library's)."""
    return dict(WORKLOADS[config][1])


def oracle_sample(nl, config, parallel=False):
    """The FP64 oracle on one step of the bench workload itself (the same
    netlist: static graph, GSP init, 3 refinement rounds, HPWL), on one host
    thread or, with parallel, on all host cores (the OpenMP build, same
    results).  Returns movable cells per second, seconds, threads used."""
    import oracle
    kw = oracle_params(config)
    threads = oracle.host_cores() if parallel else 1
    t0 = time.perf_counter()
    o = oracle.Oracle(nl, parallel=parallel, **kw)
    gx, gy = o.run(1)
    oracle.hpwl(nl, gx[:nl.num_cells], gy[:nl.num_cells], parallel=parallel)
    dt = time.perf_counter() - t0
    return nl.num_movable / dt, dt, threads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2511_10073_gb300 import netgen
    oracle.build()
    oracle.build_parallel()
    cores = oracle.host_cores()
    # each step: the oracle (OpenMP build, all host cores) on the workload's
    # own netlist: static graph, GSP init, T_hint rounds, HPWL
    nl = netgen.make_netlist(WORKLOADS[args.config][0], args.seed)
    kw = oracle_params(args.config)

    def step():
        o = oracle.Oracle(nl, parallel=True, **kw)
        gx, gy = o.run(args.seed)
        oracle.hpwl(nl, gx[:nl.num_cells], gy[:nl.num_cells], parallel=True)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = nl.num_movable * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "netlist": DESCR[args.config]},
        "cpu_baseline": {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": f"the {args.config} workload's netlist each step (full path: "
                                   "static graph, GSP init, refinement rounds, HPWL), OpenMP "
                                   f"build on {cores} host cores"},
        "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


BATCH_PARAMS = dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                    tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))


def run_batched(pl, netgen, dev, stream, args, n=64):
    """The batched serving form: n designs of uneven size (std cells
    log-uniform in 5k-500k), each built once; one step initializes all of
    them.  The plain GPU form runs the designs one after another on one
    stream.  The batched form is pl_filter_init_batch with the options the
    library's autotuner (pl_batch_autotune) picks over 16 streams: the union
    form (one launch per kernel and power over all designs) or the per-design
    form, stream count, short-row CTAs per SM.  Every form gives the same
    bits, so the HPWL differs by 0."""
    import torch
    cfgs = netgen.batch_configs(args.seed, n=n)
    nls = [netgen.make_netlist(c, 1000 + i) for i, c in enumerate(cfgs)]
    prm = pl.params(**BATCH_PARAMS)
    dnls = [pl.DeviceNetlist(nl, dev) for nl in nls]
    graphs = [pl.pl_build_graph(d, prm) for d in dnls]
    outs = [torch.empty(nl.num_cells * 2, dtype=torch.float32, device=dev) for nl in nls]
    seeds = [args.seed + i for i in range(n)]
    movable = sum(nl.num_movable for nl in nls)
    streams = [torch.cuda.Stream(device=dev) for _ in range(16)]
    ws = pl.batch_workspace(n, prm, dev)

    def plain():
        for g, o, sd in zip(graphs, outs, seeds):
            pl.pl_filter_init(g, prm, sd, None, o)

    def timed(fn, reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    plain()
    ref = [o.clone() for o in outs]
    ms_plain = timed(plain, max(1, args.steps // 2))
    best, tune_ms = pl.pl_batch_autotune(graphs, prm, seeds, outs, streams, ws)
    reps = max(1, args.steps // 2)
    ms_batch = timed(lambda: pl.pl_filter_init_batch(graphs, prm, seeds, outs, streams, best, ws), reps)
    same = all(torch.equal(a, b) for a, b in zip(ref, outs))
    other = pl.batch_opts(union_products=1 - best.union_products, streams=best.streams or 16)
    ms_other = timed(lambda: pl.pl_filter_init_batch(graphs, prm, seeds, outs, streams, other, ws), reps)
    same = same and all(torch.equal(a, b) for a, b in zip(ref, outs))
    hws = [pl.hpwl_workspace(nl.num_nets, dev) for nl in nls]
    h = torch.zeros(2 * n, dtype=torch.float64, device=dev)
    for i, (d, o, w) in enumerate(zip(dnls, outs, hws)):
        pl.pl_hpwl(d, o, h[i:i + 1], w)
        pl.pl_hpwl(d, ref[i], h[n + i:n + i + 1], w)
    hp = h.cpu().numpy()
    rel = float(abs(hp[:n].sum() - hp[n:].sum()) / hp[n:].sum())
    for g in graphs:
        g.destroy()
    form = "union" if best.union_products else "per-design"
    return {"what": f"{n} designs, std cells log-uniform 5k-500k ({movable} movable cells), "
                    "each initialized from its seed (GiFt + 3 rounds, BF16, taps {2,4,8})",
            "unit": "cells/s", "value": movable / (ms_batch / 1e3),
            "plain_gpu_value": movable / (ms_plain / 1e3), "speedup": ms_plain / ms_batch,
            "ms_per_batch": ms_batch, "plain_ms_per_batch": ms_plain,
            "autotune": {"form": form, "streams": best.streams,
                         "rows_ctas_per_sm": best.rows_ctas_per_sm, "best_trial_ms": tune_ms},
            "other_form": {"form": "per-design" if best.union_products else "union",
                           "ms_per_batch": ms_other},
            "same_bits_as_plain": same, "hpwl_rel_diff": rel,
            "timing": "wall clock of whole batches after a synchronize (host threads drive "
                      "the streams)"}


LEARNED_DIR = os.path.join(ROOT, "paper_2511_10073_gb300", "weights")


def run_learned(pl, g, dnl, nl, args, dev, stream):
    """The learned filter in place of the plain one (every trained model
    committed under the package's weights/), on the workload's netlist with
    the parameters it was trained for (the workload's, fixed nodes re-pinned
    after every power).  The same step (graph build, initializer, HPWL) for
    the plain filter and for each model, timed with CUDA events; HPWL
    difference and the movable cells' coordinate RMS difference over the die."""
    import glob

    import numpy as np
    import torch
    files = sorted(glob.glob(os.path.join(LEARNED_DIR, "learned_k*.json")))
    if not files:
        return None
    models = [json.load(open(f)) for f in files]
    prm = pl.params(**models[0]["params"])
    out_plain = torch.empty(nl.num_cells * 2, dtype=torch.float32, device=dev)
    out = torch.empty_like(out_plain)
    ws = pl.hpwl_workspace(nl.num_nets, dev)
    hp = torch.zeros(1, dtype=torch.float64, device=dev)
    mov = torch.tensor(np.asarray(nl.cell_kind) == 0, device=dev)
    die = nl.region[2] - nl.region[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps // 2)

    def timed(m, dst):
        nf = [0]

        def step():
            pl.pl_build_graph(dnl, prm, graph=g)
            if m is None:
                pl.pl_filter_init(g, prm, args.seed, None, dst)
            else:
                nf[0] = pl.pl_filter_init_learned(g, prm, m, args.seed, None, dst)
            pl.pl_hpwl(dnl, dst, hp, ws)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, float(hp.item()), nf[0]

    ms_plain, hp_plain, _ = timed(None, out_plain)
    res = {}
    for d in models:
        m = pl.LearnedModel.from_host(d, dev)
        ms, h, nf = timed(m, out)
        dd = (out - out_plain).view(-1, 2)[mov].double()
        rms = float(torch.sqrt((dd * dd).sum(1).mean() / 2).item()) / die
        key = "k" + "".join(str(x) for x in m.k)
        res[key] = {"tap_powers": list(m.k), "products_per_round": m.k[2],
                    "value": nl.num_movable / (ms / 1e3), "unit": "cells/s", "ms_per_step": ms,
                    "speedup_vs_plain_gpu": ms_plain / ms, "hpwl": h,
                    "hpwl_delta": (h - hp_plain) / hp_plain, "coord_rms_over_die": rms,
                    "fallback_rounds": nf,
                    "within_gate": abs((h - hp_plain) / hp_plain) <= 1e-3,
                    "trained_on": d.get("data")}
    ok = [k for k, v in res.items() if v["within_gate"]]
    best = max(ok, key=lambda k: res[k]["speedup_vs_plain_gpu"]) if ok else None
    return {"what": "the whole step (graph build, initializer, HPWL) with the learned filter "
                    "(k2 sparse products per round, MLP on tensor cores) against the same step "
                    "with the plain filter (max(tap_k) products per round), same netlist and seed",
            "params": {k: (list(v) if isinstance(v, (list, tuple)) else v)
                       for k, v in models[0]["params"].items()},
            "plain": {"value": nl.num_movable / (ms_plain / 1e3), "unit": "cells/s",
                      "ms_per_step": ms_plain, "hpwl": hp_plain,
                      "products_per_round": max(prm.tap_k[:prm.ntaps])},
            "gate": "|HPWL delta| <= 0.1%", "best_within_gate": best, "models": res}


def whole_job_rate(ms_local, units_per_rank, steps, dist=None, device="cpu"):
    """Whole-job throughput of a replica run: the slowest rank's time (MAX over
    ranks) for the units all ranks processed.  Returns (units/s, max ms)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(t.item())
    return world * units_per_rank * steps / (ms_max / 1e3), ms_max


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-filter leg")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched serving form")
    ap.add_argument("--profile-learned", default=None, metavar="KEY",
                    help="with --profile-one: profile the step with the committed learned model "
                         "KEY (e.g. k012) instead of the plain filter")
    ap.add_argument("--profile-one", action="store_true",
                    help="warm up, then run one step inside a CUDA profiler range and exit "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        from paper_2511_10073_gb300 import build
        build.build()
    if dist:
        dist.barrier()
    import paper_2511_10073_gb300 as pl
    from paper_2511_10073_gb300 import netgen

    cfg, kw = WORKLOADS[args.config]
    nl = netgen.make_netlist(cfg, args.seed + rank)
    prm = pl.params(**kw)
    dev = f"cuda:{local}"
    dnl = pl.DeviceNetlist(nl, dev)
    g = pl.pl_build_graph(dnl, prm)
    out = torch.empty(nl.num_cells * 2, dtype=torch.float32, device=dev)
    ws = pl.hpwl_workspace(nl.num_nets, dev)
    hp = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        pl.pl_build_graph(dnl, prm, graph=g)
        pl.pl_filter_init(g, prm, args.seed, None, out)
        pl.pl_hpwl(dnl, out, hp, ws)

    if args.profile_one and args.profile_learned:
        # the step with a committed learned model (and the parameters it was trained for)
        d = json.load(open(os.path.join(LEARNED_DIR, f"learned_{args.profile_learned}.json")))
        lm = pl.LearnedModel.from_host(d, dev)
        prm = pl.params(**d["params"])

        def step():
            pl.pl_build_graph(dnl, prm, graph=g)
            pl.pl_filter_init_learned(g, prm, lm, args.seed, None, out)
            pl.pl_hpwl(dnl, out, hp, ws)

    for _ in range(max(3, args.warmup) if not args.profile_one else args.warmup):
        step()
    torch.cuda.synchronize()
    if args.profile_one:
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            info = g.info()
            print(json.dumps({"profile_one": args.config, "movable_cells": nl.num_movable,
                              "nodes": info["N"], "static_nnz": info["static_nnz"],
                              "augmented_nnz": info["nnz"], "hub_rows": info["hub_rows"]}))
        return

    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        gid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        gid = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[local]
    sampler = ClockSampler(gid)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    pl.pl_prof_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    pl.pl_prof_enable(False)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = pl.pl_prof_read()
    movable = nl.num_movable
    value, ms_max = whole_job_rate(ms, movable, args.steps, dist, dev)

    # end to end through the C ABI from host buffers: netlist H2D, results D2H
    # Two device copies of the netlist: step i runs on copy i % 2 while the
    # copy stream brings step i + 1's netlist into the other one (once step
    # i - 1, the last user of that copy, has finished).
    fields = ("net_ptr", "pin_cell", "pin_dx", "pin_dy", "cell_w", "cell_h", "cell_kind",
              "fixed_x", "fixed_y")
    host = {k: getattr(dnl, k).cpu().pin_memory() for k in fields}
    dnls = [dnl, pl.DeviceNetlist(nl, dev)]
    out_h = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    hp_h = torch.empty(1, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_h.numel() * out_h.element_size() + 8
    cstream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d_into(j):
        cstream.wait_event(used[j])
        with torch.cuda.stream(cstream):
            for k, v in host.items():
                getattr(dnls[j], k).copy_(v, non_blocking=True)
        copied[j].record(cstream)

    def e2e_run(n):
        for j in range(2):
            used[j].record(stream)
        h2d_into(0)
        for i in range(n):
            j = i % 2
            if i + 1 < n:
                h2d_into(1 - j)
            stream.wait_event(copied[j])
            pl.pl_build_graph(dnls[j], prm, graph=g)
            pl.pl_filter_init(g, prm, args.seed, None, out)
            pl.pl_hpwl(dnls[j], out, hp, ws)
            used[j].record(stream)
            out_h.copy_(out, non_blocking=True)
            hp_h.copy_(hp, non_blocking=True)

    e2e_run(2)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0.record(stream)
    ke = max(1, args.steps // 2)
    e2e_run(ke)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, _ = whole_job_rate(e0.elapsed_time(e1), movable, ke, dist, dev)

    # phase breakdown (untimed pass, CUDA events around each call)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    pl.pl_build_graph(dnl, prm, graph=g)
    ev[1].record(stream)
    pl.pl_filter_init(g, prm, args.seed, None, out)
    ev[2].record(stream)
    pl.pl_hpwl(dnl, out, hp, ws)
    ev[3].record(stream)
    torch.cuda.synchronize()
    phases = {"build_graph_ms": ev[0].elapsed_time(ev[1]), "filter_init_ms": ev[1].elapsed_time(ev[2]),
              "hpwl_ms": ev[2].elapsed_time(ev[3])}
    info = g.info()

    # macro charge-density schedules (Sec. VI) on this netlist's macros, over
    # a 512 x 512 bin grid (a global-placement grid), one call per model
    kind = np.asarray(nl.cell_kind)
    mids = np.flatnonzero(kind == netgen.KIND_MACRO)
    mgeo = [torch.tensor(np.asarray(a, np.float32)[mids], device=dev)
            for a in (nl.fixed_x, nl.fixed_y, nl.cell_w, nl.cell_h)]
    rho = torch.empty(512 * 512, dtype=torch.float64, device=dev)
    rho_ms = {}
    for model, name in enumerate(("gauss", "exp", "linear", "sigmoid")):
        rp = pl.rho_params(model=model)
        for _ in range(2):
            pl.pl_macro_density(rp, 150, *mgeo, nl.region, 512, 512, rho)
        e0.record(stream)
        for _ in range(5):
            pl.pl_macro_density(rp, 150, *mgeo, nl.region, 512, 512, rho)
        e1.record(stream)
        torch.cuda.synchronize()
        rho_ms[name] = e0.elapsed_time(e1) / 5

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    hr_ms_avg = prof["hr_ms"] / max(1, prof["hr_launches"])
    achieved = prof["hr_bytes"] / (prof["hr_ms"] / 1e3) / 1e9 if prof["hr_ms"] > 0 else None
    traffic = None
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        traffic = tr.get(args.config)
    except Exception:
        pass
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded netlist generator)",
        "config": {"workload": args.config, "netlist": DESCR[args.config],
                   "movable_cells": movable, "nodes": info["N"], "static_nnz": info["static_nnz"],
                   "augmented_nnz": info["nnz"], "hub_rows": info["hub_rows"],
                   "l2": "inputs larger than L2 (each sparse product streams >300 MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"kernel": "one sparse product of the refinement filter (A4): k_spmm_rows (short rows, "
                               "window slots) + k_spmm_hub, k_bin_partials, k_hub_rows (second "
                               "stream)",
                     "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": "measured" if pk else "fallback",
                     "avg_launch_ms": hr_ms_avg, "launches": prof["hr_launches"],
                     "algorithmic_bytes_per_launch": prof["hr_bytes"] / max(1, prof["hr_launches"])},
        "gpu_launches": prof["launches"],
        "phases": phases,
        "macro_density": {"what": "pl_macro_density at t = 150 of T = 300 (Sec. VI), this netlist's "
                                  f"{len(mids)} macros over 512 x 512 bins, FP64",
                          "ms_per_call": rho_ms},
        "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clocks,
    }
    if not args.no_learned:
        lr = run_learned(pl, g, dnl, nl, args, dev, stream)
        if lr is not None:
            line["learned"] = lr
    if not args.no_batch:
        line["batched"] = run_batched(pl, netgen, dev, stream, args)
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        oracle.build_parallel()
        v1, dt1, _ = oracle_sample(nl, args.config)
        vp, dtp, cores = oracle_sample(nl, args.config, parallel=True)
        what = (f"one step of the bench workload itself ({args.config}: static graph, GSP init, "
                f"3 refinement rounds, HPWL)")
        line["cpu_baseline"] = {"value": vp, "unit": "cells/s", "cores": cores, "kind": "oracle",
                                "sample": f"{what}, {dtp:.1f} s on {cores} host cores (OpenMP "
                                          "build, same results as the single-threaded oracle)",
                                "single_thread": {"value": v1, "unit": "cells/s", "cores": 1,
                                                  "sample": f"{what}, {dt1:.1f} s"}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
