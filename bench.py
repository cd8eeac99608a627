#!/usr/bin/env python
"""Benchmark of the batched GWN containment query on one GB300.

Workload (default): 16 models of trimmed bicubic rational patches (overlapping
perturbed box/cylinder unions, 1k-40k patches each, weights U[0.8, 1.2], an
outer polygonal trim loop and 0-2 polygonal holes per patch), queries
log-uniform in [65,536, 4,194,304] per model, uniform in each model's box --
the synthetic stand-in for the paper's CAD collection (Section 4.4).  One
step queries every model once (FP32 bulk with FP64 repair, beta chosen to meet
max |dGWN| <= 1e-4).  value = queries/s with points already on the device;
e2e = the same through the C ABI's host-buffer batch call
(gwn_query_batch_host: pinned host points in, values and labels out, copies
inside the timed region).  accuracy = the step's outputs against the exact
direct sum on the GPU (65,536 seeded queries per model) and, in the CPU leg,
against the FP64 oracle on the queries the GPU flagged plus seeded ones.  The
default run also measures configurations 1-3 (other_configs) and the serving
loop (serving).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl gwn|reference]

Multi-GPU: the query is data-parallel with no exchange step; N ranks run N
independent replicas of the whole step ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
T_START = time.time()


def log(msg):
    print(f"[bench {time.time() - T_START:7.1f}s] {msg}", file=sys.stderr, flush=True)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

BETA = 0.0              # 0: the build's autotuner picks beta and beta_leaf per model for max |dGWN| <= 1e-4
DIRECT_SAMPLE = 40960   # queries per model for the plain direct-sum comparison (fills the GPU)
ORACLE_FLAGGED = 2      # queries per model that the GPU flagged (repaired / near band) for the CPU oracle
ORACLE_SEEDED = 1       # seeded queries per model for the CPU oracle (about 10-20 s in all on 16 cores)
ORACLE_SEED = 4242
ACCURACY_SAMPLE = 65536  # seeded queries per model compared with the exact GPU direct sum
ACCURACY_SEED = 2026
WORKLOAD_NAME = ("cad16: 16 models of trimmed bicubic rational patches (box/cylinder unions), "
                 "queries uniform in each model's box")


def patches_box(patches):
    pts = np.concatenate([p.ctrl.reshape(-1, 3) for p in patches], axis=0)
    return pts.min(axis=0), pts.max(axis=0)


def build_workload(scale_queries: float = 1.0, n_models: int = 16):
    from synth import configs
    return configs.cad_batch_3d(query_scale=scale_queries)[:n_models]


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(ms, units_per_rank, world, device):
    """Replicas: every rank processes units_per_rank in ms.  Returns the
    slowest rank's ms and the whole-job rate (units of all ranks / that time)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3)


def flops_traversal(w, order3=False):
    # per internal node / leaf visited: far test (10); per Taylor evaluation: 72
    # at order 2, 120 with the order-3 terms (the quadratic and quartic of the
    # third-order moments); per query and cluster taken by its packet's local
    # expansion: 7 (one lane forms the cluster's ~200-flop expansion for the 32
    # queries of the warp, and the warp sums 10 coefficients)
    return (10 * (w["nodes"] + w["leaf_tests"]) + (120 if order3 else 72) * w["far"] +
            7 * w.get("local_nodes", 0))


FAST_NODE_FLOPS = 34    # a node read from a curve's node table: r, |r|, s.r, s x r, the integrand (+ 2 SFU ops)


def flops_leaves(w):
    # per Gauss-Legendre node of a degree-D boundary curve evaluated from its
    # Bernstein form: 28 D + 70 (value and derivative by Horner's rule, string
    # potential); per node read from a node table: 34; per foot-point search
    # 2000; per leaf evaluation set-up 30
    return (28 * w["gl_deg"] + 70 * w["gl_nodes"] + FAST_NODE_FLOPS * w["fast_nodes"] + 2000 * w["hits"] +
            30 * w["leaves"])


def fp32_peak_tflops(sm_mhz, sms):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def run_oracle_sample(workload, per_model, threads):
    import oracle
    t0 = time.perf_counter()
    nq = 0
    for patches, q in workload:
        oracle.gwn3d(patches, q[:per_model], n_threads=threads)
        nq += min(per_model, q.shape[0])
    return nq, time.perf_counter() - t0


def reference_arm(args):
    """The oracle (plain FP64 CPU direct sum) timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    workload = build_workload()
    threads = os.cpu_count() or 1
    per = 1
    for _ in range(args.warmup):
        run_oracle_sample(workload, per, threads)
    tot_q, tot_t = 0, 0.0
    for _ in range(args.steps):
        nq, dt = run_oracle_sample(workload, per, threads)
        tot_q += nq
        tot_t += dt
    val = tot_q / tot_t
    sample = f"{per} query per model x 16 models per step (exact FP64 direct sum over every patch)"
    line = {"metric": "GWN queries/s (batched containment, 16 trimmed-NURBS models)", "value": val,
            "unit": "queries/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "models": len(workload),
                       "patches": sum(len(p) for p, _ in workload),
                       "queries_per_step": sum(q.shape[0] for _, q in workload), "sample": sample},
            "cpu_baseline": {"value": val, "unit": "queries/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_leg(gwn, phase_s: float, log_fn):
    """Serving workload: 8 resident models behind the gwn_serve_* loop.

    Phase 1 (saturation): the first requests of the trace, about phase_s seconds
    of work, are submitted at once; sustained throughput = points / time to
    drain.  Phase 2 (open loop, a load sweep): Poisson arrivals at 0.25, 0.5,
    0.75 and 0.9 of the saturated request rate, phase_s seconds each; p50/p99
    of submit -> results ready, and the most requests whose device work
    overlapped.
    """
    import threading as th
    from synth import configs

    specs = configs.serve_models()
    models = []
    for dim, prims, lo, hi in specs:
        models.append(gwn.gwn_build_2d(prims) if dim == 2 else gwn.gwn_build_3d(prims))
    rng = np.random.default_rng(7)
    pools = [configs.uniform_queries(lo, hi, 2_000_000, rng).astype(np.float32) for _, _, lo, hi in specs]
    log_fn("serving: 8 models built")

    def run(times, midx, sizes, open_loop):
        srv = gwn.Server(n_slots=4)
        ids = [srv.add_model(m) for m in models]
        rids = []
        done = th.Event()

        def poller():
            k = 0
            while k < len(times):
                while k >= len(rids):
                    if done.wait(0.001) and k >= len(rids):
                        return
                srv.poll(rids[k][0], rids[k][1], timeout_ms=120000)
                k += 1

        pt = th.Thread(target=poller)
        pt.start()
        t0 = time.perf_counter()
        for t, mi, n in zip(times, midx, sizes):
            if open_loop:
                dt = t - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            off = int(rng.integers(0, pools[mi].shape[0] - n + 1))
            rids.append((srv.submit(ids[mi], pools[mi][off:off + n]), int(n)))
        done.set()
        pt.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return st, wall

    t_all, m_all, n_all = configs.serve_trace(2000.0, 60.0)
    # saturation: enough requests for about phase_s seconds at a first guess of 5e6 points/s
    k = int(np.searchsorted(np.cumsum(n_all), 5e6 * phase_s)) + 1
    st, wall = run(t_all[:k], m_all[:k], n_all[:k], open_loop=False)
    sat_qps = st["points_completed"] / wall
    sat_rps = k / wall
    log_fn(f"serving: saturation {sat_qps:.3e} points/s, {sat_rps:.1f} req/s, "
           f"max overlap on the GPU {st['max_gpu_overlap']}")
    sweep = []
    for i, load in enumerate((0.25, 0.5, 0.75, 0.9)):
        rate = load * sat_rps
        t_o, m_o, n_o = configs.serve_trace(rate, phase_s, seed=configs.BASE_SEED + 7 + i)
        st2, wall2 = run(t_o, m_o, n_o, open_loop=True)
        sweep.append({"load": load, "rate_req_s": rate, "duration_s": phase_s, "requests": int(st2["completed"]),
                      "p50_ms": st2["p50_ms"], "p99_ms": st2["p99_ms"], "mean_ms": st2["mean_ms"],
                      "points_per_s": st2["points_completed"] / wall2, "max_in_flight": int(st2["max_in_flight"]),
                      "max_gpu_overlap": int(st2["max_gpu_overlap"])})
        log_fn(f"serving: load {load} ({rate:.1f} req/s): p50 {st2['p50_ms']:.1f} ms, p99 {st2['p99_ms']:.1f} ms")
    for m in models:
        m.release()
    return {"metric": "serving latency, submit -> results ready", "unit": "ms",
            "models": "8 resident: 2 loops_2d (19,000 curves), 2 sphere_3d (384 patches), "
                      "4 cad_3d (1.5k-17k patches)",
            "sizes": "log-normal, median 16,384 points, sigma 1.5, clamped to [1000, 2e6]",
            "saturation": {"requests": k, "points_per_s": sat_qps, "requests_per_s": sat_rps,
                           "max_gpu_overlap": int(st["max_gpu_overlap"])},
            "load_sweep": sweep, "slots": 4, "precision": "fp32 bulk + fp64 repair"}


def config_leg(config: int, steps: int, warmup: int) -> dict:
    """One of the single-model configurations: 1 (2D star, exact FP64), 2 (2D
    nested loops, 1024^2 grid, FP32 + repair), 3 (trimmed sphere, 1M uniform
    queries, FP32 + repair).  Times the BVH query and the plain direct sum (on a
    sample, per-query time extrapolated) with CUDA events, and checks every
    query's value and label against the exact direct sum on the GPU (config 1:
    the FP64 direct sum; configs 2 and 3: the accuracy module's reference)."""
    import torch
    import paper_2605_19200_gb300 as gwn
    from paper_2605_19200_gb300 import accuracy
    from synth import configs

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    if config == 1:
        prims, q = configs.star_2d()
        dim, prec, qbeta, kw, direct_n = 2, gwn.PREC_FP64, 1e9, {"beta": 8.0, "precision": gwn.PREC_FP64}, 16384
        name = "1: 64-curve star, 2D, all FP64 (exact: tree with beta 1e9)"
    elif config == 2:
        prims, q = configs.loops_2d()
        dim, prec, qbeta, kw, direct_n = 2, gwn.PREC_FP32_REPAIR, 0.0, {"beta": 0.0}, 65536
        name = "2: 200 loops, 19,000 curves, 1024^2 grid, FP32 bulk + FP64 repair"
    else:
        prims, q = configs.sphere_3d()
        dim, prec, qbeta, kw, direct_n = 3, gwn.PREC_FP32_REPAIR, 0.0, {"beta": 0.0}, 65536
        name = "3: trimmed sphere, 384 patches, 1M uniform queries, FP32 bulk + FP64 repair"
    build = gwn.gwn_build_2d if dim == 2 else gwn.gwn_build_3d
    m = build(prims, **kw)
    md = accuracy.build_reference(prims, dim)
    pts = torch.from_numpy(q).to(torch.float64 if prec == gwn.PREC_FP64 else torch.float32).to(dev).contiguous()

    def timed(model, p, mode, beta):
        n = p.shape[0]
        out = (torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.int32, device=dev), None)
        for _ in range(max(1, warmup)):
            model.query(p, precision=prec, mode=mode, beta=beta, out=out, stream=stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            model.query(p, precision=prec, mode=mode, beta=beta, out=out, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        return n * steps / (a.elapsed_time(b) / 1e3), out

    qps, out = timed(m, pts, gwn.MODE_BVH, qbeta)
    dqps, _ = timed(md, pts[:direct_n].contiguous(), gwn.MODE_DIRECT, 0.0)
    if config == 1:
        wr, _, _ = md.query(pts, mode=gwn.MODE_DIRECT, precision=gwn.PREC_FP64, stream=stream)
        ref_name = "GPU FP64 direct sum over every curve, all 16,384 queries"
    else:
        wr, _, _ = accuracy.reference_values(md, pts, stream=stream)
        ref_name = "exact GPU direct sum (FP32 leaves, FP64 sum, FP64 near half-integers), every query"
    torch.cuda.synchronize()
    acc = accuracy.compare(out[0].cpu().numpy(), out[1].cpu().numpy(), wr.cpu().numpy())
    acc["reference"] = ref_name
    info = m.info()
    return {"metric": "GWN queries/s", "config": name, "value": qps, "unit": "queries/s",
            "direct_sum": {"value": dqps, "sample": f"{min(direct_n, pts.shape[0])} queries"},
            "speedup": qps / dqps, "beta": info["beta"], "beta_leaf": info["beta_leaf"],
            "leaves": info["n_leaves"], "steps": steps, "accuracy": acc}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gwn", choices=["gwn", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--models", type=int, default=16, help="first K models of the workload (default all 16)")
    ap.add_argument("--query-scale", type=float, default=1.0, help="fraction of each model's queries (default 1)")
    ap.add_argument("--beta", type=float, default=BETA)
    ap.add_argument("--beta-leaf", type=float, default=0.0)
    ap.add_argument("--local-ratio", type=float, default=0.0,
                    help="packet local expansion ratio of the models (<= 0: off, the default)")
    ap.add_argument("--tree-builder", type=int, default=-1, choices=[-1, 0, 1],
                    help="0: Karras LBVH; 1: top-down sweep; -1: the library's default (1)")
    ap.add_argument("--order", type=int, default=3, choices=[2, 3],
                    help="Taylor order of the models' build (3: the autotuner picks order 2 or 3 per model)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the single-model configurations 1-3")
    ap.add_argument("--streams", type=int, default=16,
                    help="streams of the batched query (one graph launch per step); 0 = one gwn_query per model")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="length of each serving phase")
    ap.add_argument("--kernels-only", action="store_true",
                    help="timed steps only (no e2e, direct-sum or CPU legs); for profiler runs")
    ap.add_argument("--config", type=int, default=0, choices=[0, 1, 2, 3],
                    help="1-3: time one of the single-model configurations instead of the 16-model workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.config:
        print(json.dumps(config_leg(args.config, args.steps, args.warmup)), flush=True)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2605_19200_gb300 as gwn

    t0 = time.perf_counter()
    workload = build_workload(args.query_scale, args.models)
    log("workload generated")
    models, points, outs = [], [], []
    for patches, q in workload:
        m = gwn.gwn_build_3d(patches, beta=args.beta, beta_leaf=args.beta_leaf, order=args.order,
                             tree_builder=args.tree_builder, local_ratio=args.local_ratio)
        models.append(m)
        pt = torch.from_numpy(q.astype(np.float32)).to(dev)
        points.append(pt)
        n = pt.shape[0]
        outs.append((torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
                     torch.empty(n, dtype=torch.int32, device=dev)))
    setup_s = time.perf_counter() - t0
    log(f"built {len(models)} models; (beta, beta_leaf) per model: "
        f"{[(round(m.info()['beta'], 1), round(m.info()['beta_leaf'], 1)) for m in models]}")
    total_q = sum(p.shape[0] for p in points)
    tuned = [(round(m.info()["beta"], 2), round(m.info()["beta_leaf"], 2)) for m in models]
    knobs = [(m.info()["bin_points_per_cell"], m.info()["stack_depth"]) for m in models]
    repair_betas = [(round(m.info()["beta_repair"], 2), round(m.info()["beta_repair_leaf"], 2)) for m in models]
    eval_orders = [m.info()["eval_order"] for m in models]
    local_ratios = [m.info()["local_ratio"] for m in models]
    n_leaves = sum(m.info()["n_leaves"] for m in models)
    n_patches = sum(len(p) for p, _ in workload)
    stream = torch.cuda.current_stream(dev)
    batch = gwn.Batch(n_streams=args.streams) if args.streams > 0 else None

    def step():
        if batch is not None:
            # all models and point sets in one CUDA-graph launch (captured on the first call)
            batch.query(models, points, outs, stream=stream)
        else:
            for m, p, o in zip(models, points, outs):
                m.query(p, out=o, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
        torch.cuda.synchronize()
        log("warm-up step")
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps' launches
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clk.stop()
    log(f"timed {args.steps} steps: {ms:.1f} ms/step")
    ms, value = aggregate_ranks(ms, total_q, world, dev)

    if args.kernels_only:
        if rank == 0:
            print(json.dumps({"metric": "GWN queries/s (kernels-only run)", "value": value, "unit": "queries/s",
                              "ms_per_step": ms, "queries_per_step": total_q}), flush=True)
        return

    # kernel-level numbers (untimed passes): event timing of the traversal, the
    # node-table and the full exact-leaf kernels on the query stream, and the
    # algorithmic work counters
    us = {"k_trav3": 0.0, "k_pair_fast": 0.0, "k_pair_eval": 0.0}
    fl = {"k_trav3": 0.0, "k_pair_fast": 0.0, "k_pair_eval": 0.0}
    repaired, pairs, near, full_pairs = 0, 0, 0, 0
    work_tot = {"fast_nodes": 0, "gl_nodes": 0, "hits": 0, "nodes": 0, "far": 0, "local_nodes": 0}
    for m, p, o in zip(models, points, outs):
        m.query(p, out=o, stream=stream, profile=True)
        s = m.last_query_stats()
        us["k_trav3"] += s["trav_us"]
        us["k_pair_fast"] += s["fast_us"]
        us["k_pair_eval"] += s["full_us"]
        m.query(p, out=o, stream=stream, count_work=True)
        w = m.last_query_stats()
        fl["k_trav3"] += flops_traversal(w, m.info()["eval_order"] >= 3)
        fl["k_pair_fast"] += FAST_NODE_FLOPS * w["fast_nodes"]
        fl["k_pair_eval"] += flops_leaves(w) - FAST_NODE_FLOPS * w["fast_nodes"]
        repaired += w["repaired"]
        pairs += w["pairs"]
        near += w["near_band"]
        full_pairs += w["full_pairs"]
        for k in ("fast_nodes", "gl_nodes", "hits", "nodes", "far", "local_nodes"):
            work_tot[k] += w[k]
    log("profiled and counted")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = fp32_peak_tflops(sm_mhz, sms)
    dominant = max(us, key=us.get)
    # per launch: algorithmic flops / event-timed duration (both summed over the
    # step's launches of the kernel, first round of each chunk)
    achieved = fl[dominant] / (us[dominant] * 1e-6) / 1e12
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "traffic_note": "ncu DRAM counters of the current kernels are in profiles/, not in this run",
                "peak_note": f"FP32 FMA issue: {sms} SMs x 128 lanes x 2 flops x {sm_mhz:.0f} MHz (median under load)",
                "ms_per_step": {k: v / 1e3 for k, v in us.items()},
                "tflops": {k: (fl[k] / (us[k] * 1e-6) / 1e12 if us[k] > 0 else None) for k in us}}

    # e2e through the C ABI with host buffers: gwn_query_batch_host copies every
    # model's points in and its values and labels out (one cudaMemcpyAsync per
    # buffer on the item's stream, captured with the kernels in the plan's
    # graph since the buffers are page-locked); timed over the same step count
    host_pts = [p.cpu().pin_memory() for p in points]
    host_out = [(torch.empty(p.shape[0], dtype=torch.float64).pin_memory(),
                 torch.empty(p.shape[0], dtype=torch.int32).pin_memory(), None) for p in points]
    hbatch = gwn.Batch(n_streams=max(1, args.streams))

    def step_e2e():
        hbatch.query_host(models, host_pts, host_out, stream=stream)

    for _ in range(max(3, args.warmup)):
        step_e2e()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t1) / args.steps
    log(f"e2e {e2e_s * 1e3:.1f} ms/step (gwn_query_batch_host)")
    _, e2e_value = aggregate_ranks(e2e_s * 1e3, total_q, world, dev)
    h2d = sum(p.numel() * p.element_size() for p in points)
    d2h = sum(p.shape[0] * (8 + 4) for p in points)
    e2e_diff = max(float(np.max(np.abs(ho[0].numpy() - o[0].cpu().numpy()))) for ho, o in zip(host_out, outs))
    hbatch.close()

    # plain GPU direct sum (every unsubdivided patch exact) on a sample of each
    # model's queries; the same model, with a wide FP64 band near half-integers,
    # is the exact reference of the accuracy check (65,536 seeded queries per model)
    from paper_2605_19200_gb300 import accuracy
    direct_q, direct_ms, acc_stats = 0, 0.0, []
    for mi, ((patches, q), p, o) in enumerate(zip(workload, points, outs)):
        md = accuracy.build_reference(patches, 3)
        sub = p[:DIRECT_SAMPLE].contiguous()
        md.query(sub, mode=gwn.MODE_DIRECT, stream=stream)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        md.query(sub, mode=gwn.MODE_DIRECT, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        # per-query cost is independent of the batch size: extrapolate to the model's queries
        direct_ms += a.elapsed_time(b) * (p.shape[0] / sub.shape[0])
        direct_q += p.shape[0]
        rng = np.random.default_rng(ACCURACY_SEED + mi)
        sel = np.sort(rng.choice(p.shape[0], size=min(ACCURACY_SAMPLE, p.shape[0]), replace=False))
        wr, _, _ = accuracy.reference_values(md, p[torch.from_numpy(sel).to(dev)].contiguous(), stream=stream)
        torch.cuda.synchronize()
        acc_stats.append(accuracy.compare(o[0].cpu().numpy()[sel], o[1].cpu().numpy()[sel], wr.cpu().numpy()))
        del md
    direct_qps = direct_q / (direct_ms / 1e3)
    acc = accuracy.merge(acc_stats)
    acc["reference"] = ("exact GPU direct sum over every unsubdivided patch (FP32 leaves, FP64 sum, FP64 near "
                        f"band, exact FP64 within {accuracy.REFERENCE_BAND} of half-integers)")
    acc["sample"] = f"{ACCURACY_SAMPLE} seeded queries per model x {len(models)} models"
    acc["label_rule"] = "round half away from zero; labels within 1e-6 of a half-integer not compared (Section 4.3)"
    log(f"direct sum {direct_qps:.3e} q/s; accuracy {acc['max_abs_dgwn']:.2e}, "
        f"{acc['label_mismatches']} label mismatches of {acc['labels_compared']}")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle (exact FP64 direct sum over every patch, CPU) on the queries
        # the GPU flagged (repaired or near band: the hardest ones) plus seeded
        # ones, timed on the host cores and compared with the GPU's values
        import oracle
        threads = os.cpu_count() or 1
        flag = gwn.QS_REPAIRED | gwn.QS_NEAR
        per_model = []
        for mi, ((patches, q), o) in enumerate(zip(workload, outs)):
            st = o[2].cpu().numpy()
            flagged = np.flatnonzero(st & flag)[:ORACLE_FLAGGED]
            rng = np.random.default_rng(ORACLE_SEED + mi)
            seeded = rng.choice(q.shape[0], size=ORACLE_SEEDED, replace=False)
            per_model.append(np.unique(np.concatenate([flagged, seeded])))
        t0 = time.perf_counter()
        oracle_w = []
        for (patches, q), idx in zip(workload, per_model):
            lo, hi = patches_box(patches)
            w_o, fl = oracle.gwn3d(patches, q[idx].astype(np.float64), near_thr=1e-6 * float(np.linalg.norm(hi - lo)),
                                   n_threads=threads)
            oracle_w.append((w_o, fl))
        dt = time.perf_counter() - t0
        nq = sum(len(i) for i in per_model)
        stats = []
        for (w_o, fl), idx, o in zip(oracle_w, per_model, outs):
            ok = (fl & 1) == 0   # labels next to the surface are not unique
            wg, lg = o[0].cpu().numpy()[idx], o[1].cpu().numpy()[idx]
            st = accuracy.compare(wg, lg, w_o)
            # labels are compared away from the surface too (the oracle's near flag)
            st["label_mismatches"] = int(np.sum((lg != np.round(w_o)) & ok &
                                                (np.abs(w_o - np.floor(w_o) - 0.5) > 1e-6)))
            stats.append(st)
        oc = accuracy.merge(stats)
        n_flagged = sum(int(np.sum((o[2].cpu().numpy()[idx] & flag) != 0)) for idx, o in zip(per_model, outs))
        sample = (f"{nq} queries: up to {ORACLE_FLAGGED} per model that the GPU flagged (repaired or near band), "
                  f"{n_flagged} in all, plus {ORACLE_SEEDED} seeded per model; exact FP64 direct sum, {dt:.1f} s")
        cpu = {"value": nq / dt, "unit": "queries/s", "cores": threads, "kind": "oracle", "sample": sample}
        acc["oracle_check"] = {"checked": oc["checked"], "flagged": n_flagged, "max_abs_dgwn": oc["max_abs_dgwn"],
                               "label_mismatches": oc["label_mismatches"]}
        log(f"oracle: {nq} queries in {dt:.1f} s, max |dGWN| {oc['max_abs_dgwn']:.2e}")

    other = None
    if rank == 0 and world == 1 and not args.no_configs:
        other = []
        for c in (1, 2, 3):
            other.append(config_leg(c, max(3, min(args.steps, 10)), 3))
            log(f"config {c}: {other[-1]['value']:.3e} q/s, accuracy {other[-1]['accuracy']['max_abs_dgwn']:.2e}")

    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = serving_leg(gwn, args.serve_seconds, log)

    # kernels per chunk of up to 2^20 points: box, bin, scan, scatter; 3 rounds of traversal, pair histogram,
    # scan, pair sort, node-table pairs, full pairs (+ round switch x2); near band, overflow, finish, the
    # chunk's own repair x4 (normally empty), counter accumulate; per query: repair x4 + its accumulate
    launches_per_step = sum(32 * math.ceil(p.shape[0] / (1 << 20)) + 5 for p in points)
    line = {
        "metric": "GWN queries/s (batched containment, 16 trimmed-NURBS models)",
        "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME,
                   "models": len(models), "patches": n_patches, "leaves": n_leaves, "queries_per_step": total_q,
                   "beta": "autotuned" if args.beta == 0 else args.beta, "beta_per_model": tuned,
                   "bin_points_per_cell_stack_depth_per_model": knobs,
                   "repair_beta_per_model": repair_betas,
                   "tolerance": 1e-4, "order": args.order, "eval_order_per_model": eval_orders,
                   "tree": "Karras LBVH" if args.tree_builder == 0 else "top-down sweep",
                   "local_ratio_per_model": local_ratios,
                   "precision": "fp32 bulk + fp64 repair",
                   "l2": f"inputs larger than L2 ({total_q * 12 / 1e6:.0f} MB of points per step)",
                   "parallelism": f"replicas x{world}", "setup_s": round(setup_s, 1),
                   "launch": (f"gwn_query_batch: one CUDA graph launch per step over {args.streams} streams"
                              if batch is not None else "one gwn_query per model")},
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "gwn_query_batch_host (pinned host buffers, one graph launch)",
                "steps": args.steps, "max_abs_diff_vs_device_run": e2e_diff},
        "roofline": roofline,
        "accuracy": acc,
        "direct_sum": {"value": direct_qps, "unit": "queries/s",
                       "sample": f"{DIRECT_SAMPLE} queries per model, FP32, per-query time extrapolated",
                       "speedup": value / direct_qps},
        "work": {"pairs_per_query": pairs / total_q, "near_band_pairs_per_query": near / total_q,
                 "repaired_fraction": repaired / total_q,
                 "full_evaluator_pair_fraction": full_pairs / max(pairs, 1),
                 "table_nodes_per_query": work_tot["fast_nodes"] / total_q,
                 "bernstein_nodes_per_query": work_tot["gl_nodes"] / total_q,
                 "foot_point_searches_per_query": work_tot["hits"] / total_q,
                 "nodes_visited_per_query": work_tot["nodes"] / total_q,
                 "taylor_terms_per_query": work_tot["far"] / total_q,
                 "packet_local_terms_per_query": work_tot["local_nodes"] / total_q},
        "clocks": clocks,
        "gpu_launches": launches_per_step * args.steps,
    }
    if other is not None:
        line["other_configs"] = other
    if serving is not None:
        line["serving"] = serving
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
