"""Benchmark: AWG-PCG solves per second to a 1e-8 relative residual on one GB300.

Workload (default): 2D heterogeneous diffusion, 512 x 512 cells (n = 262144),
coefficient 1 with 20 seeded horizontal channels of width 2 at 1e6, 16 x 16
box subdomains grown by 2 layers, GenEO threshold tau = 0.1, b ~ N(0, 1).
One step = one full PCG solve (x_0 = 0, stop at ||b - A x|| <= 1e-8 ||b||)
preconditioned by H_3,ad with H_2 = H^NN_hyb(0.1); the setup (GenEO block
eigensolver from the learned start, network trained on the device on other
instances) runs once before the timed region.  Forms timed: FP64 (plain),
the mixed storage forms (float32 local operators; W in float32, bfloat16 or
scaled float16; float64 recurrences and coarse solves), and the batched
forms (suffix _block): one step = one block PCG solve of --nrhs right-hand
sides (default 32), each column with its own recurrence to 1e-8, W passes of
the float16 form on the tensor cores.  `value` is the fastest form, in
solves (right-hand sides brought to 1e-8) per second.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl awg|reference]
Under torchrun (N > 1) every rank solves its own copy of the problem
(independent replicas: the solver does not shard one problem over GPUs).
"""

from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG solves/sec to 1e-8 rel. residual: mixed+learned+batched vs plain FP64, 1 GB300"
UNIT = "solves/s"
RTOL = 1e-8
WORKLOAD = ("2D heterogeneous diffusion 512x512 (n=262144), 20 channels of width 2 at 1e6, "
            "16x16=256 box subdomains, overlap 2, tau=0.1, single RHS ~ N(0,1), H3,ad + H_hyb^NN")


def _problem(name):
    import awg_inputs as gi
    if name == "config2":
        return gi.config2()
    if name == "config1":
        return gi.config1()
    if name.startswith("channels"):
        L = int(name[len("channels"):])
        return gi.channels2d(L, q=L // 32, nchan=max(1, round(20 * L / 512)), contrast=1e6, seed=2,
                             overlap=2, tau=0.1)
    raise ValueError(name)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"awg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------- oracle arms
def oracle_sample(steps: int = 1):
    """Time the CPU oracle's PCG (its own setup untimed) on a 128 x 128 instance
    of the same generator (4 x 4 boxes of the same 32 x 32 size, overlap 2,
    5 channels), and scale solves/s to the full workload by the number of
    subdomains (the per-solve work of every step is per subdomain)."""
    import awg_inputs as gi
    import oracle as O
    p = gi.channels2d(128, q=4, nchan=5, contrast=1e6, seed=2, overlap=2, tau=0.1)
    t0 = time.perf_counter()
    st = O.setup_problem(p)
    setup_s = time.perf_counter() - t0
    times, its = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        res = O.pcg(lambda v: st.A @ v, p.b, lambda r: O.H3_ad_apply(st, r), rtol=RTOL)
        times.append(time.perf_counter() - t0)
        its.append(res.iters)
    sample_rate = 1.0 / statistics.median(times)
    scale = p.nparts / 256.0
    return {"value": sample_rate * scale, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle H3,ad PCG solve on the 128x128 instance of the same generator "
                       f"(16 subdomains of the same size; setup untimed, {setup_s:.1f} s); "
                       f"{sample_rate:.3f} solves/s measured, scaled by 16/256 subdomains"),
            "iters": its, "sample_solve_s": statistics.median(times)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, args.steps)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(1)
    t0 = time.perf_counter()
    cb = oracle_sample(steps)
    wall = time.perf_counter() - t0
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "CPU oracle (NumPy/SciPy FP64)"},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
FP64_TFLOPS = 1.197  # measured float64 FMA rate of this GPU (TFLOP/s)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def roofline_of(form, info):
    """Roofline of the dominant kernel class of a timed form (largest summed
    CUDA-event time): algorithmic bytes (or flops) per launch over the
    average event-timed launch.  Algorithmic bytes are the minimum traffic of
    one launch: the operator read once (W with w bytes per element, the
    local pseudo-inverses with g bytes), its input and output vectors once.
    Float64 passes with one FMA per 8-byte element, and the float64 coarse
    GEMMs of the block form, are bound by the float64 pipes, not by HBM."""
    n, nm, nnz = info["n"], info["n_minus"], info["nnz"]
    n0, sum_ns, dense = info["n0"], info["sum_ns"], info["dense_total"]
    ldw = (nm + 7) // 8 * 8
    prec = form["prec"]
    from paper_2106_10913_gb300 import FP64, MIXED_BF16, MIXED_FP16, MIXED_FP32
    w = {FP64: 8, MIXED_FP32: 4, MIXED_BF16: 2, MIXED_FP16: 2}[prec]
    g = 8 if prec == FP64 else 4
    sc = 4 if prec == MIXED_FP16 else 0
    prof = form["prof"]
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    cls = {}
    if not form["block"]:
        cls["wt"] = ("k_wt_partial (W^T r)", "bytes", n * ldw * w + 8 * n + sc * n)
        cls["wd"] = ("k_w_d (W d)", "bytes", n * ldw * w + 16 * n + 8 * nm + sc * n)
        cls["local"] = ("k_local_gemv (batched local pseudo-inverses)", "bytes", dense * g + 16 * sum_ns)
        cls["spmv"] = ("k_spmv", "bytes", 12 * nnz + 4 * (n + 1) + 16 * n)
    else:
        K = form["nrhs"]
        K = 16 if K <= 16 else (32 if K <= 32 else 64)
        v = 8 if prec == FP64 else 4  # internal block vectors
        tc = prec in (MIXED_FP16, MIXED_BF16)
        cls["wt"] = ("k_umma_wt (tcgen05 W^T B)" if tc else "kb_wt_partial (W^T B)", "bytes",
                     n * ldw * w + (2 * K * n * 2 if tc else n * K * v) + ldw * K * 4)
        cls["wd"] = ("k_umma_wd (tcgen05 W D)" if tc else "kb_w_d (W D)", "bytes",
                     n * ldw * w + (2 * K * ldw * 2 if tc else ldw * K * v) + n * K * 4)
        cls["local"] = ("kb_local_gemm (batched local pseudo-inverses, K columns)", "bytes",
                        dense * g + 2 * sum_ns * K * v)
        # E^-1 twice and F^-1 once per apply: average float64 flops per launch
        cls["coarse"] = ("kb_dense_part + kb_dense_sum (float64 E^-1, F^-1 on K columns)", "flops",
                         2 * K * (2 * n0 * n0 + nm * nm) / 3.0)
    cand = {k: prof["ms"][k] for k in cls if prof["count"][k] > 0}
    dom = max(cand, key=cand.get)
    name, kind, units = cls[dom]
    per_launch_ms = prof["ms"][dom] / prof["count"][dom]
    out = {"kernel": name, "avg_launch_ms": per_launch_ms, "launches": prof["count"][dom],
           "kernel_share_of_step": prof["ms"][dom] / form["ms"], "traffic": None}
    if kind == "flops":
        achieved = units / (per_launch_ms / 1000.0) / 1e12
        out.update({"bound": "alu", "achieved": achieved, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_TFLOPS, "algorithmic_flops_per_launch": units,
                    "peak_source": "measured float64 FMA rate 1.197 TFLOP/s"})
        return out
    achieved = units / (per_launch_ms / 1000.0) / 1e9
    out.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "algorithmic_bytes_per_launch": units, "peak_source": hbm_src})
    if prec == FP64 and dom in ("wt", "wd", "local"):
        # one float64 FMA per 8-byte element (per K columns in the block form)
        kk = form["nrhs"] if form["block"] else 1
        out["bound"] = "alu"
        out["peak"] = FP64_TFLOPS * 1e3 * 8 / 2 / kk
        out["frac"] = achieved / out["peak"]
        out["peak_source"] = "measured float64 FMA rate 1.197 TFLOP/s x 4 bytes/flop / columns"
    return out


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: every rank contributes its own, all get the max."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, per_step: int, ms: float) -> float:
    """Whole-job solves per second: every rank (an independent replica)
    brings `per_step` right-hand sides to 1e-8 per step, timed by the
    slowest rank."""
    return world * steps * per_step / (ms / 1000.0)


def run_awg(args):
    import torch
    import torch.distributed as dist
    from paper_2106_10913_gb300 import (AWGSolver, FP64, MIXED_BF16, MIXED_FP16, MIXED_FP32, awg_pcg, awg_pcg_block,
                                        awg_pcg_block_async,
                                        awg_profile, awg_profile_read)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    p = _problem(args.config)
    geneo_opts, train = {}, None
    if args.geneo == "learned":
        params, train = train_start_network()
        geneo_opts = {"geneo_solver": 2, "learned_params": params}
    elif args.geneo == "block":
        geneo_opts = {"geneo_solver": 1}
    t0 = time.perf_counter()
    # storage forms to build: float64 always, plus those of the timed forms
    pmask = 1
    for nm_ in args.forms.split(","):
        pmask |= 1 << {"fp64": 0, "mixed_fp32": 1, "mixed_bf16": 2,
                       "mixed_fp16": 3}[re.sub(r"_(block|graph)\d*$", "", nm_)]
    sol = AWGSolver(p.rowptr, p.colidx, p.val, p.part, p.nparts, p.overlap, p.tau,
                    precisions=pmask, verbose=int(args.verbose), **geneo_opts)
    setup_s = time.perf_counter() - t0
    info = dict(sol.info)
    info["dense_total"] = int(np.sum(sol.array("ns").astype(np.int64) ** 2))
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    forms = {}
    timed_mask = 0xFF  # every kernel class
    all_forms = {"fp64": FP64, "mixed_fp32": MIXED_FP32, "mixed_bf16": MIXED_BF16,
                 "mixed_fp16": MIXED_FP16}
    # batched forms: K right-hand sides per block solve, column 0 the
    # benchmark's b, the others seeded N(0, 1); a width suffix (e.g.
    # mixed_fp16_block32) overrides --nrhs
    Kmax = max([args.nrhs] + [int(m.group(3)) for m in (re.match(r"(.*)_(block|graph)(\d+)$", f)
                                                         for f in args.forms.split(",")) if m])
    import awg_inputs as gi
    Ball = gi.block_rhs(p, Kmax)
    bAll = torch.from_numpy(Ball).cuda()
    xAll = torch.zeros_like(bAll)
    g_its = torch.zeros(Kmax, dtype=torch.int32, device="cuda")
    g_rel = torch.zeros(Kmax, dtype=torch.float64, device="cuda")
    g_st = torch.zeros(1, dtype=torch.int32, device="cuda")

    for name in args.forms.split(","):
        m = re.match(r"(.*)_(block|graph)(\d*)$", name)
        graph = bool(m) and m.group(2) == "graph"
        block = bool(m)
        base = m.group(1) if m else name
        K = (int(m.group(3)) if m.group(3) else args.nrhs) if m else 1
        prec = all_forms[base]
        bB, xB = bAll[:K], xAll[:K]
        if graph:
            solve = (lambda prec=prec, bB=bB, xB=xB, K=K:
                     awg_pcg_block_async(sol.h, bB, xB, g_its[:K], g_rel[:K], g_st, RTOL, precision=prec))
        elif block:
            solve = lambda prec=prec, bB=bB, xB=xB: awg_pcg_block(sol.h, bB, xB, RTOL, prec, check=False)
        else:
            solve = lambda prec=prec: awg_pcg(sol.h, b, x, RTOL, prec, check=False)
        per_step = K if block else 1
        for _ in range(args.warmup):
            solve()
        barrier()
        awg_profile(sol.h, timed_mask)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its, rels, sts, cols = [], [], [], {}
        with ClockSampler(local) as clk:
            barrier()
            torch.cuda.nvtx.range_push(f"timed_{name}")
            ev0.record(stream)
            for _ in range(args.steps):
                r = solve()
                if r is not None:
                    st, it, rel = r
                    its.append(max(it))
                    rels.append(max(rel))
                    sts.append(st)
                    cols = {c: int(it[c]) for c in (0, 1, 77, 127) if c < len(it)}
            ev1.record(stream)
            torch.cuda.nvtx.range_pop()
            barrier()
        prof = awg_profile_read(sol.h)
        awg_profile(sol.h, 0)
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
        if not its:  # graph-driven solves: device results of the last step
            its = [int(g_its[:K].max().item())]
            rels = [float(g_rel[:K].max().item())]
            sts = [int(g_st.item())]
            cols = {c: int(g_its[c].item()) for c in (0, 1, 77, 127) if c < K}
        # every solver reports the TRUE relative residual of the columns it
        # stopped as converged (the graph-driven loop confirms the recurrence
        # residual on b - A x inside the graph)
        ok = all(s == 0 for s in sts) and max(rels) <= RTOL
        forms[name] = {"prec": prec, "block": block, "graph": graph, "nrhs": per_step, "ms": ms,
                       "value": job_throughput(world, args.steps, per_step, ms),
                       "ms_per_step": ms / args.steps, "iters": its[0], "iters_cols": cols, "relres": max(rels),
                       "ok": ok, "prof": prof, "clocks": clk.summary()}

    best = max((f for f in forms.values() if f["ok"]), key=lambda f: f["value"],
               default=next(iter(forms.values())))
    best_name = [k for k, v in forms.items() if v is best][0]
    # kernels inside a graph loop are not event-timed: the roofline of a
    # graph-driven form comes from the host-driven run of the same kernels
    rform = best
    if best["graph"]:
        base = re.sub(r"_graph\d*$", "", best_name)
        twins = [k for k, v in forms.items() if not v["graph"] and v["block"] and k.startswith(base + "_block")]
        if twins:
            rform = forms[max(twins, key=lambda k: forms[k]["nrhs"])]
    roofline = roofline_of(rform, info)
    if rform is not best:
        roofline["timed_in"] = [k for k, v in forms.items() if v is rform][0]

    # end to end: host buffers through the public API (H2D b, solve, D2H x)
    hb = torch.from_numpy(np.ascontiguousarray(Ball[:best["nrhs"]]) if best["block"] else p.b).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty_like(hb, device="cuda")
    dx = torch.zeros_like(db)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        db.copy_(hb, non_blocking=True)
        if best["graph"]:
            awg_pcg_block_async(sol.h, db, dx, g_its[:best["nrhs"]], g_rel[:best["nrhs"]], g_st, RTOL,
                                precision=best["prec"])
        elif best["block"]:
            awg_pcg_block(sol.h, db, dx, RTOL, best["prec"], check=False)
        else:
            awg_pcg(sol.h, db, dx, RTOL, best["prec"], check=False)
        hx.copy_(dx, non_blocking=True)
        stream.synchronize()
    e1.record(stream)
    barrier()
    ems = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    e2e = {"value": job_throughput(world, args.steps, best["nrhs"], ems), "unit": UNIT,
           "h2d_bytes_per_step": int(hb.numel() * 8), "d2h_bytes_per_step": int(hx.numel() * 8),
           "form": best_name}

    from paper_2106_10913_gb300 import awg_get_info
    tuned = awg_get_info(sol.h)
    autotune = {"widths": [16, 32, 64], "wt_ctas_per_sm": tuned["block_wt_ctas"],
                "dense_blocks_per_sm": tuned["block_dense_bps"]}
    batch = batched_problems(args, barrier) if args.batch_problems > 0 else None

    if rank == 0:
        cb = oracle_sample(1) if (world == 1 and not args.no_cpu_baseline) else None
        line = {
            "metric": METRIC, "value": best["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {FP64: "f64", MIXED_FP32: "f32+f64", MIXED_BF16: "bf16+f32+f64",
                      MIXED_FP16: "f16+f32+f64"}[best["prec"]],
            "data": "synthetic",
            "config": {"workload": WORKLOAD + (f"; batched form: {best['nrhs']} right-hand sides per block "
                                               "solve (column 0 the benchmark b, the rest seeded N(0,1)), "
                                               "each column its own PCG to 1e-8" if best["block"] else ""),
                       "form": best_name, "nrhs_per_step": best["nrhs"], "n": p.n, "nparts": p.nparts,
                       "overlap": p.overlap, "tau": p.tau, "rtol": RTOL,
                       "n0": info["n0"], "n_minus": info["n_minus"], "iters": best["iters"],
                       "l2": "inputs larger than L2 (W and local operators are GBs)",
                       "setup_s": round(setup_s, 2),
                       "setup_ms": dict(zip(("structure", "split", "local", "geneo", "E", "W", "F",
                                             "total"), (round(v, 1) for v in info["setup_ms"]))),
                       "geneo": {"solver": args.geneo, "block_steps_max": info["geneo_its_max"],
                                 "block_steps_sum": info["geneo_its_sum"],
                                 "dense_subdomains": info["geneo_dense"], "training": train},
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "block_autotune": autotune},
            "forms": {k: {"value": v["value"], "ms_per_step": v["ms_per_step"], "nrhs": v["nrhs"],
                          "iters": v["iters"], "iters_cols": v["iters_cols"], "relres": v["relres"],
                          "ok": v["ok"],
                          "kernel_ms": {c: round(t, 3) for c, t in v["prof"]["ms"].items()},
                          "launches": v["prof"]["launches"]} for k, v in forms.items()},
            "speedup_vs_plain_fp64": (best["value"] / forms["fp64"]["value"]) if "fp64" in forms else None,
            "batched_problems": batch,
            "roofline": roofline,
            "cpu_baseline": ({k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
                             if cb else None),
            "e2e": e2e,
            "gpu_launches": int(best["prof"]["launches"]),
            "clocks": best["clocks"],
            "kernel_ms": {k: round(v, 3) for k, v in best["prof"]["ms"].items()},
        }
        print(json.dumps(line), flush=True)
    sol.close()
    if world > 1:
        dist.destroy_process_group()


def batched_problems(args, barrier):
    """Independent problems solved together (the batched-problem workload at
    reduced size): P channel problems of the batch generator (side L drawn
    from [Lmin, Lmax], q x q boxes, contrast 10^U(4,6), one right-hand side
    each), every one with its own handle.  Plain: one float64 single-RHS
    solve after the other.  Batched: the mixed float16 graph-driven solves of
    all problems enqueued from one host thread (each handle on its own
    streams, no host synchronisation until the last), then one wait."""
    import torch
    import awg_inputs as gi
    from paper_2106_10913_gb300 import AWGSolver, FP64, MIXED_FP16, awg_pcg, awg_pcg_block_async
    lo, hi = (int(v) for v in args.batch_sides.split(","))
    probs = gi.batch_channels(args.batch_problems, Lmin=lo, Lmax=hi)
    t0 = time.perf_counter()
    sols = [AWGSolver(q.rowptr, q.colidx, q.val, q.part, q.nparts, q.overlap, q.tau, precisions=0b1001)
            for q in probs]
    setup_s = time.perf_counter() - t0
    bs = [torch.from_numpy(q.b).cuda() for q in probs]
    xs = [torch.zeros_like(v) for v in bs]
    B2 = [v[None, :].contiguous() for v in bs]
    X2 = [torch.zeros_like(v) for v in B2]
    its = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in probs]
    rel = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in probs]
    sts = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in probs]
    stream = torch.cuda.current_stream()

    def plain():
        out = []
        for s_, v, x_ in zip(sols, bs, xs):
            out.append(awg_pcg(s_.h, v, x_, RTOL, FP64, check=False))
        return out

    streams = [torch.cuda.Stream() for _ in probs]

    def batched():
        # one stream per problem: the solves overlap on the device
        for j, s_ in enumerate(sols):
            streams[j].wait_stream(stream)
            awg_pcg_block_async(s_.h, B2[j], X2[j], its[j], rel[j], sts[j], RTOL, precision=MIXED_FP16,
                                stream=streams[j])
        for sj in streams:
            stream.wait_stream(sj)

    res = {}
    for name, fn in (("plain_fp64", plain), ("batched_mixed_fp16_graph", batched)):
        for _ in range(max(1, args.warmup)):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r = fn()
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        if name == "plain_fp64":
            ok = all(st == 0 and rr[0] <= RTOL for st, _, rr in r)
            iters = [it[0] for _, it, _ in r]
        else:
            ok = all(int(t.item()) == 0 for t in sts) and max(float(t.item()) for t in rel) <= RTOL
            iters = [int(t.item()) for t in its]
        res[name] = {"value": args.steps * len(probs) / (ms / 1000.0), "unit": UNIT,
                     "ms_per_batch": ms / args.steps, "ok": ok, "iters": iters}
    for s_ in sols:
        s_.close()
    res["problems"] = [q.name for q in probs]
    res["setup_s"] = round(setup_s, 2)
    res["speedup"] = res["batched_mixed_fp16_graph"]["value"] / res["plain_fp64"]["value"]
    return res


def train_start_network(seeds=(3, 4, 5), steps=400, lr=1e-2):
    """Trains the start-block network on the device: features and leverage
    targets of three 128 x 128 channel instances (4 x 4 subdomains of the
    same 32 x 32 boxes as the benchmark problem, other seeds), full-batch
    Adam in float32 kernels.  Returns (params, summary)."""
    import torch
    import awg_inputs as gi
    from paper_2106_10913_gb300 import (AWGSolver, LEARNED_NFEAT, MIXED_FP32, awg_learned_data,
                                        awg_learned_train)
    t0 = time.perf_counter()
    Fs, ts = [], []
    for sd in seeds:
        q = gi.channels2d(128, q=4, nchan=5, contrast=1e6, seed=sd, overlap=2, tau=0.1)
        sol = AWGSolver(q.rowptr, q.colidx, q.val, q.part, q.nparts, q.overlap, q.tau)
        S = sol.info["sum_ns"]
        F = torch.zeros((S, LEARNED_NFEAT), dtype=torch.float64, device="cuda")
        t = torch.zeros(S, dtype=torch.float64, device="cuda")
        awg_learned_data(sol.h, F, t)
        torch.cuda.synchronize()
        sol.close()
        Fs.append(F)
        ts.append(t)
    F, t = torch.cat(Fs), torch.cat(ts)
    rng = np.random.default_rng(0)
    th0 = np.zeros(385)
    o = 0
    for fo, fi in ((16, 5), (16, 16), (1, 16)):  # Glorot-uniform weights, zero biases
        lim = np.sqrt(6.0 / (fi + fo))
        th0[o:o + fo * fi] = rng.uniform(-lim, lim, fo * fi)
        o += fo * fi + fo
    th, loss = awg_learned_train(F, t, th0, steps, lr, precision=MIXED_FP32)
    return th, {"instances": ["channels128 seed %d" % sd for sd in seeds], "samples": int(F.shape[0]),
                "steps": steps, "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
                "seconds": round(time.perf_counter() - t0, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="awg", choices=["awg", "reference"])
    ap.add_argument("--config", default="config2")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nrhs", type=int, default=64,
                    help="right-hand sides per step of the batched forms without a width suffix (<= 64 for "
                         "_block, <= 128 for _graph)")
    ap.add_argument("--batch-problems", type=int, default=8,
                    help="independent problems of the batched-problem measurement (0: skip)")
    ap.add_argument("--batch-sides", default="128,256", help="range of their grid sides")
    ap.add_argument("--forms", default="fp64,mixed_fp32,mixed_bf16,mixed_fp16,mixed_fp16_block32,mixed_fp16_block,"
                                      "mixed_fp32_block,mixed_fp16_graph128,mixed_fp32_graph128",
                    help="comma-separated storage forms to time; a _block suffix times the "
                         "batched (multi-right-hand-side) solve of --nrhs columns, _graph the same "
                         "solve as one CUDA graph launch with a device-side loop")
    ap.add_argument("--geneo", default="learned", choices=["learned", "block", "dense"],
                    help="GenEO eigensolver of the setup: block solver from the learned start "
                         "(network trained on the device on smaller instances), from a random "
                         "start, or the dense eigensolver")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_awg(args)


if __name__ == "__main__":
    main()
