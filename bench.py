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


WORKLOADS = {
    "config3": ("3D log-normal diffusion 96^3 (n=884736), sigma 3, correlation length 8, 512 uneven k-means "
                "subdomains, overlap 2, tau=0.1"),
    "config4": ("Q1 plane-strain elasticity 384x384 (n=295680), layered Young's modulus 1 / 1e5, 16x16 node boxes, "
                "overlap 2, tau=0.1, its 32 right-hand sides"),
}


def _workload(name, p):
    if name == "config2":
        return WORKLOAD
    return WORKLOADS.get(name, f"{p.name} (n={p.n}, {p.nparts} subdomains, overlap {p.overlap}, tau={p.tau})")


def _problem(name):
    import awg_inputs as gi
    if name == "config2":
        return gi.config2()
    if name == "config1":
        return gi.config1()
    if name == "config3":
        return gi.config3()
    if name == "config4":
        return gi.config4()
    if name.startswith("grf"):  # grf<L>: the 3D log-normal generator at L^3 with L^3 / 1728 k-means parts
        L = int(name[3:])
        return gi.grf3d(L, k=max(2, round(L ** 3 / 1728)))
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
GOLDEN = os.path.join(ROOT, "tests", "golden", "config2_oracle.json")


def _oracle_full_size_state(seed=0):
    """The oracle's setup record for the benchmark problem at its FULL size
    with operators of the shapes its own setup produces there (A itself;
    the 256 grown subdomains; per subdomain an n^s x n^s eigenvector block
    with the oracle's n^s_- non-positive eigenvalues; GenEO blocks of the
    oracle's per-subdomain mode counts; E and F of sizes n0 = 3204 and
    n_- = 3092 with their Cholesky factors; the dense n x n_- W), filled with
    seeded random values.  The oracle's own setup of this problem takes a
    quarter of an hour on the host; the counts come from its stored run
    (tests/golden/config2_oracle.json, written by the committed script that
    calls only the oracle).  The apply and PCG functions that run on this
    record are the oracle's, unmodified: their cost depends on these shapes,
    not on the values."""
    import scipy.linalg as sla
    import scipy.sparse as sp
    import awg_inputs as gi
    import oracle as O
    ref = json.load(open(GOLDEN))
    p = gi.config2()
    rng = np.random.default_rng(seed)
    A = O.csr_from(p.rowptr, p.colidx, p.val, p.n)
    subs = O.grow_subdomains(A, p.part, p.nparts, p.overlap)
    d, Ds = O.partition_of_unity(subs, p.n)
    nm_s = ref["n_minus_per_subdomain"]
    nst_s = ref["n_strict_per_subdomain"]
    modes = ref["modes_per_subdomain"]
    splits, rows, cols, vals = [], [], [], []
    col = 0
    for idx, m_minus, m_strict, k in zip(subs, nm_s, nst_s, modes):
        m = idx.size
        lam = np.concatenate([-rng.random(m_minus), 1.0 + rng.random(m - m_minus)])
        splits.append(O.LocalSplit(lam, rng.standard_normal((m, m)), int(m_minus), int(m_strict), 1e-12))
        if k:
            rr, cc = np.meshgrid(idx, np.arange(col, col + k), indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(rng.standard_normal(m * k))
            col += k
    n0, nm = ref["n0"], ref["n_minus"]
    st = O.Setup(A=A, n=p.n, subs=subs, d=d, Ds=Ds, B=None, splits=splits, tau=p.tau)
    st.Z = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(p.n, n0))

    def spd(k):
        G = rng.standard_normal((k, k))
        return G @ G.T + k * np.eye(k)

    st.E = spd(n0)
    st.E_cho = sla.cho_factor(st.E, lower=True)
    st.W = rng.standard_normal((p.n, nm))
    st.Vhat = sp.csc_matrix((p.n, nm))
    st.F = spd(nm)
    st.F_cho = sla.cho_factor(st.F, lower=True)
    return p, st, int(ref["pcg"]["iters"])


def oracle_sample(steps: int = 1, warmup: int = 0):
    """Times the CPU oracle's PCG (H_3,ad) on the benchmark problem at full
    size (_oracle_full_size_state): one run of its pcg with maxit = 3 and
    `steps` runs with maxit = 1 (one step each) give the time of one PCG
    iteration (half the difference) and of the start (initial residual and
    first apply); a solve is the start plus the oracle's own 30 iterations
    on this problem."""
    import oracle as O
    t0 = time.perf_counter()
    p, st, iters = _oracle_full_size_state()
    build_s = time.perf_counter() - t0

    def run(maxit):
        t = time.perf_counter()
        O.pcg(lambda v: st.A @ v, p.b, lambda r: O.H3_ad_apply(st, r), rtol=1e-300, maxit=maxit)
        return time.perf_counter() - t

    for _ in range(warmup):
        run(1)
    t3 = run(3)
    t1s = [run(1) for _ in range(steps)]
    t1 = statistics.median(t1s)
    t_it = max((t3 - t1) / 2.0, 0.0)
    t_start = t1 - t_it
    solve_s = t_start + iters * t_it
    return {"value": 1.0 / solve_s, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"oracle H3,ad PCG on the full 512x512 problem (n=262144, 256 subdomains, n0=3204, "
                       f"n_-=3092) with operators of the shapes of its setup there (random values; their "
                       f"setup, built in {build_s:.0f} s, is not timed): pcg with maxit 3 and 1 gives "
                       f"{t_it:.2f} s per iteration and {t_start:.2f} s to start; a solve = start + "
                       f"{iters} iterations (the oracle's count on this problem, stored)"),
            "s_per_iteration": t_it, "solve_s": solve_s, "step_s": t1}


def oracle_sample_one_thread():
    """The same oracle timing with one host thread: a child process with the
    BLAS thread counts set to 1 before numpy loads (solves/s, or None if the
    child fails)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; r = bench.oracle_sample(1); "
            "print(json.dumps({'value': r['value'], 's_per_iteration': r['s_per_iteration']}))")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             cwd=os.path.dirname(os.path.abspath(__file__)), timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except Exception:
        return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, args.steps)
    t0 = time.perf_counter()
    cb = oracle_sample(steps, warmup=min(args.warmup, 1))
    wall = time.perf_counter() - t0
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": min(args.warmup, 1),
            "ms_per_step": 1000.0 * cb["step_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "CPU oracle (NumPy/SciPy FP64)",
                       "step": "one oracle pcg run with maxit 1 and one with maxit 3 (4 PCG iterations "
                               "and 6 applies of H_3,ad at full size)"},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _pad(v, m):
    return (v + m - 1) // m * m


def block_bytes(info, K, prec):
    """Algorithmic bytes (minimum traffic) per launch of the block path's
    kernel classes for K columns, and per PCG iteration of H_3,ad (the sum
    over the launches of one iteration).  Operators are read once per pass
    (W with w bytes per element, the tensor-core images of the float32 local
    pseudo-inverses, the bfloat16 slices of E^-1 and F^-1, A, the Z and V_-
    arenas), block vectors once per pass in the type the kernel reads."""
    from paper_2106_10913_gb300 import FP64, MIXED_BF16, MIXED_FP16, MIXED_FP32
    n, nnz, n0, nm, S = info["n"], info["nnz"], info["n0"], info["n_minus"], info["sum_ns"]
    ldw = _pad(nm, 8)
    w = {FP64: 8, MIXED_FP32: 4, MIXED_BF16: 2, MIXED_FP16: 2}[prec]
    v = 8 if prec == FP64 else 4
    tc = prec in (MIXED_FP16, MIXED_BF16)
    ns = info["ns"]
    tiles = int(sum(((m + 127) // 128) * ((m + 31) // 32) for m in ns)) * 16384
    zb, vmb = info["z_entries"], info["vm_entries"]

    def oz(dim):  # one float64-accurate coarse product
        dimp, ldk = _pad(dim, 128), _pad(dim, 64)
        return (8 * dimp * ldk * 2                 # bfloat16 slices of the matrix
                + 2 * dim * K * 8                  # X read twice (column maxima, digits)
                + 8 * K * ldk * 2                  # X slices written
                + 2 * 8 * dimp * K * 16            # int64 partials written and read
                + dim * K * 8)                     # Y written
    per = {
        "spmv": (12 * nnz + 4 * (n + 1) + 16 * n * K                                  # q = A p (float64)
                 + 2 * (8 * nnz + 4 * (n + 1) + 3 * v * n * K + 4 * (n + 1) + 8 * S + vmb * v)) / 3.0,
        "local": tiles + 3 * S * K * 4 if (tc or prec == MIXED_FP32) else info["dense_total"] * 8 + 2 * S * K * 8,
        "wt": n * ldw * w + (2 * K * n * 2 if tc else n * K * v) + ldw * K * 4,
        "wd": n * ldw * w + (2 * K * ldw * 2 if tc else ldw * K * v) + n * K * 4,
        "coarse": (2 * oz(n0) + oz(nm)) / 3.0,
        "subdomain": (2 * (zb * v + S * K * v) + 2 * (vmb * v + S * K * v)) / 4.0,
        "prolong": (2 * (zb * v + 3 * n * K * v + 4 * (n + 1) + 8 * S) + (S * K * v + n * K * v)) / 3.0,
    }
    # PCG vectors per iteration (float64 r, x, p, q; float32 z and r copy):
    # x, r update (p, q, x, r read; x, r written; r32 written), r.z, p update
    vec_iter = n * K * (8 * 6 + 4) + n * K * (8 + 4) + n * K * (4 + 16)
    launches = {"spmv": 3, "local": 1, "wt": 1, "wd": 1, "coarse": 3, "subdomain": 4, "prolong": 3}
    iter_bytes = sum(per[k] * launches[k] for k in per) + vec_iter
    return per, iter_bytes


# DRAM bytes per launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) over the algorithmic bytes of the same launch, on
# the 320x320 channel case of the 64-column float16-W block solve
# (profiles/block64_local_w_dram_channels320.md); the traffic of a launch
# on another size is this ratio times its algorithmic bytes (the traffic of
# these streaming kernels grows in proportion to the operator they read)
DRAM_RATIO_K64_FP16 = {"local": 805319680 / 798215168, "wt": 251152640 / 247659520, "wd": 237962752 / 247659520}


def roofline_of(form, info):
    """Roofline of the dominant kernel class of a timed form (largest summed
    CUDA-event time in one extra solve with the apply's streams serialised):
    algorithmic bytes (or flops) per launch over the average event-timed
    launch, against the measured HBM copy bandwidth or,
    for the float64-accurate coarse products on the tensor cores, the
    measured sustained bfloat16 tensor rate (whichever bounds the launch's
    algorithmic work: its bfloat16 slice-product flops or its bytes).  For
    block forms also the whole iteration: the algorithmic bytes of one PCG
    iteration (every pass of block_bytes) over the measured time per
    iteration, against the HBM copy bandwidth."""
    from paper_2106_10913_gb300 import FP64, MIXED_BF16, MIXED_FP16, MIXED_FP32
    n, nm, nnz = info["n"], info["n_minus"], info["nnz"]
    n0, sum_ns, dense = info["n0"], info["sum_ns"], info["dense_total"]
    ldw = (nm + 7) // 8 * 8
    prec = form["prec"]
    w = {FP64: 8, MIXED_FP32: 4, MIXED_BF16: 2, MIXED_FP16: 2}[prec]
    g = 8 if prec == FP64 else 4
    sc = 4 if prec == MIXED_FP16 else 0
    prof = form["prof"]
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    bf16 = float(peaks.get("bf16_tflops_sustained", 1700.0))
    bf16_src = "measured (sustained)" if "bf16_tflops_sustained" in peaks else "fallback"
    names = {"wt": "k_umma_wt (tcgen05 W^T B)", "wd": "k_umma_wd (tcgen05 W D)",
             "local": "k_local_bimg + k_umma_local (tcgen05 TF32x3 local solves)",
             "coarse": "k_oz_colmax + k_oz_xslice + k_oz_gemm + k_oz_sum (float64-accurate E^-1, F^-1 "
                       "products, bfloat16 slices on tcgen05)",
             "spmv": "kb_spmv_dot (float64 q = A p) + kb_aplus (A_+ action)",
             "subdomain": "kb_tgemv + kb_tg_sum (Z^T X, V_-^T X)",
             "prolong": "kb_blk_prolong + kb_prolong"}
    cls = {}
    if not form["block"]:
        cls["wt"] = ("k_wt_partial (W^T r)", n * ldw * w + 8 * n + sc * n)
        cls["wd"] = ("k_w_d (W d)", n * ldw * w + 16 * n + 8 * nm + sc * n)
        cls["local"] = ("k_local_gemv (batched local pseudo-inverses)", dense * g + 16 * sum_ns)
        cls["spmv"] = ("k_spmv", 12 * nnz + 4 * (n + 1) + 16 * n)
        iter_bytes = None
    else:
        K = form["nrhs"]
        K = 16 if K <= 16 else (32 if K <= 32 else 64)
        per, iter_bytes = block_bytes(info, K, prec)
        for k, b in per.items():
            cls[k] = (names[k], b)
    cand = {k: prof["ms"][k] for k in cls if prof["count"][k] > 0}
    dom = max(cand, key=cand.get)
    name, units = cls[dom]
    per_launch_ms = prof["ms"][dom] / prof["count"][dom]
    out = {"kernel": name, "avg_launch_ms": per_launch_ms, "launches": prof["count"][dom],
           "kernel_share_of_solve": prof["ms"][dom] / prof["profiled_solve_ms"], "traffic": None,
           "timing": "CUDA events around each launch of one extra solve run with the apply's streams "
                     "serialised (AWG_PROF_SERIAL), after the timed steps"}
    if form["block"] and K == 64 and prec == MIXED_FP16 and dom in DRAM_RATIO_K64_FP16:
        out["traffic"] = DRAM_RATIO_K64_FP16[dom] * units
        out["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum on the 320x320 case, scaled "
                                 "by the algorithmic bytes of this launch")
    achieved = units / (per_launch_ms / 1000.0) / 1e9
    out.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "algorithmic_bytes_per_launch": units, "peak_source": f"{hbm_src} HBM copy bandwidth"})
    if dom == "coarse" and form["block"]:
        # bfloat16 slice products: 36 per product, 2 dim^2 K flops each
        flops = 36 * 2 * K * (2 * n0 * n0 + nm * nm) / 3.0
        t_tensor = flops / (bf16 * 1e12)
        t_hbm = units / (hbm * 1e9)
        if t_tensor > t_hbm:
            ach = flops / (per_launch_ms / 1000.0) / 1e12
            out.update({"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                        "algorithmic_flops_per_launch": flops,
                        "peak_source": f"{bf16_src} bfloat16 tensor rate"})
        out["hbm_frac"] = achieved / hbm
    if prec == FP64 and dom in ("wt", "wd", "local") and not form["block"]:
        out["note"] = "float64 form: one FMA per 8-byte element, bound by the float64 pipes"
    if iter_bytes is not None:
        ms_it = form["ms"] / form["steps"] / max(1, form["iters"])
        out["iteration"] = {"algorithmic_bytes": iter_bytes, "ms": ms_it,
                            "achieved_gbs": iter_bytes / (ms_it / 1000.0) / 1e9,
                            "frac": iter_bytes / (ms_it / 1000.0) / 1e9 / hbm,
                            "note": "one PCG iteration of the block solve (all passes of block_bytes) over the "
                                    "measured time per iteration of the timed form"}
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
                                        awg_pcg_block_async, awg_profile, awg_profile_read, PROF_COUNT,
                                        PROF_SERIAL)

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
    ns_arr = sol.array("ns").astype(np.int64)
    info["dense_total"] = int(np.sum(ns_arr ** 2))
    info["ns"] = ns_arr.tolist()
    info["z_entries"] = int(np.dot(ns_arr, sol.array("modes").astype(np.int64)))
    info["vm_entries"] = int(np.dot(ns_arr, sol.array("n_minus").astype(np.int64)))
    b1 = p.b if p.b.ndim == 1 else p.b[0]  # single-RHS forms: the first right-hand side
    b = torch.from_numpy(np.ascontiguousarray(b1)).cuda()
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
    if p.b.ndim == 2 and p.b.shape[0] >= Kmax:  # a workload with its own right-hand sides
        Ball = np.ascontiguousarray(p.b[:Kmax])
    else:
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
        awg_profile(sol.h, PROF_COUNT)  # the timed steps: launches counted, no events
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
        launches = awg_profile_read(sol.h)["launches"]
        awg_profile(sol.h, 0)
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
        # one more solve, untimed, with every kernel class bracketed by CUDA
        # events and the apply's two streams serialised, so that the event
        # times are kernel times (the kernel breakdown and the roofline)
        awg_profile(sol.h, timed_mask | PROF_SERIAL)
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        solve()
        pe1.record(stream)
        torch.cuda.synchronize()
        prof = awg_profile_read(sol.h)
        awg_profile(sol.h, 0)
        prof["profiled_solve_ms"] = pe0.elapsed_time(pe1)
        prof["launches"] = launches
        if not its:  # graph-driven solves: device results of the last step
            its = [int(g_its[:K].max().item())]
            rels = [float(g_rel[:K].max().item())]
            sts = [int(g_st.item())]
            cols = {c: int(g_its[c].item()) for c in (0, 1, 77, 127) if c < K}
        # every solver reports the TRUE relative residual of the columns it
        # stopped as converged (the graph-driven loop confirms the recurrence
        # residual on b - A x inside the graph)
        ok = all(s == 0 for s in sts) and max(rels) <= RTOL
        forms[name] = {"prec": prec, "block": block, "graph": graph, "nrhs": per_step, "ms": ms, "steps": args.steps,
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
    hb = torch.from_numpy(np.ascontiguousarray(Ball[:best["nrhs"]]) if best["block"] else b1).pin_memory()
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
        cb1 = oracle_sample_one_thread() if cb else None
        line = {
            "metric": METRIC, "value": best["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {FP64: "f64", MIXED_FP32: "f32+f64", MIXED_BF16: "bf16+f32+f64",
                      MIXED_FP16: "f16+f32+f64"}[best["prec"]],
            "data": "synthetic",
            "config": {"workload": _workload(args.config, p) + (f"; batched form: {best['nrhs']} right-hand sides per block "
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
                          "kernel_ms_profiled_solve": {c: round(t, 3) for c, t in v["prof"]["ms"].items()},
                          "profiled_solve_ms": round(v["prof"]["profiled_solve_ms"], 3),
                          "launches": v["prof"]["launches"]} for k, v in forms.items()},
            "speedup_vs_plain_fp64": (best["value"] / forms["fp64"]["value"]) if "fp64" in forms else None,
            "batched_problems": batch,
            "roofline": roofline,
            "cpu_baseline": ({**{k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                              "one_thread": cb1} if cb else None),
            "e2e": e2e,
            "gpu_launches": int(best["prof"]["launches"]),
            "clocks": best["clocks"],
            # per kernel class, CUDA-event time of one serialised solve of the
            # roofline's form (kernels inside graph loops carry no events)
            "kernel_ms": {k: round(v, 3) for k, v in rform["prof"]["ms"].items()},
            "kernel_ms_form": [k for k, v in forms.items() if v is rform][0],
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


def learned_start_eval(train_seeds=range(1000, 1200), test_seeds=range(2000, 2020), nex=96, steps=400, lr=1e-2):
    """The learned start on the elasticity workload's generator: the network
    is trained on the device on the eigenpairs that the setup itself finds
    for 200 seeded coefficient draws (layer thicknesses from seeds
    1000-1199; 96 x 96 elements in 4 x 4 node boxes, the subdomain size of
    the 384 x 384 workload), then the GenEO block eigensolver runs on 20
    held-out draws (seeds 2000-2019) from the learned start and from the
    random start.  Reported: summed and largest solver steps, subdomains
    sent to the dense eigensolver and GenEO stage time, per start, and
    whether the mode counts agree (they must: both are certified)."""
    import torch
    import awg_inputs as gi
    from paper_2106_10913_gb300 import (AWGSolver, LEARNED_NFEAT, MIXED_FP32, awg_learned_data,
                                        awg_learned_train)
    q = nex // 24
    t0 = time.perf_counter()
    Fs, ts = [], []
    for sd in train_seeds:
        pr = gi.config4(nex, nrhs=1, seed=sd, q=q)
        sol = AWGSolver(pr.rowptr, pr.colidx, pr.val, pr.part, pr.nparts, pr.overlap, pr.tau, geneo_solver=1)
        S = sol.info["sum_ns"]
        F = torch.zeros((S, LEARNED_NFEAT), dtype=torch.float64, device="cuda")
        t = torch.zeros(S, dtype=torch.float64, device="cuda")
        awg_learned_data(sol.h, F, t)
        torch.cuda.synchronize()
        sol.close()
        Fs.append(F)
        ts.append(t)
    data_s = time.perf_counter() - t0
    F, t = torch.cat(Fs), torch.cat(ts)
    rng = np.random.default_rng(0)
    th0 = np.zeros(385)
    o = 0
    for fo, fi in ((16, 5), (16, 16), (1, 16)):
        lim = np.sqrt(6.0 / (fi + fo))
        th0[o:o + fo * fi] = rng.uniform(-lim, lim, fo * fi)
        o += fo * fi + fo
    t1 = time.perf_counter()
    th, loss = awg_learned_train(F, t, th0, steps, lr, precision=MIXED_FP32)
    train_s = time.perf_counter() - t1
    res = {"random": {"steps_sum": 0, "steps_max": 0, "dense": 0, "geneo_ms": 0.0},
           "learned": {"steps_sum": 0, "steps_max": 0, "dense": 0, "geneo_ms": 0.0}}
    counts_agree = True
    for sd in test_seeds:
        pr = gi.config4(nex, nrhs=1, seed=sd, q=q)
        modes = {}
        for name, opts in (("random", {"geneo_solver": 1}), ("learned", {"geneo_solver": 2, "learned_params": th})):
            sol = AWGSolver(pr.rowptr, pr.colidx, pr.val, pr.part, pr.nparts, pr.overlap, pr.tau, **opts)
            r = res[name]
            r["steps_sum"] += int(sol.info["geneo_its_sum"])
            r["steps_max"] = max(r["steps_max"], int(sol.info["geneo_its_max"]))
            r["dense"] += int(sol.info["geneo_dense"])
            r["geneo_ms"] += float(sol.info["setup_ms"][3])
            modes[name] = sol.array("modes").tolist()
            sol.close()
        counts_agree &= modes["random"] == modes["learned"]
    return {"train": {"draws": len(list(train_seeds)), "samples": int(F.shape[0]), "adam_steps": steps,
                      "loss_first": float(loss[0]), "loss_last": float(loss[-1]), "data_s": round(data_s, 1),
                      "train_s": round(train_s, 2)},
            "held_out_draws": len(list(test_seeds)), "mode_counts_agree": bool(counts_agree), **res}


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
    ap.add_argument("--learned-eval", action="store_true",
                    help="only the learned-start evaluation on the elasticity generator (one JSON line)")
    args = ap.parse_args()
    if args.learned_eval:
        print(json.dumps({"learned_start_eval": learned_start_eval()}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_awg(args)


if __name__ == "__main__":
    main()
