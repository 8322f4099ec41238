"""Benchmark of the sketched Tucker core update on GB300 (one JSON line).

A step is one sketched core update (leverage scores -> product-distribution
sampling -> dedupe -> gather and weights -> Kronecker Gram / right-hand side ->
ridge solve) on the 3-way dense workload 512 x 512 x 512 FP32, Tucker rank
(8,8,8) (core dimension d = 512), sigma = 0.05, lambda = 1e-2, m = 50,000
sampled rows.  The exact core update (TTM chain + factor eigendecompositions)
on the same inputs is timed beside it, and the ridge-loss ratio of the two
cores is reported.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16|tf32|fp32|fp64]
    python bench.py --impl reference ...   # the CPU oracle, timed on host cores

Timing: CUDA events on the library's stream around each call, L2 flushed
(256 MiB write) before every timed step; W untimed warm-up steps; barrier +
synchronize around the timed region; max over ranks.  Multi-GPU runs are
independent replicas (the update has no data-path collective).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "core-update ms, sketched vs exact, 1 GB300 at <=1.01x ridge loss; Kron rows/s"
WORKLOAD = "dense3_512_r8_f32"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP64 CUDA-core peak: 1.25 TFLOP/s (the GB300 nominal FP64 rate).
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e-3
# tcgen05 dense peak relative to BF16: TF32 runs at half the BF16 rate.
TC_RATIO = {"bf16": 1.0, "tf32": 0.5}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--prec", default="auto")
    p.add_argument("--reg", default="exact")
    p.add_argument("--solver", default="kpcg", choices=["fp64", "mixed", "kpcg"],
                   help="ridge solver of the timed update (the others are timed beside it)")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the 128^4 and 1024^3-at-10% workloads timed beside the headline")
    p.add_argument("--m-ladder", action="store_true",
                   help="the smallest m on a x2 ladder from the workload's m whose median ridge-loss "
                        "ratio over 10 seeds is <= 1.01 (with --impl reference: by the oracle on "
                        "the host); prints its own JSON line, not the headline")
    p.add_argument("--kernel-case", choices=["grouped", "walk2", "headline"], default=None,
                   help="a small case of one kernel family for ncu captures (grouped: the "
                        "1024^3 Gram shapes, I_1 = 1024, d = 4096, m = 5e5, on a dense "
                        "1024 x 128 x 128 tensor; walk2: the 128^4 two-level walks at "
                        "m = 8e5; headline: three sketched updates of the 512^3 workload at "
                        "m = 1e5 and three exact ones, nothing else); prints its own JSON "
                        "line, not the headline")
    p.add_argument("--stage-roofline", action="store_true",
                   help="time the sampler and the gather at 2^27 draws (their HBM/ALU rooflines); "
                        "prints its own JSON line, not the headline")
    return p.parse_args()


def load_traffic():
    """DRAM bytes per launch of a kernel on a workload, from the committed ncu summaries."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        tab = json.load(f)
    return {(e["kernel"], e["workload"]): e["dram_bytes_per_launch"] for e in tab.get("entries", [])}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 0) for i in threadpool_info()), default=0)
        if n:
            return n
    except Exception:
        pass
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return len(os.sched_getaffinity(0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix=f"clocks_gpu{self.gpu}_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=self.f,
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
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_timing(w, Xh, F, reg, budget=12.0):
    """Milliseconds of one oracle sketched core update on the host cores.

    Small workloads run whole updates (up to 5 within the budget).  Large ones
    (d > 1024 or observed entries) run the sampling in full, the normal
    equations over a prefix of the sampled rows scaled linearly to all rows
    (their cost is linear in the rows), and the full d x d Cholesky solve."""
    import numpy as np
    from oracle import core_update as CU, sampling as S
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    missing = isinstance(Xh, dict)
    if not missing and w.d <= 1024:
        times = []
        t_start = time.perf_counter()
        while not times or (time.perf_counter() - t_start) < budget and len(times) < 5:
            t0 = time.perf_counter()
            oracle_step(Xh, F, w, reg)
            times.append((time.perf_counter() - t0) * 1e3)
        return statistics.mean(times), (f"{len(times)} full sketched core updates of the same "
                                        f"workload (numpy FP64 oracle, m = {w.m})")
    dims = tuple(Xh["dims"]) if missing else tuple(Xh.shape)
    t0 = time.perf_counter()
    sk = CU.sketch(F, dims, w.m, w.seed_sample, 0, regc, Xh["keys"] if missing else None)
    x = (CU.gather_observed(Xh["keys"], Xh["vals"], sk["keys"]) if missing
         else CU.gather_dense(Xh, sk["keys"], dims))
    t_sample = time.perf_counter() - t0
    n = sk["keys"].size
    n_sub = min(n, 4096)
    while True:
        t0 = time.perf_counter()
        G, hv, D = CU.sketched_normal_equations(F, dims, sk["keys"][:n_sub], sk["w"][:n_sub],
                                                x[:n_sub])
        t_ne = time.perf_counter() - t0
        if n_sub >= n or 2 * t_ne > budget / 2 or n_sub >= 1 << 16:
            break
        n_sub = min(n, 2 * n_sub)
    t0 = time.perf_counter()
    CU.cholesky_solve(CU.regularised_matrix(G, D, w.lam, regc), hv)
    t_solve = time.perf_counter() - t0
    total = t_sample + t_ne * n / n_sub + t_solve
    return total * 1e3, (f"numpy FP64 oracle: leverage, sampling of all {w.m} rows (T = {sk['T']}) "
                         f"and the d = {w.d} Cholesky solve in full; normal equations timed on "
                         f"{n_sub} of the {n} sampled rows and scaled to all rows")


def oracle_exact_timing(w, Xh, F):
    """(ms, description) of one exact core update by the oracle on the host cores
    (dense: the n-mode product chain and the factor eigendecompositions); the
    exact observed-entry update, the Gram of every observed row, is not run."""
    if isinstance(Xh, dict):
        return None, ("not run: the exact observed-entry update is the Gram of all observed "
                      "rows, |Omega| d (d + 1) flop (1.8e15 at 1024^3 with d = 4096), hours "
                      "on the host")
    from oracle import core_update as CU
    t0 = time.perf_counter()
    CU.exact_core_kron_eig(Xh, F, w.lam)
    return (time.perf_counter() - t0) * 1e3, "one exact core update (numpy FP64 oracle)"


def oracle_step(X, F, w, reg):
    from oracle import core_update as CU, sampling as S
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    return CU.sketched_core(X, F, w.lam, w.m, w.seed_sample, 0, regc)


def oracle_ladder(w, X, F, reg):
    """The x2 ladder of the headline computed by the oracle on the host (the
    library draws the same rows and its cores agree to 1e-6, so the ratios and
    m_star are the GPU arm's too)."""
    import numpy as np
    from oracle import core_update as CU, sampling as S
    regc = S.REG_EXACT if reg == "exact" else S.REG_AUGMENTED
    X = np.asarray(X, dtype=np.float64)
    F = [np.asarray(a, dtype=np.float64) for a in F]
    ktx = CU.kt_x(X, F)
    xx = float(np.sum(X * X))
    opt = CU.ridge_loss_dense(X, F, CU.exact_core_kron_eig(X, F, w.lam, ktx), w.lam, xx, ktx)

    def ratio_of(m, s):
        g = CU.sketched_core(X, F, w.lam, m, w.seed_sample + s, 0, regc)["g"]
        return CU.ridge_loss_dense(X, F, g, w.lam, xx, ktx) / opt
    return _ladder(ratio_of, w.m)


def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only), on the GPU arm's
    workload, m and configuration."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    w = synth.WORKLOADS[args.workload]
    if w.observed < 1.0:
        X = synth.observed_entries(w)
        F = X["factors"]
        x_bytes = X["keys"].nbytes + X["vals"].nbytes
    else:
        P = synth.tucker_problem(w)
        X, F = P["X"], P["factors"]
        x_bytes = X.nbytes
    small = w.observed >= 1.0 and w.d <= 1024
    ladder, m_star = (oracle_ladder(w, X, F, args.reg) if small else ([], None))
    wm = dataclasses.replace(w, m=m_star or w.m)
    for _ in range(max(0, min(args.warmup, 1))):
        if small:
            oracle_step(X, F, wm, args.reg)
    times, sample = [], ""
    for _ in range(args.steps):
        if small:
            t0 = time.perf_counter()
            oracle_step(X, F, wm, args.reg)
            times.append((time.perf_counter() - t0) * 1e3)
            sample = (f"{args.steps} full sketched core updates of the workload at m = {wm.m} "
                      "(numpy FP64 oracle)")
        else:
            ms_est, sample = oracle_timing(wm, X, F, args.reg, budget=6.0)
            times.append(ms_est)
    ms = statistics.mean(times)
    cores = cpu_cores()
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            # the same workload configuration as the GPU arm; the oracle itself computes
            # in FP64 (explicit sampled rows, FP64 Cholesky)
            "config": workload_config(w, ours_prec(args), args.reg, args.solver, wm.m, x_bytes),
            "oracle_arithmetic": "fp64",
            "m_ladder": {"target": LADDER_TARGET, "seeds": LADDER_SEEDS, "rows": ladder,
                         "m_star": m_star},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "oracle_exact": dict(zip(("ms", "sample"), oracle_exact_timing(wm, X, F))),
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over the process group (the
    slowest replica sets the job's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def grouped_gram(w):
    """Whether the library groups the tensor-core Gram by the leading index (the
    same test as the library's: order >= 3, R_1 a power of two <= 16, d / R_1 >= 128,
    at most 8192 (segment, tile) pairs, A^(1) within 200 KB as FP32)."""
    R1, N = w.ranks[0], len(w.ranks)
    if N < 3 or R1 > 16 or R1 & (R1 - 1) or w.d % R1:
        return False
    dp = w.d // R1
    tiles = (dp + 255) // 256
    I1 = w.dims[0]
    return dp >= 128 and I1 * tiles * (tiles + 1) // 2 <= 8192 and I1 * R1 * 4 <= 200 * 1024


def narrow_gram(w, m):
    """Whether the library forms the narrow grouped Gram (the library's test: order
    >= 3, R_1 in {2, 4, 8, 16}, d / R_1 <= 64, m >= 2 I_1, A^(1) within 96 KB as FP32)."""
    R1, N = w.ranks[0], len(w.ranks)
    if N < 3 or R1 < 2 or R1 > 16 or R1 & (R1 - 1) or w.d % R1:
        return False
    I1 = w.dims[0]
    return w.d // R1 <= 64 and m >= 2 * I1 and I1 * R1 * 4 <= 96 * 1024


def ours_prec(args):
    """Gram precision of the GPU arm (the same choice main() makes)."""
    prec = args.prec
    if prec == "auto":
        prec = os.environ.get("TUCKER_BENCH_PREC", "tf32")
    return prec


def workload_config(w, prec, reg, solver, m, x_bytes):
    """The workload a line is measured on; m is the sample count it is timed at
    (the smallest m on the ladder whose median ridge-loss ratio meets 1.01x)."""
    return {"workload": w.name, "solver": solver, "dims": list(w.dims), "ranks": list(w.ranks),
            "d": w.d, "m": m, "m_workload": w.m, "lambda": w.lam, "sigma": w.sigma,
            "x_dtype": w.dtype, "observed": w.observed, "gram_prec": prec, "reg": reg,
            "seed": w.seed_sample,
            "l2": f"flushed before every timed step (256 MiB write); X is {x_bytes / 2**20:.0f} MiB"}


def run_kernel_case(args):
    """Three sketched TF32 updates of a small case of one kernel family, so that one
    launch can be captured with every ncu section:
      grouped: the Gram grouped by the leading index at the 1024^3-at-10% shapes
        (I_1 = 1024, ranks 16, d = 4096, m = 5e5) on a dense 1024 x 128 x 128 FP32
        tensor (under 1 GB on the device);
      walk2: the two-level walks of the 128^4 workload's FP64 residual and right-hand
        side (ranks 8^4, m = 8e5) on a dense 128^4 FP32 tensor (1 GiB)."""
    import numpy as np
    import torch
    import synth
    from paper_2107_10654_gb300 import tucker as T
    if args.kernel_case == "headline":
        # the timed workload's kernels alone: its sample count at the 1.01 ladder (m* = 1e5)
        w = synth.WORKLOADS[WORKLOAD]
        P = synth.tucker_problem(w)
        X = torch.from_numpy(P["X"]).cuda()
        F = [torch.from_numpy(a).cuda() for a in P["factors"]]
        h = T.Handle(solver=args.solver)
        ms, ex = [], []
        for _ in range(3):
            st = T.tucker_core_update_sketched(h, X, F, w.lam, 100000, w.seed_sample, 0, "exact",
                                               "tf32", stats=True)[1]
            ms.append(st["ms_total"])
        for _ in range(3):
            T.tucker_core_update_exact(h, X, F, w.lam, "fp64")
        torch.cuda.synchronize()
        print(json.dumps({"mode": "kernel_case", "case": "headline", "workload": w.name,
                          "m": 100000, "ms": ms}))
        h.close()
        return
    g = synth.rng(4321)
    if args.kernel_case == "walk2":
        dims, ranks, m = (128, 128, 128, 128), (8, 8, 8, 8), 800000
    else:
        dims, ranks, m = (1024, 128, 128), (16, 16, 16), 500000
    F = [torch.from_numpy(g.standard_normal((i, r)).astype(np.float32)).cuda()
         for i, r in zip(dims, ranks)]
    X = torch.from_numpy(g.standard_normal(dims).astype(np.float32)).cuda()
    h = T.Handle(solver=args.solver)
    sts = [T.tucker_core_update_sketched(h, X, F, 0.1, m, 7, 0, "exact", "tf32", stats=True)[1]
           for _ in range(3)]
    print(json.dumps({"mode": "kernel_case", "case": args.kernel_case, "dims": dims,
                      "ranks": ranks, "m": m,
                      "ms": [s["ms_total"] for s in sts],
                      "ms_gram": [s["ms_gram"] for s in sts],
                      "ms_gram_kernel": [s["ms_gram_kernel"] for s in sts]}))
    h.close()


def run_stage_roofline(args):
    """Sampler and gather at 2^27 draws from the 512^3 tensor, whose per-stage
    times at the workload's m are launch-bound.  Rank-(2,2,2) factors keep the
    Gram and the solve negligible; the stages are timed by the library's events."""
    import numpy as np
    import torch
    import synth
    from paper_2107_10654_gb300 import tucker as T
    w = synth.WORKLOADS["dense3_512_r8_f32"]
    P = synth.tucker_problem(w)
    g = synth.rng(w.seed_data + 5)
    F = [torch.from_numpy(g.standard_normal((i, 2)).astype(np.float32)).cuda() for i in w.dims]
    X = torch.from_numpy(P["X"]).cuda()
    m = 1 << 27
    h = T.Handle()
    T.tucker_core_update_sketched(h, X, F, w.lam, m, w.seed_sample, 0, "exact", "bf16")
    sts = [T.tucker_core_update_sketched(h, X, F, w.lam, m, w.seed_sample, 0, "exact", "bf16",
                                         stats=True)[1] for _ in range(3)]
    pk, src = peaks()
    ms_s = statistics.mean(s["ms_sample"] for s in sts)
    ms_g = statistics.mean(s["ms_gather"] for s in sts)
    n_u = sts[-1]["n_unique"]
    # sampler: 8 B key written per draw (CDFs are read once into shared memory)
    samp_gbs = 8.0 * m / (ms_s * 1e-3) / 1e9
    # gather, per unique row: key 8 + count 4 + x 4 read, three u32 indices + w, x, p (FP64)
    # + sqrt(w) (FP32) written = 56 B; the x read costs a 32 B sector (84 B with sectors)
    gath_alg = 56.0 * n_u / (ms_g * 1e-3) / 1e9
    gath_sec = 84.0 * n_u / (ms_g * 1e-3) / 1e9
    line = {"mode": "stage_roofline", "draws": m, "n_unique": n_u, "workload": "512^3 X, rank (2,2,2)",
            "sampler": {"ms": ms_s, "bytes_per_draw": 8, "achieved_gbs": samp_gbs,
                        "frac_of_hbm": samp_gbs / pk["hbm_gbs"]},
            "gather": {"ms": ms_g, "bytes_per_row": 56, "achieved_gbs": gath_alg,
                       "frac_of_hbm": gath_alg / pk["hbm_gbs"], "with_32B_sector_gbs": gath_sec,
                       "frac_with_sectors": gath_sec / pk["hbm_gbs"]},
            "peak_hbm_gbs": pk["hbm_gbs"], "peak_source": src,
            "stage_ms": {k: statistics.mean(s[k] for s in sts) for k in
                         ("ms_leverage", "ms_sample", "ms_dedupe", "ms_gather", "ms_gram", "ms_solve")}}
    print(json.dumps(line), flush=True)
    h.close()


LADDER_SEEDS = 10
LADDER_STEPS = 4          # m, 2m, 4m, 8m, 16m at most
LADDER_TARGET = 1.01


def _ladder(ratio_of, m0):
    """Median (and max) ridge-loss ratio over LADDER_SEEDS seeds at m0 * 2^k,
    k = 0, 1, ... until the median meets LADDER_TARGET."""
    rows = []
    m = m0
    for _ in range(LADDER_STEPS + 1):
        r = [ratio_of(m, s) for s in range(LADDER_SEEDS)]
        rows.append({"m": m, "median_ratio": statistics.median(r), "max_ratio": max(r)})
        if rows[-1]["median_ratio"] <= LADDER_TARGET:
            break
        m *= 2
    m_star = rows[-1]["m"] if rows[-1]["median_ratio"] <= LADDER_TARGET else None
    return rows, m_star


def run_m_ladder(args):
    """The sample count the 1.01x loss target needs on this workload: a x2 ladder
    from the workload's m, 10 sampling seeds per step.  The sampled rows are
    bit-identical between the library and the oracle and the cores agree to
    1e-6, so either side gives the same ratios; the GPU arm also times the
    update at the workload's m and at the m found."""
    import numpy as np
    import synth
    w = synth.WORKLOADS[args.workload]
    missing = w.observed < 1.0
    seeds = [w.seed_sample + s for s in range(LADDER_SEEDS)]
    line = {"mode": "m_ladder", "impl": args.impl, "workload": w.name, "target": LADDER_TARGET,
            "seeds": LADDER_SEEDS, "reg": args.reg}
    if args.impl == "reference":
        from oracle import core_update as CU, sampling as S
        if missing:
            print(json.dumps(dict(line, unavailable="the oracle's loss over 1.07e8 observed "
                                  "entries takes hours; the GPU arm computes this ladder")))
            return
        regc = S.REG_EXACT if args.reg == "exact" else S.REG_AUGMENTED
        P = synth.tucker_problem(w)
        X = np.asarray(P["X"], dtype=np.float64)
        F = [np.asarray(a, dtype=np.float64) for a in P["factors"]]
        ktx = CU.kt_x(X, F)
        xx = float(np.sum(X * X))
        opt = CU.ridge_loss_dense(X, F, CU.exact_core_kron_eig(X, F, w.lam, ktx), w.lam, xx, ktx)

        def ratio_of(m, s):
            g = CU.sketched_core(X, F, w.lam, m, seeds[s], 0, regc)["g"]
            return CU.ridge_loss_dense(X, F, g, w.lam, xx, ktx) / opt
        t0 = time.perf_counter()
        rows, m_star = _ladder(ratio_of, w.m)
        line.update({"ladder": rows, "m_star": m_star, "oracle_s": time.perf_counter() - t0,
                     "cores": cpu_cores()})
        print(json.dumps(line), flush=True)
        return
    import torch
    from paper_2107_10654_gb300 import tucker as T
    prec = ours_prec(args)
    dev = torch.device("cuda", 0)
    if missing:
        O = synth.observed_entries(w)
        X = T.CooTensor(torch.from_numpy(O["keys"].view(np.int64)).to(dev),
                        torch.from_numpy(O["vals"]).to(dev), w.dims)
        F = [torch.from_numpy(a).to(dev) for a in O["factors"]]
    else:
        P = synth.tucker_problem(w)
        X = torch.from_numpy(P["X"]).to(dev)
        F = [torch.from_numpy(a).to(dev) for a in P["factors"]]
    h = T.Handle(solver=args.solver)
    exact_prec = "bf16" if missing else "fp64"
    opt = T.tucker_ridge_loss(h, X, F, w.lam, T.tucker_core_update_exact(h, X, F, w.lam, exact_prec))

    def ratio_of(m, s):
        g = T.tucker_core_update_sketched(h, X, F, w.lam, m, seeds[s], 0, args.reg, prec)
        return T.tucker_ridge_loss(h, X, F, w.lam, g) / opt

    def ms_at(m):
        for _ in range(3):
            T.tucker_core_update_sketched(h, X, F, w.lam, m, seeds[0], 0, args.reg, prec)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(h.stream)
        for _ in range(5):
            T.tucker_core_update_sketched(h, X, F, w.lam, m, seeds[0], 0, args.reg, prec)
        ev[1].record(h.stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 5

    rows, m_star = _ladder(ratio_of, w.m)
    line.update({"ladder": rows, "m_star": m_star, "gram_prec": prec, "solver": args.solver,
                 "ms_at_m": ms_at(w.m), "ms_at_m_star": ms_at(m_star) if m_star else None})
    print(json.dumps(line), flush=True)
    h.close()


def gpu_inputs(w, dev, pinned=False):
    """(X on the device, factors on the device, host copies, input bytes) of a workload."""
    import numpy as np
    import torch
    import synth
    from paper_2107_10654_gb300 import tucker as T
    if w.observed < 1.0:
        O = synth.observed_entries(w)
        host_in = [torch.from_numpy(O["keys"].view(np.int64)), torch.from_numpy(O["vals"])]
        F_h, X_h = O["factors"], O
    else:
        P = synth.tucker_problem(w)
        X_h, F_h = P["X"], P["factors"]
        host_in = [torch.from_numpy(X_h)]
    if pinned:
        host_in = [t.pin_memory() for t in host_in]
    F_pin = [torch.from_numpy(a) for a in F_h]
    if pinned:
        F_pin = [a.pin_memory() for a in F_pin]
    dev_in = [t.to(dev) for t in host_in]
    F = [a.to(dev) for a in F_pin]
    X = T.CooTensor(dev_in[0], dev_in[1], w.dims) if w.observed < 1.0 else dev_in[0]
    in_bytes = sum(t.numel() * t.element_size() for t in host_in)
    return X, F, {"X_h": X_h, "F_h": F_h, "host_in": host_in, "F_pin": F_pin, "dev_in": dev_in}, in_bytes


class Timer:
    """CUDA events on the library's stream around each step, L2 flushed before each."""

    def __init__(self, stream, flush):
        self.stream, self.flush = stream, flush

    def __call__(self, fn, k):
        import torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        out = []
        for i in range(k):
            self.flush.fill_(float(i))
            ev[i][0].record(self.stream)
            out.append(fn())
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], out


STAGES = ("ms_leverage", "ms_sample", "ms_dedupe", "ms_gather", "ms_gram", "ms_solve")
RIDGE_LAMBDA = 1e8
# fiber draws of each sketched factor update in the ALS sweeps the benchmark times
FACTOR_M = 16384


def ridge_alg1_count(d, d_eff, eps=0.1, delta=0.1):
    """Alg. 1 line 3's s: with the exact ridge scores (d_eff given) beta' =
    d / (d_eff + d min{1, d - d_eff}) (Eq. beta_prime); classical scores
    (d_eff None) beta' = 1/2."""
    bp = 0.5 if d_eff is None else d / (d_eff + d * min(1.0, d - d_eff))
    return math.ceil(4.0 * d / bp * max(420.0 * math.log(4.0 * d / delta), 1.0 / (delta * eps)))


def measure_workload(h, w, X, F, prec, reg, steps, warmup, timer, m_override=None):
    """The sketched core update of one workload on the GPU: the sample count the
    1.01x ridge-loss target needs (median over LADDER_SEEDS sampling seeds on a x2
    ladder from the workload's m), the update timed at that m (asynchronous calls,
    no per-stage events) and at the workload's own m, the stage split, the exact
    update (the plain method) and the loss ratios."""
    import torch
    from paper_2107_10654_gb300 import tucker as T
    missing = w.observed < 1.0
    exact_prec = prec if missing else "fp64"
    g_ex = T.tucker_core_update_exact(h, X, F, w.lam, exact_prec)
    loss_ex = T.tucker_ridge_loss(h, X, F, w.lam, g_ex)
    seeds = [w.seed_sample + s for s in range(LADDER_SEEDS)]

    def ratio_of(m, s):
        g = T.tucker_core_update_sketched(h, X, F, w.lam, m, seeds[s], 0, reg, prec)
        return T.tucker_ridge_loss(h, X, F, w.lam, g) / loss_ex
    ladder, m_star = _ladder(ratio_of, w.m)
    m_t = m_override or m_star or ladder[-1]["m"]
    g = torch.empty(w.d, dtype=torch.float64, device=F[0].device)

    def upd(m, stats):
        return T.tucker_core_update_sketched(h, X, F, w.lam, m, w.seed_sample, 0, reg, prec,
                                             core_out=g, stats=stats)
    out = {"m": w.m, "m_star": m_star, "m_timed": m_t, "ladder": ladder}
    for m, key in ((m_t, "at_m_star"), (w.m, "at_workload_m")):
        if key == "at_workload_m" and m == m_t:
            out[key] = out["at_m_star"]
            continue
        _, st0 = upd(m, True)
        loss = T.tucker_ridge_loss(h, X, F, w.lam, g) / loss_ex
        for _ in range(warmup):
            upd(m, False)
        torch.cuda.synchronize()
        h.set_sync(False)
        ms, _ = timer(lambda: upd(m, False), steps)
        h.sync()
        h.set_sync(True)
        _, sts = timer(lambda: upd(m, True), steps)
        stats = [s for _, s in sts]
        rec = {"ms": statistics.mean(ms), "ms_min": min(ms), "loss_ratio": loss,
               "stage_ms": {k: statistics.mean(s[k] for s in stats) for k in STAGES},
               "ms_with_stage_events": statistics.mean(sum(s[k] for k in STAGES) for s in stats),
               "n_unique": stats[-1]["n_unique"], "n_real": stats[-1]["n_real"],
               "n_draws": stats[-1]["n_draws"], "refine_iters": stats[-1]["refine_iters"],
               "inner_iters": stats[-1]["inner_iters"],
               "kernel_ms": {"gram": statistics.mean(s["ms_gram_kernel"] for s in stats),
                             "factor_or_convert": statistics.mean(s["ms_factor"] for s in stats),
                             "first_cg_solve": statistics.mean(s["ms_inner"] for s in stats)},
               "launches": int(statistics.mean(s["launches"] for s in stats)),
               "raw_steps_ms": ms}
        out[key] = rec
    n_ex = steps if not missing else min(steps, 3)
    h.set_sync(False)
    ex_ms, _ = timer(lambda: T.tucker_core_update_exact(h, X, F, w.lam, exact_prec, core_out=g_ex),
                     n_ex)
    h.sync()
    h.set_sync(True)
    out["exact_ms"] = statistics.mean(ex_ms)
    out["exact_prec"] = exact_prec
    out["speedup_vs_exact"] = out["exact_ms"] / out["at_m_star"]["ms"]
    out["speedup_vs_exact_at_workload_m"] = out["exact_ms"] / out["at_workload_m"]["ms"]
    return out


def main():
    args = parse()
    if args.m_ladder:
        run_m_ladder(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.stage_roofline:
        run_stage_roofline(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_2107_10654_gb300 import tucker as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    w = synth.WORKLOADS[args.workload]
    prec = ours_prec(args)
    missing = w.observed < 1.0
    X, F, hb, in_bytes = gpu_inputs(w, dev, pinned=True)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MiB > L2

    h = T.Handle(solver=args.solver)
    stream = h.stream
    timer = Timer(stream, flush)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        head = measure_workload(h, w, X, F, prec, args.reg, args.steps, args.warmup, timer)
        m_t = head["m_timed"]
        # end to end through the public API: host (pinned) inputs in, core out to host;
        # two alternating device buffers, so nothing (the observed-entry hash) carries over
        core_host = torch.empty(w.d, dtype=torch.float64).pin_memory()
        bufs = [[torch.empty_like(t) for t in hb["dev_in"]] for _ in range(2)]
        Fe = [torch.empty_like(a) for a in F]
        e2e_ms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                for a, b in zip(bufs[i % 2], hb["host_in"]):
                    a.copy_(b, non_blocking=True)
                for a, b in zip(Fe, hb["F_pin"]):
                    a.copy_(b, non_blocking=True)
            Xe = T.CooTensor(bufs[i % 2][0], bufs[i % 2][1], w.dims) if missing else bufs[i % 2][0]
            g = T.tucker_core_update_sketched(h, Xe, Fe, w.lam, m_t, w.seed_sample, 0, args.reg,
                                              prec)
            with torch.cuda.stream(stream):
                core_host.copy_(g, non_blocking=True)
            stream.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del bufs
        # the other ridge solvers on the same workload and m, timed the same way
        others = {}
        for other in ("mixed", "fp64", "kpcg"):
            if other == args.solver:
                continue
            h2 = T.Handle(stream=stream, solver=other)
            g_alt = torch.empty(w.d, dtype=torch.float64, device=dev)

            def alt(stats=False):
                return T.tucker_core_update_sketched(h2, X, F, w.lam, m_t, w.seed_sample, 0,
                                                     args.reg, prec, core_out=g_alt, stats=stats)
            for _ in range(args.warmup):
                alt()
            h2.set_sync(False)
            k = min(args.steps, 10)
            alt_ms, _ = timer(alt, k)
            h2.sync()
            h2.set_sync(True)
            _, st = alt(True)
            g_head = T.tucker_core_update_sketched(h, X, F, w.lam, m_t, w.seed_sample, 0, args.reg,
                                                   prec)
            others[other] = {"ms": statistics.mean(alt_ms), "ms_solve": st["ms_solve"],
                             "refine_iters": st["refine_iters"],
                             "rel_diff_vs_timed": float(torch.linalg.norm(g_alt - g_head) /
                                                        torch.linalg.norm(g_head))}
            h2.close()
        # ALS sweeps (Alg. 2) and the adjoint of the frozen-sketch solve (not the headline)
        extra = {}
        if not missing:
            Fa = [a.clone() for a in F]
            ca = T.tucker_core_update_exact(h, X, F, w.lam, "fp64")
            # "sketched": sketched core, exact factors; "sketched_factors": both sketched
            # (FACTOR_M fiber draws per factor update)
            for kind in ("sketched", "exact", "sketched_factors"):
                sk = kind != "exact"
                T.tucker_set_factor_sketch(h, FACTOR_M if kind == "sketched_factors" else 0)
                T.tucker_als_sweep(h, X, Fa, ca, w.lam, sk, m_t, w.seed_sample, 0, args.reg, prec)
                ms_s, _ = timer(lambda: T.tucker_als_sweep(h, X, Fa, ca, w.lam, sk, m_t,
                                                           w.seed_sample, 1, args.reg, prec),
                                min(args.steps, 3))
                extra[f"als_sweep_ms_{kind}"] = statistics.mean(ms_s)
            # ten sweeps of each from the same N(0,1) start: final loss and RMSE
            quality = {}
            c0, F0 = synth.init_state(w)
            for kind in ("exact", "sketched", "sketched_factors"):
                sk = kind != "exact"
                T.tucker_set_factor_sketch(h, FACTOR_M if kind == "sketched_factors" else 0)
                Fq = [torch.from_numpy(a.astype(w.np_dtype)).to(dev) for a in F0]
                cq = torch.from_numpy(c0.reshape(-1).astype(np.float64)).to(dev)
                try:
                    for sw in range(10):
                        loss, rmse = T.tucker_als_sweep(h, X, Fq, cq, w.lam, sk, m_t,
                                                        w.seed_sample, sw, args.reg, prec)
                    quality[kind] = {"loss": loss, "rmse": rmse}
                except T.TuckerError as e:              # reported, not hidden
                    quality[kind] = {"error": str(e), "sweep": sw}
            T.tucker_set_factor_sketch(h, 0)
            extra["als_factor_m"] = FACTOR_M
            extra["als_ten_sweeps"] = quality
            # the CP-ALS variant: one sweep of sketched CP factor updates of rank R_1
            # (FACTOR_M draws per mode) from the workload's factors
            Fc = [a.clone() for a in F]
            T.tucker_cp_als_sweep(h, X, Fc, w.lam, FACTOR_M, w.seed_sample, 0)
            ms_cp, _ = timer(lambda: T.tucker_cp_als_sweep(h, X, Fc, w.lam, FACTOR_M,
                                                           w.seed_sample, 1), min(args.steps, 5))
            extra["cp_als_sweep_ms"] = statistics.mean(ms_cp)
            extra["cp_rank"] = int(F[0].shape[1])
            lev = T.tucker_leverage_scores(h, F)[0]
            smp = T.tucker_sample_rows(h, w.dims, w.ranks, lev, m_t, w.seed_sample, 0, args.reg)
            gf, stf = T.tucker_core_update_sketched(h, X, F, w.lam, 0, 0, 0, args.reg, prec,
                                                    fixed=smp, stats=True)
            gbar = torch.ones(w.d, dtype=torch.float64, device=dev)
            T.tucker_core_solve_adjoint(h, X, F, w.lam, args.reg, prec, smp, stf["solve_id"], gf, gbar)
            ms_a, _ = timer(lambda: T.tucker_core_solve_adjoint(h, X, F, w.lam, args.reg, prec, smp,
                                                                stf["solve_id"], gf, gbar),
                            min(args.steps, 5))
            extra["adjoint_ms"] = statistics.mean(ms_a)
        # lambda-ridge leverage sampling of K (Lemma 4.1, lambda > 0) beside the classical
        # product sampler on the same tensor with a strong ridge (lambda = 1e8: d_eff(K)
        # is about half of d), each on a x2 ladder from m = w.m / 8
        ridge_cfg = None
        if not missing and not args.no_configs and rank == 0:
            wr = dataclasses.replace(w, lam=RIDGE_LAMBDA, m=max(1, w.m // 8))
            _, _, K_r, deff = T.tucker_ridge_tables(h, F, wr.lam)
            ridge_cfg = {"lambda": wr.lam, "d_eff": deff, "d": w.d,
                         "alg1_count_ridge": ridge_alg1_count(w.d, deff),
                         "alg1_count_classical": ridge_alg1_count(w.d, None)}
            for regm in ("ridge", "exact"):
                recr = measure_workload(h, wr, X, F, prec, regm, min(args.steps, 10), args.warmup,
                                        timer)
                ridge_cfg[regm] = {k: recr[k] for k in ("m_star", "ladder", "exact_ms")} | {
                    "ms_at_m_star": recr["at_m_star"]["ms"],
                    "loss_ratio_at_m_star": recr["at_m_star"]["loss_ratio"],
                    "stage_ms_at_m_star": recr["at_m_star"]["stage_ms"]}
        X_h, F_h = hb["X_h"], hb["F_h"]
        f_bytes = sum(a.numel() * a.element_size() for a in hb["F_pin"])
        del X, F, hb
        torch.cuda.empty_cache()
        # the other workloads of the path, timed the same way in the same run
        configs = {}
        if not args.no_configs and rank == 0:
            for name in ("dense4_128_r8_f32", "missing3_1024_r16_f32"):
                if name == w.name:
                    continue
                wc = synth.WORKLOADS[name]
                Xc, Fc, _, cbytes = gpu_inputs(wc, dev)
                hc = T.Handle(stream=stream, solver=args.solver)
                rec = measure_workload(hc, wc, Xc, Fc, prec, args.reg, min(args.steps, 10),
                                       args.warmup, timer)
                rec["config"] = workload_config(wc, prec, args.reg, args.solver, rec["m_timed"],
                                                cbytes)
                configs[name] = rec
                hc.close()
                del Xc, Fc
                torch.cuda.empty_cache()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    ms = head["at_m_star"]["ms"]
    ms_ex = head["exact_ms"]
    ms_e2e = statistics.mean(e2e_ms)
    if world > 1:
        ms, ms_ex, ms_e2e = max_over_ranks([ms, ms_ex, ms_e2e], dev)
    rec = head["at_m_star"]
    kms = rec["kernel_ms"]
    stage = rec["stage_ms"]
    n_real = rec["n_real"]
    pk, src = peaks()
    d = w.d
    traffic_tab = load_traffic()

    def gram_roofline():
        # n_u d (d + 1) flop for the symmetric product plus 2 n_u d for the row build;
        # grouped by the leading index the tensor cores form n_u d' (d' + 1), d' = d / R_1
        flops = n_real * d * (d + 1) + 2 * n_real * d
        grouped = prec in ("bf16", "tf32") and grouped_gram(w)
        narrow = prec in ("bf16", "tf32") and not grouped and narrow_gram(w, rec["n_draws"])
        if grouped or narrow:
            dp = d // w.ranks[0]
            flops = n_real * dp * (dp + 1) + 2 * n_real * dp
        if prec in ("bf16", "tf32"):
            peak = pk["bf16_tflops"] * TC_RATIO[prec]
            bound, note = "tensor", f"{prec} tcgen05: {src} bf16 burst x {TC_RATIO[prec]}"
            kernel = (f"k_syrk_tc<{prec}>" + (" grouped by i_1" if grouped else "")
                      if not narrow else "k_tcg_narrow (per-i_1 Grams, TF32 hi + lo)")
        elif prec == "fp32":
            peak = FP32_PEAK_TFLOPS
            bound, note, kernel = "alu", "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz", "k_syrk_simt<float>"
        else:
            peak = FP64_PEAK_TFLOPS
            bound, note, kernel = "alu", "FP64 nominal 1.25 TFLOP/s", "k_syrk_simt<double>"
        achieved = flops / (kms["gram"] * 1e-3) / 1e12
        return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_tab.get((kernel, w.name)),
                "kernel": kernel, "peak_source": note, "kernel_ms": kms["gram"],
                "flop_per_launch": flops, "launches_per_update": 1}

    def solve_roofline():
        if args.solver == "kpcg":
            # one CG solve: per iteration the product with M~ (2 d^2 flop) and P^-1 (4 d sum R_n)
            solves = rec["refine_iters"] + 1
            iters = max(1, rec["inner_iters"]) / solves
            flops = iters * (2 * d * d + 4 * d * sum(w.ranks))
            kernel = "k_kpcg_cluster" if d <= 576 else "k_kpcg"
            kms_one = kms["first_cg_solve"]
            note = ("FP32 FMA nominal of all 152 SMs (152 x 128 x 2 x 2.07 GHz); the solve runs on "
                    + ("one 8-CTA cluster" if d <= 576 else "a cooperative grid") +
                    " and is latency-bound (a few iterations of d-vector work per launch)")
            launches = solves
        else:
            # the method's work is the factorisation, d^3 / 3 flop
            flops = d ** 3 / 3
            kernel = ("k_chol_coop<double>" if args.solver == "fp64" else
                      "k_chol32_cluster" if d <= 512 else "k_chol_coop<float>")
            kms_one = kms["factor_or_convert"]
            note = "FP32 FMA nominal 80.5 TFLOP/s" if args.solver == "mixed" else "FP64 nominal 1.25 TFLOP/s"
            launches = 1
        peak = FP64_PEAK_TFLOPS if args.solver == "fp64" else FP32_PEAK_TFLOPS
        achieved = flops / (kms_one * 1e-3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_tab.get((kernel, w.name)),
                "kernel": kernel, "peak_source": note, "kernel_ms": kms_one,
                "flop_per_launch": flops, "launches_per_update": launches}

    # the dominant kernel of the timed update: the larger total time per update
    roof_solve, roof_gram = solve_roofline(), gram_roofline()
    t_solve = roof_solve["kernel_ms"] * roof_solve["launches_per_update"]
    roof = roof_solve if t_solve >= roof_gram["kernel_ms"] else roof_gram

    cpu = None
    if rank == 0 and not args.no_cpu:
        wm = dataclasses.replace(w, m=m_t)
        value, sample = oracle_timing(wm, X_h, F_h, args.reg)
        ex_ms, ex_sample = oracle_exact_timing(wm, X_h, F_h)
        cpu = {"value": value, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
               "sample": sample, "exact_value": ex_ms, "exact_sample": ex_sample}

    if rank == 0:
        line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
                "config": workload_config(w, prec, args.reg, args.solver, m_t, in_bytes),
                "exact_ms": ms_ex, "speedup_vs_exact": ms_ex / ms,
                "loss_ratio": rec["loss_ratio"],
                "m_ladder": {"target": LADDER_TARGET, "seeds": LADDER_SEEDS, "rows": head["ladder"],
                             "m_star": head["m_star"]},
                "at_workload_m": {k: head["at_workload_m"][k] for k in
                                  ("ms", "loss_ratio", "stage_ms", "refine_iters", "inner_iters")},
                "speedup_vs_exact_at_workload_m": head["speedup_vs_exact_at_workload_m"],
                "ms_with_stage_events": rec["ms_with_stage_events"],
                "kron_rows_per_s": n_real / (stage["ms_gram"] * 1e-3) * world,
                "n_unique": rec["n_unique"], "refine_iters": rec["refine_iters"],
                "inner_iters": rec["inner_iters"], "stage_ms": stage,
                "exact_hbm_gbs": None if missing else in_bytes / (ms_ex * 1e-3) / 1e9,
                "solver": args.solver, "other_solvers": others, **extra,
                "roofline": roof, "roofline_gram": roof_gram, "roofline_solve": roof_solve,
                "configs": {k: {kk: vv for kk, vv in v.items() if kk != "ladder"} | {"ladder": v["ladder"]}
                            for k, v in configs.items()},
                "ridge_sampling": ridge_cfg,
                "cpu_baseline": cpu,
                "e2e": {"value": ms_e2e, "unit": "ms",
                        "h2d_bytes_per_step": int(in_bytes + f_bytes),
                        "d2h_bytes_per_step": int(w.d * 8)},
                "clocks": clk.summary(), "gpu_launches": rec["launches"] * args.steps}
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
