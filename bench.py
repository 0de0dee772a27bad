#!/usr/bin/env python
"""Benchmark of the sparse-DFT recovery IPM on GB300.

Default line (the largest single-GPU configuration): one step = the learned warm
start (network inference and the predicted interior point) plus one mixed-precision
interior-point solve, to a 1e-6 relative duality gap, of the 512^3 workload
(synthetic: 100000 frequencies, background 1e-3, noise 0.01, radius-2 balls removed
on a period-8 lattice, lambda = 0.05 lambda_max).  Inputs are resident on the device
when the timed region starts; the 25 GB solver state is far larger than L2.  The line
carries the cold FP64 plain solve of the same instance and the ratio, the per-class
CUDA-event breakdown of one warm solve with the dominant class's roofline, KKT
products at 512^3 and 256^3, the 512^2 FP64 solve, an end-to-end time through the C
ABI with pinned host buffers and the oracle's (extrapolated) time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

Prints one JSON line.  Several GPUs run independent replicas (one instance per rank,
no collective on the data path); value = timed wall / solves of all ranks.
--impl reference times the CPU oracle (numpy FP64, direct DFT) on the host cores.
"""

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

METRIC = "IPM solve time to 1e-6 rel. duality gap; KKT matvecs/s and HBM GB/s vs FP64 plain"
FP64_PEAK_TFLOPS = 1.25          # nominal GB300 FP64 rate (no measured FP64 entry in the peaks file)
# FP64 pipe operations per second (an FMA, an add or a multiply is one operation): the
# nominal rate counts an FMA as two flops, so the pipe issues 1.25e12 / 2 = 6.25e11 per
# second, about 2 per clock per SM at 152 SMs and 2.07 GHz
FP64_PIPE_TOPS = FP64_PEAK_TFLOPS / 2
# FP64 pipe operations per coordinate of the Newton-system kernels (counted from their
# code): the predictor 40 (three Newton reciprocals, Sigma, Lambda, P^{-1}, the residuals,
# the affine direction and its second-order terms), prepare after it 14 (the corrector's
# right-hand side, z = P^{-1} r, r^T z); prepare alone (no predictor) 31
FP64_OPS_PREDICTOR, FP64_OPS_PREPARE_PC, FP64_OPS_PREPARE = 40, 14, 31
GAP_TOL = 1e-6
WORKLOADS = {
    "1d": ("1d n=256 FP64 plain IPM: 8 N(0,1) frequencies, noise 0.01, 10% missing at random, "
           "lambda = 0.05 lambda_max, gap 1e-6", "fp64"),
    "2d": ("2d 512x512 FP64 plain IPM: 200 Laplace(0,1) frequencies, noise 0.02, radius-3 discs on a "
           "period-16 lattice (11.3% missing), lambda = 0.02 lambda_max, gap 1e-6", "fp64"),
    "3d": ("3d 256^3 mixed IPM (FP32 FFT products in PCG, FP64 residual/diagonals/reductions): 5000 N(0,1) "
           "frequencies, background 1e-3, noise 0.01, radius-2 balls on a period-8 lattice, "
           "lambda = 0.05 lambda_max, gap 1e-6", "mixed"),
    "warm512": ("512^3, 100000 frequencies, background 1e-3 and noise 0.01, radius-2 balls on a period-8 lattice, "
                "lambda = 0.05 lambda_max, gap 1e-6: learned warm start (network inference included) + mixed "
                "precision solve, against the cold-start FP64 solve of the same instance", "mixed"),
    "infer256": ("warm-start network inference (features + four 3x3x3 convolutions 8->32->32->32->4, BF16 "
                 "tensor cores) on the slot grid 129 x 256 x 256 of the 256^3 workload", "bf16"),
    "kkt256": ("products with the condensed KKT matrix K (FP32 FFT passes of G, FP64 p, q and diagonal) on the 256^3 "
               "workload, mixed precision, back to back through kkt_apply", "mixed"),
    "conv256": ("one 32->32 3x3x3 convolution layer (bias, ReLU, BF16 in, FP32 out) of the warm-start network on "
                "the 129 x 256 x 256 slot grid of the 256^3 workload, tcgen05 tensor cores", "bf16"),
    "paper": ("the paper's own synthetic 3D problem (Sec. 4.1: separable cos + 2 sin signal of frequencies 1, 2, 3, "
              "U(0,1) noise, about 15% missing as radius-2 balls on a period-6 lattice), N x N x N, FP64 plain IPM, "
              "lambda = 0.05 lambda_max, gap 1e-6", "fp64"),
    "batch": ("batch of 48 independent 3D problems, sides drawn from {32,48,64,96,128}, 0.25% frequencies, "
              "Bragg-ball masks (period 8-16, radius 1-2, random offsets), noise 0.01, lambda = 0.05 lambda_max, "
              "gap 1e-6, mixed precision, all solved by one graph launch", "mixed"),
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-kkt", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="run the IPM and PCG loops from the host (use_graph = 0: the same kernels, launched one by "
                         "one; ncu cannot profile kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--size", type=int, default=256, help="--workload paper: grid side N (N x N x N)")
    ap.add_argument("--sigma-rule", type=int, default=None,
                    help="centring rule of every solve (library option sigma_rule; default: the library's)")
    ap.add_argument("--sigma-min", type=float, default=None, help="library option sigma_min (default: the library's)")
    ap.add_argument("--exact-residual", type=int, default=None,
                    help="library option exact_residual (default: the library's)")
    ap.add_argument("--cg-tol", type=float, default=None, help="library option cg_tol (default: the library's)")
    ap.add_argument("--workload", choices=["1d", "2d", "3d", "batch", "warm512", "infer256", "conv256", "kkt256", "paper"],
                    default="warm512",
                    help="warm512 (default): 512^3, learned warm start + mixed precision against the cold FP64 "
                         "solve; 2d: 512^2 FP64; 1d: n=256 FP64; 3d: 256^3 mixed precision; "
                         "batch: 48 uneven 3D problems in one graph launch, mixed precision; "
                         "infer256: the warm-start network alone on the 256^3 slot grid (tensor-core roofline); "
                         "conv256: one of its 32->32 convolution layers; kkt256: KKT products at 256^3 (mixed)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


_OPT_OVERRIDES = {}


def _options(binding, **kw):
    """binding.default_options with the command line's solver overrides applied."""
    kw.update(_OPT_OVERRIDES)
    return binding.default_options(**kw)


def _workload_desc(name):
    return WORKLOADS[name][0]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_solve_seconds(w):
    import numpy as np  # noqa: F401
    from oracle import ipm as oipm
    from oracle.lasso import Problem
    t0 = time.perf_counter()
    prob = Problem(w.dims, w.mask.astype(bool), w.y, 1.0)
    prob.lam = w.lam_rel * prob.lambda_max()
    res = oipm.solve(prob, gap_tol=GAP_TOL, sigma_rule="single", sigma_min=0.01)   # the library's default rule
    return time.perf_counter() - t0, res


def _cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2502_04217_gb300.synth import make_problem
    if args.workload == "warm512":
        return _run_reference_512(args)
    if args.workload in ("3d", "batch", "infer256", "conv256", "kkt256") or (
            args.workload == "paper" and args.size > 32):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle on this workload takes hours on the host "
                          "cores; its CPU baseline is reported (extrapolated from a bounded sample) in the GPU line"}))
        return 0
    w = make_problem("paper", dims=(args.size,)) if args.workload == "paper" else make_problem(args.workload)
    for _ in range(args.warmup):
        _oracle_solve_seconds(w)
    times = []
    res = None
    for _ in range(args.steps):
        t, res = _oracle_solve_seconds(w)
        times.append(t)
    v = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_desc(args.workload), "parallelism": "host cores of rank 0"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": _cores(), "kind": "oracle",
                         "sample": f"full oracle solve (numpy FP64, direct DFT by Vandermonde matrices) of the "
                                   f"{args.workload} workload to gap 1e-6, per step"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "solve": {"ipm_iters": res["ipm_iters"], "cg_iters_total": int(sum(res["cg_counts"])),
                  "rel_gap": res["gap"], "primal": res["primal"]},
    }
    print(json.dumps(line))
    return 0


def _run_reference_512(args):
    """The oracle on the 512^3 workload: a direct-DFT IPM there takes days, so each step is a
    bounded sample -- one oracle product with M_perp^T M_perp at 256^3, timed -- scaled to
    512^3 (x16) and by the products the plain FP64 method takes on this instance.  The value
    is that extrapolated solve time, labelled as such."""
    for _ in range(min(args.warmup, 1)):
        _oracle_product_512_seconds()
    ts, t256 = [], []
    for _ in range(args.steps):
        t512, t = _oracle_product_512_seconds()
        ts.append(t512 * COLD_FP64_PRODUCTS_512)
        t256.append(t)
    v = sum(ts) / len(ts)
    sample = (f"per step one oracle product with M_perp^T M_perp at 256^3 (numpy FP64 direct DFT, mean "
              f"{sum(t256) / len(t256):.2f} s), scaled by n (N0 + N1 + N2) to 512^3 (x16) and by the "
              f"{COLD_FP64_PRODUCTS_512} products of the plain FP64 IPM on this instance: an extrapolated solve time")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * v, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "extrapolated": True,
        "config": {"workload": _workload_desc("warm512"), "dims": [512, 512, 512],
                   "parallelism": "host cores of rank 0"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": _cores(), "kind": "oracle", "extrapolated": True,
                         "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


CLASSES = {"fft_row": 0, "fft_col": 1, "fft_middle": 2, "pcg_update": 3, "ipm_other": 4, "prepare": 6, "step": 7,
           "certificate": 8}


def _breakdown(binding, h):
    """Per-class launches and summed CUDA-event milliseconds since the last profile reset."""
    out = {}
    for nm, k in CLASSES.items():
        n, ms = binding.ipm_profile_get(h, k)
        out[nm] = {"launches": int(n), "ms": ms}
    return out


def _class_model(dims, prec, res, opt):
    """Algorithmic work of each kernel class over one solve, from the solve's own counts.

    Products with G: the PCG products (cg_iters_total; FP32 passes in mixed mode) and
    the FP64 products that computed G beta exactly (kkt_products - cg_iters_total -
    refinements = exact_products).  Bytes per half-spectrum slot (H slots; a beta-layout vector is 16 B
    per slot, a two-block PCG vector 32 B):
      PCG product: first row pass reads z, p and writes p (96 B) and the work buffer;
        last row pass reads the buffer, p, Lambda1, Lambda2 and writes q (96 B);
      FP64 product: reads beta (16 B), writes G beta (16 B);
      every pass between reads and writes the work buffer (8 B per slot in FP32, 16 B in
        FP64); the middle pass also reads the mask bits (n / 8 B);
      pcg_update: reads x, r, p, q and P^{-1}'s three coefficients, writes x, r, z (272 B);
      prepare: reads beta, z, s1, s2, nu1, nu2, G beta, c (128 B), writes 1/s1, 1/s2,
        Lambda1, Lambda2, P^{-1}'s coefficients (112 B) and x, r, z, p (128 B; the
        right-hand side too, 32 B, only with FP64 residual replacement);
        with the predictor-corrector (sigma_rule 2) the class holds two kernels: the
        predictor reads the iterate (128 B) and writes 1/s, Lambda, P^{-1}, the two
        second-order terms and the affine right-hand side (176 B), prepare reads that
        right-hand side, the terms, 1/s and P^{-1} (144 B) and writes x, r, z, p (128 B);
      step: step_length reads x, beta, z, s, nu, 1/s (160 B), step_update reads the same
        and writes beta, z, s, nu (96 B); with the predictor-corrector step_length also
        reads the two terms (32 B) and writes the direction ds, dnu (64 B), which
        step_update reads instead of 1/s and the terms;
      certificate: reads beta, G beta, c (48 B);
      G beta carried (exact_residual 0, CG, no refinement): the last pass of a PCG
        product also writes (G p)_beta (16 B), pcg_update updates G x (48 B), prepare
        clears G x (16 B), step_update updates G beta (reads G beta and G x, writes G beta:
        48 B) and reads c (16 B) for the certificate's four sums, so that the certificate
        reads beta, G beta and c only at the first point and after an exact product.
    FLOPs: 5 L log2 L per complex transform of length L, 2.5 L log2 L per real one.
    FP64 pipe operations of the Newton-system class: FP64_OPS_* per coordinate (2H).
    Returns {class: (working launches, flops, bytes[, FP64 pipe operations])} for one solve.
    """
    import math
    d = len(dims)
    Nl = dims[-1]
    M = 1
    for x in dims[:-1]:
        M *= x
    H = (Nl // 2 + 1) * M
    n = Nl * M
    mixed = prec == "mixed"
    pc = opt.sigma_rule == 2                       # predictor-corrector kernels in the prepare class
    incr = not opt.exact_residual and opt.krylov == 0 and opt.refine_every == 0   # G beta carried
    esz = 8 if mixed else 16                 # bytes of one complex value of the PCG passes
    n_pcg = res["cg_iters_total"]
    n_res = res["kkt_products"] - res["cg_iters_total"] - res.get("refinements", 0)   # FP64 G beta
    it = res["ipm_iters"]
    out = {}
    mid_flops = M * 2 * 2.5 * Nl * math.log2(max(Nl, 2))
    gp = 16 * H if incr else 0
    nP = n_res + n_pcg                              # products of either kind
    if d == 1:
        res_b = 16 * H + 16 * H + n / 8
        pcg_b = 96 * H + 96 * H + gp + n / 8
        out["fft_middle"] = (nP, nP * mid_flops, n_res * res_b + n_pcg * pcg_b)
    else:
        L = dims[1] if d == 3 else dims[0]
        row_flops = (H // L) * 5 * L * math.log2(L)
        res_row = (16 * H + 16 * H) + (16 * H + 16 * H)
        pcg_row = (96 * H + esz * H) + (esz * H + 96 * H + gp)
        out["fft_row"] = (2 * nP, 2 * nP * row_flops, n_res * res_row + n_pcg * pcg_row)
        out["fft_middle"] = (nP, nP * mid_flops,
                             n_res * (32 * H + n / 8) + n_pcg * (2 * esz * H + n / 8))
        if d == 3:
            col_flops = (H // dims[0]) * 5 * dims[0] * math.log2(dims[0])
            out["fft_col"] = (2 * nP, 2 * nP * col_flops,
                              n_res * 2 * 32 * H + n_pcg * 2 * 2 * esz * H)
    out["pcg_update"] = (n_pcg, 0.0, n_pcg * (272 * H + (48 * H if incr else 0)))
    gx = 16 * H if incr else 0
    rhs = 32 * H if (mixed and opt.refine_every > 0) else 0
    if pc:
        out["prepare"] = (2 * it, 0.0, it * ((128 + 176) * H + (144 + 128) * H + rhs + gx),
                          it * 2 * H * (FP64_OPS_PREDICTOR + FP64_OPS_PREPARE_PC))
    else:
        out["prepare"] = (it, 0.0, it * (128 * H + 112 * H + 128 * H + rhs + gx), it * 2 * H * FP64_OPS_PREPARE)
    # with the predictor-corrector step_length also reads the two terms and writes the direction
    # (+32 + 64 B); step_update reads the direction instead of 1/s and the terms (same count);
    # with G beta carried step_update also updates G beta (48 B) and reads c (16 B)
    out["step"] = (2 * it, 0.0, it * (160 * H + 160 * H + 96 * H + (64 * H if incr else 0) + (96 * H if pc else 0)))
    return out


def _rooflines(dims, prec, res, breakdown, steps, opt):
    """Per-class achieved rates over the breakdown's event times (HBM GB/s over algorithmic
    bytes for every class; FP64 TFLOP/s for the FFT classes of FP64 solves) and the
    dominant class (the most event time among the modelled classes)."""
    model = _class_model(dims, prec, res, opt)
    peak = _peaks().get("hbm_gbs", 6800.0)
    cert = breakdown.get("certificate", {"launches": 0})
    Hn = _sizes(dims)[0]
    # a certificate reads beta, G beta and c (48 B per slot) at the first point and after each
    # exact G beta product; with G beta carried it otherwise takes step_update's sums
    n_cert = cert["launches"] // max(steps, 1)
    incr = not opt.exact_residual and opt.krylov == 0 and opt.refine_every == 0
    if incr:
        exact = res["kkt_products"] - res["cg_iters_total"] - res.get("refinements", 0)
        n_cert = min(n_cert, exact + (0 if res.get("warm_start") else 1))
    model["certificate"] = (n_cert, 0.0, n_cert * 48 * Hn)
    classes = {}
    for nm, (work, flops, nbytes, *ops) in model.items():
        b = breakdown.get(nm)
        if not b or not b["launches"] or b["ms"] <= 0:
            continue
        t = b["ms"] / 1e3
        c = {"launches": b["launches"], "working_launches": work * steps, "ms": round(b["ms"], 4),
             "algorithmic_bytes": nbytes * steps, "gbs": nbytes * steps / t / 1e9,
             "frac_of_hbm": nbytes * steps / t / 1e9 / peak}
        if flops:
            c["algorithmic_flops"] = flops * steps
            c["tflops"] = flops * steps / t / 1e12
        if ops:
            c["fp64_ops"] = ops[0] * steps
            c["fp64_tops"] = ops[0] * steps / t / 1e12
            c["frac_of_fp64_pipe"] = c["fp64_tops"] / FP64_PIPE_TOPS
        classes[nm] = c
    dom = max(classes, key=lambda k: classes[k]["ms"])
    return classes, dom


def _roofline_line(dims, prec, res, breakdown, steps, workload, opt):
    """The JSON roofline object of the dominant class (see _rooflines), with every class's
    figures beside it; FP64 FFT classes are reported against the FP64 ALU peak."""
    classes, dom = _rooflines(dims, prec, res, breakdown, steps, opt)
    c = classes[dom]
    peak = _peaks().get("hbm_gbs", 6800.0)
    if prec == "fp64" and dom.startswith("fft"):
        r = {"bound": "alu", "achieved": c["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "frac": c["tflops"] / FP64_PEAK_TFLOPS,
             "peak_source": "nominal GB300 FP64 rate (profiling recipe; no FP64 entry in MEASURED_PEAKS.json)"}
    elif c.get("frac_of_fp64_pipe", 0.0) > c["frac_of_hbm"]:
        r = {"bound": "alu", "achieved": c["fp64_tops"], "peak": FP64_PIPE_TOPS,
             "unit": "T FP64 pipe operations/s (FMA, add, multiply: one each)", "frac": c["frac_of_fp64_pipe"],
             "algorithmic_fp64_ops": c["fp64_ops"],
             "peak_source": "nominal GB300 FP64 rate 1.25 TFLOP/s (profiling recipe) / 2 flops per FMA; "
                            "the class's HBM fraction is in classes"}
    else:
        r = {"bound": "hbm", "achieved": c["gbs"], "peak": peak, "unit": "GB/s", "frac": c["frac_of_hbm"],
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    r.update({"kernel": dom, "traffic": _traffic(dom, workload), "per_launch_us": 1e3 * c["ms"] / c["launches"],
              "launches": c["launches"], "working_launches": c["working_launches"],
              "algorithmic_bytes": c["algorithmic_bytes"], "algorithmic_flops": c.get("algorithmic_flops"),
              "event_ms": c["ms"], "ncu_share": _ncu_share(dom, workload),
              "how": "achieved = algorithmic bytes (or FLOPs) of the class's working launches over the summed "
                     "CUDA-event time of all its launches (launches that find nothing to do included)",
              "classes": classes,
              "breakdown": {k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in breakdown.items()}})
    return r


def _ncu_share(kernel_class, workload):
    """Share of the class in the committed ncu launch list of this workload
    (profiles/shares_<workload>.txt, lines "class<TAB>share"), or None."""
    try:
        rows = {}
        with open(os.path.join(ROOT, "profiles", f"shares_{workload}.txt")) as f:
            for ln in f:
                if "\t" in ln and not ln.startswith("#"):
                    k, v = ln.rstrip("\n").split("\t", 1)
                    rows[k] = v
        if rows.get("csrc_sha256") != _csrc_sha256():
            return None
        return float(rows[kernel_class]) if kernel_class in rows else None
    except Exception:
        return None


def _sizes(dims):
    Nl = dims[-1]
    M = 1
    for x in dims[:-1]:
        M *= x
    return (Nl // 2 + 1) * M, Nl * M


def run_ours(args):
    import numpy as np
    import torch

    from paper_2502_04217_gb300 import binding
    from paper_2502_04217_gb300.synth import make_problem

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load()
    stream = torch.cuda.current_stream()
    w = make_problem("paper", dims=(args.size,)) if args.workload == "paper" else make_problem(args.workload, index=rank)
    prec = WORKLOADS[args.workload][1]
    opt = _options(binding, precision=binding.IPM_MIXED if prec == "mixed" else binding.IPM_FP64,
                                  gap_tol=GAP_TOL, lambda_relative=1, use_graph=0 if args.host_loop else 1)
    mask_d = torch.from_numpy(np.ascontiguousarray(w.mask)).cuda()
    y_d = torch.from_numpy(np.ascontiguousarray(w.y)).cuda()
    h = binding.ipm_create(w.dims, mask_d, y_d, w.lam_rel, opt, stream=stream.cuda_stream)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 512 MB > 129 MB L2

    def one_step(timed):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = binding.ipm_solve(h)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), res

    for _ in range(args.warmup):
        one_step(False)
    # ---- timed region --------------------------------------------------------------
    binding.ipm_profile_enable(h, False)           # resets the launch counter
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    res = None
    torch.cuda.nvtx.range_push("solve")          # lets ncu select exactly the timed solves
    for _ in range(args.steps):
        ms, res = one_step(True)
        step_ms.append(ms)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches, _ = binding.ipm_profile_get(h, 5)
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = t.item()
    value = total_ms / 1e3 / (args.steps * ws)

    # ---- the same steps again with per-launch CUDA events (kernel breakdown) ---------
    binding.ipm_profile_enable(h, True)
    for _ in range(args.steps):
        one_step(True)
    breakdown = _breakdown(binding, h)
    binding.ipm_profile_enable(h, False)
    roofline = _roofline_line(w.dims, prec, res, breakdown, args.steps, args.workload, opt)

    # ---- end to end through the C ABI with pinned host buffers -------------------------
    mask_h = torch.from_numpy(np.ascontiguousarray(w.mask)).pin_memory()
    y_h = torch.from_numpy(np.ascontiguousarray(w.y)).pin_memory()
    H, n = binding.ipm_sizes(h)
    spec_h = torch.empty(2 * H, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        binding.ipm_set_problem(h, mask_h, y_h, w.lam_rel)
        binding.ipm_solve(h)
        binding.ipm_get_spectrum(h, spec_h)
        t1 = time.perf_counter()
        if i > 0:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e = {"value": sum(e2e_ms) / len(e2e_ms) / 1e3, "unit": "s",
           "h2d_bytes_per_step": int(mask_h.numel() * 1 + y_h.numel() * 8),
           "d2h_bytes_per_step": int(spec_h.numel() * 8)}

    # ---- KKT matvec throughput, FP32 G-apply with FP64 diagonal (3D 256^3) -------------
    kkt = None
    if not args.no_kkt and rank == 0 and args.workload == "2d":
        kkt = _kkt_throughput(binding, torch, np)

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        if len(w.dims) == 3 and int(np.prod(w.dims)) > 40000:
            t_g = _oracle_g_seconds(w)
            side = "x".join(str(d) for d in w.dims)
            cpu = {"value": t_g * res["kkt_products"], "unit": "s", "cores": _cores(), "kind": "oracle",
                   "extrapolated": True,
                   "sample": f"one oracle product with M_perp^T M_perp at {side} ({t_g:.2f} s, direct DFT) times the "
                             f"{res['kkt_products']} products of the GPU solve"}
        else:
            t, ores = _oracle_solve_seconds(w)
            cpu = {"value": t, "unit": "s", "cores": _cores(), "kind": "oracle",
                   "sample": f"one full oracle solve (numpy FP64, direct DFT) of the same {args.workload} "
                             "workload to gap 1e-6"}
    tiles = binding.ipm_describe(h)
    binding.ipm_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": _workload_desc(args.workload), "dims": list(w.dims), "gap_tol": GAP_TOL,
                       "l2": "flushed between steps (512 MB write outside the timed events)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "launch": "host-driven loops" if args.host_loop else "one CUDA graph per solve"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "solve": {"ipm_iters": res["ipm_iters"], "cg_iters_total": res["cg_iters_total"],
                      "kkt_products": res["kkt_products"], "rel_gap": res["rel_gap"], "primal": res["primal"],
                      "step_ms": [round(x, 3) for x in step_ms]},
            "kkt_matvec": kkt,
            "fft_tiles": tiles,
        }
        if args.workload == "paper":
            line["paper_context"] = _paper_context(args.size)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


# The paper's Table "artificial" (Sec. 5): total solve times of its own synthetic
# problem on a GH200 GPU and an unnamed CPU, FP64 implied, stopped at a primal-dual
# residual of 1e-8 (not our relative duality gap).  Context only: another machine,
# another stopping rule.
PAPER_ARTIFICIAL_S = {8: (0.0031, 0.63), 16: (0.013, 0.72), 32: (0.10, 0.68), 64: (1.29, 0.71), 96: (4.49, 0.79),
                      128: (10.34, 1.07), 192: (41.78, 3.22), 256: (101.38, 5.88), 384: (367.78, 20.66),
                      512: (929.26, 104.55), 560: (1290.77, 159.66)}


def _paper_context(N):
    if N not in PAPER_ARTIFICIAL_S:
        return None
    cpu, gpu = PAPER_ARTIFICIAL_S[N]
    return {"paper_gpu_s": gpu, "paper_cpu_s": cpu, "hardware": "GH200 (paper) / CPU unnamed",
            "stopping": "paper: primal-dual residual 1e-8; here: relative duality gap 1e-6",
            "source": "Table artificial, Sec. 5"}


def _oracle_g_seconds(w):
    import numpy as np
    from oracle.lasso import Problem
    prob = Problem(w.dims, w.mask.astype(bool), w.y, 1.0)
    beta = np.random.default_rng(0).standard_normal(prob.n)
    t0 = time.perf_counter()
    prob.G(beta)
    return time.perf_counter() - t0


def _csrc_sha256():
    import hashlib
    hs = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2502_04217_gb300", "csrc")
    for nm in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, nm), "rb") as f:
            hs.update(f.read())
    return hs.hexdigest()


def _traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu summary
    profiles/traffic_<workload>.txt (lines "csrc_sha256<TAB>hex" and "kernel<TAB>bytes"),
    or None when there is none or the CUDA sources changed since it was taken."""
    try:
        rows = {}
        with open(os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")) as f:
            for ln in f:
                if "\t" in ln and not ln.startswith("#"):
                    k, v = ln.rstrip("\n").split("\t", 1)
                    rows[k] = v
        if rows.get("csrc_sha256") != _csrc_sha256():
            return None
        return float(rows[kernel]) if kernel in rows else None
    except Exception:
        return None


def _kkt_throughput(binding, torch, np, reps=20, w=None, h=None, label="3d 256^3 mixed (FP32 FFT, FP64 diagonal)"):
    """Back-to-back products with K through kkt_apply (inside the NVTX range "kkt"): on the
    handle h with its current Sigma, else on a new mixed-precision handle of the 256^3
    workload with Sigma1 = 1/2, Sigma2 = 2."""
    from paper_2502_04217_gb300.synth import make_problem
    stream = torch.cuda.current_stream()
    own = h is None
    if own:
        w = w if w is not None else make_problem("3d")
        opt = _options(binding, precision=binding.IPM_MIXED, lambda_relative=1)
        h = binding.ipm_create(w.dims, w.mask, w.y, w.lam_rel, opt, stream=stream.cuda_stream)
    p = q = None
    try:
        H, n = binding.ipm_sizes(h)
        if own:
            ones = torch.ones(2 * H, dtype=torch.float64, device="cuda")
            binding.ipm_set_sigma(h, ones, ones * 0.5, ones * 2.0, ones)
            del ones
        p = torch.randn(4 * H, dtype=torch.float64, device="cuda")
        binding.ipm_pack_beta(h, p[: 2 * H].clone(), p[: 2 * H])
        binding.ipm_pack_beta(h, p[2 * H:].clone(), p[2 * H:])
        q = torch.empty_like(p)
        for _ in range(3):
            binding.kkt_apply(h, p, q)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("kkt")
        e0.record(stream)
        for _ in range(reps):
            binding.kkt_apply(h, p, q)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        t = e0.elapsed_time(e1) / 1e3 / reps
        # the same products with per-launch CUDA events (the library's profile mode): the
        # five passes' own device time, without the gaps between synchronous calls
        binding.ipm_profile_enable(h, True)
        for _ in range(reps):
            binding.kkt_apply(h, p, q)
        bd = _breakdown(binding, h)
        binding.ipm_profile_enable(h, False)
        t_dev = sum(bd[c]["ms"] for c in ("fft_row", "fft_col", "fft_middle")) / 1e3 / reps
        # compulsory bytes of one product: p, q (FP64, 2 blocks), Lambda1, Lambda2 (FP64), mask bits
        algo = (4 * H * 8) * 2 + (2 * H * 8) * 2 + n / 8
        peak = _peaks().get("hbm_gbs", 6800.0)
        return {"workload": label, "matvecs_per_s": 1.0 / t,
                "ms_per_matvec": t * 1e3, "algorithmic_bytes": algo, "algorithmic_gbs": algo / t / 1e9,
                "hbm_peak_gbs": peak, "frac_of_hbm": algo / t / 1e9 / peak, "reps": reps,
                "kernel_ms_per_matvec": t_dev * 1e3, "kernel_frac_of_hbm": algo / t_dev / 1e9 / peak,
                "timing": "ms_per_matvec: CUDA events around back-to-back kkt_apply calls on the stream (each call "
                          "returns after its work); kernel_ms_per_matvec: the sum of the five passes' per-launch "
                          "CUDA-event times (the events keep the passes from overlapping their launches)",
                "tiles": binding.ipm_describe(h)}
    finally:
        del p, q
        if own:
            binding.ipm_destroy(h)


def run_batch(args):
    """48 uneven problems per step, solved by one graph launch (ranks split the problems)."""
    import numpy as np
    import torch

    from paper_2502_04217_gb300 import binding
    from paper_2502_04217_gb300.synth import batch_workloads

    ws_n, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load()
    allw = batch_workloads(48)
    # the 48 problems are split across ranks (cost n log2 n, largest first to the lightest rank)
    from paper_2502_04217_gb300 import shard
    ws = [allw[i] for i in shard.rank_share([w.dims for w in allw], ws_n, rank)]
    stream = torch.cuda.current_stream()
    opt = _options(binding, precision=binding.IPM_MIXED, gap_tol=GAP_TOL, lambda_relative=1)
    b = binding.ipm_create_batch([(w.dims, w.mask, w.y, w.lam_rel) for w in ws], opt, stream=stream.cuda_stream)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = binding.ipm_solve_batch(b)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), res

    for _ in range(args.warmup):
        step()
    members = [binding.ipm_batch_member(b, i) for i in range(len(ws))]
    for h in members:
        binding.ipm_profile_enable(h, False)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, res = [], None
    for _ in range(args.steps):
        ms, res = step()
        step_ms.append(ms)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = sum(binding.ipm_profile_get(h, 5)[0] for h in members)
    total_ms = shard.max_over_ranks(sum(step_ms), dist, device="cuda")
    value = total_ms / 1e3 / args.steps
    # aggregate algorithmic bytes of all FFT passes of all members, per batch
    nbytes = 0.0
    for w, r in zip(ws, res):
        for cls, (_, _, by, *_ops) in _class_model(w.dims, "mixed", r, opt).items():
            if cls.startswith("fft"):
                nbytes += by
    peak = _peaks().get("hbm_gbs", 6800.0)
    # what the concurrent branches buy: the same members solved one after another
    serial = 0.0
    for h in members:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        binding.ipm_solve(h)
        e1.record(stream)
        e1.synchronize()
        serial += e0.elapsed_time(e1) / 1e3
    all_bytes = 0.0
    for w, r in zip(ws, res):
        all_bytes += sum(v[2] for v in _class_model(w.dims, "mixed", r, opt).values())
    ach = all_bytes / value / 1e9
    roofline = {"bound": "hbm", "kernel": "every kernel class of every member (aggregate)", "achieved": ach,
                "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "algorithmic_bytes": all_bytes, "fft_passes_algorithmic_bytes": nbytes,
                "fft_passes_frac": nbytes / value / 1e9 / peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "note": "graph branches run concurrently, so per-kernel event times do not exist; algorithmic bytes "
                        "of every kernel class (bench._class_model) of every member over the batch wall time"}
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        t_cpu, solved, extrap = 0.0, 0, 0
        for w, r in zip(ws, res):
            if max(w.dims) <= 48:
                t, _ = _oracle_solve_seconds(w)
                solved += 1
            else:
                t = _oracle_g_seconds(w) * r["kkt_products"]
                extrap += 1
            t_cpu += t
        cpu = {"value": t_cpu, "unit": "s", "cores": _cores(), "kind": "oracle", "extrapolated": extrap > 0,
               "sample": f"{solved} members (sides <= 48) solved fully by the oracle; {extrap} larger members: one "
                         "oracle product with M_perp^T M_perp times the GPU solve's product count"}
    # end to end: every member's inputs re-uploaded from pinned host memory, spectra read back
    pins = [(torch.from_numpy(np.ascontiguousarray(w.mask)).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(w.y)).pin_memory()) for w in ws]
    specs = []
    for h in members:
        H, n = binding.ipm_sizes(h)
        specs.append(torch.empty(2 * H, dtype=torch.float64).pin_memory())
    e2e_ms = []
    for i in range(args.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for h, (m, y), w in zip(members, pins, ws):
            binding.ipm_set_problem(h, m, y, w.lam_rel)
        binding.ipm_solve_batch(b)
        for h, sp in zip(members, specs):
            binding.ipm_get_spectrum(h, sp)
        if i > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e = {"value": sum(e2e_ms) / len(e2e_ms) / 1e3, "unit": "s",
           "h2d_bytes_per_step": int(sum(m.numel() + 8 * y.numel() for m, y in pins)),
           "d2h_bytes_per_step": int(sum(8 * sp.numel() for sp in specs))}
    binding.ipm_destroy_batch(b)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": _workload_desc("batch"), "problems": len(allw),
                       "problems_this_rank": len(ws), "voxels": int(sum(np.prod(w.dims) for w in allw)),
                       "l2": "flushed between steps (512 MB write outside the timed events)",
                       "parallelism": "problems split across ranks" if ws_n > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "serial_members_s": serial, "concurrency_speedup": serial / value,
            "all_classes_hbm_frac": all_bytes / value / 1e9 / peak,
            "solve": {"problems_per_s": len(allw) / value, "ipm_iters": [r["ipm_iters"] for r in res],
                      "cg_iters_total": int(sum(r["cg_iters_total"] for r in res)),
                      "max_rel_gap": max(r["rel_gap"] for r in res),
                      "step_ms": [round(x, 3) for x in step_ms]},
        }))
    if dist:
        dist.destroy_process_group()
    return 0


def _fp64_2d_extra(binding, torch, reps=10):
    """The 512^2 FP64 plain solve (the 2d workload), a short extra measurement beside the
    default line: solve time (CUDA events, L2 flushed between solves) and counts."""
    import numpy as np
    from paper_2502_04217_gb300.synth import make_problem
    w = make_problem("2d")
    stream = torch.cuda.current_stream()
    opt = _options(binding, precision=binding.IPM_FP64, gap_tol=GAP_TOL, lambda_relative=1)
    h = binding.ipm_create(w.dims, np.ascontiguousarray(w.mask), np.ascontiguousarray(w.y), w.lam_rel, opt,
                           stream=stream.cuda_stream)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")
    try:
        ts, res = [], None
        for i in range(reps + 3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = binding.ipm_solve(h)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                ts.append(e0.elapsed_time(e1))
        return {"workload": _workload_desc("2d"), "ms_per_solve": sum(ts) / len(ts), "ipm_iters": res["ipm_iters"],
                "cg_iters_total": res["cg_iters_total"], "kkt_products": res["kkt_products"],
                "rel_gap": res["rel_gap"], "solves": reps}
    finally:
        binding.ipm_destroy(h)
        del flush


# Products with M_perp^T M_perp the oracle's IPM performs on the 512^3 instance: the
# plain FP64 method with the library's default rules takes 8 IPM iterations and 43 PCG
# iterations there (measured on a GB300 with this library), and the oracle forms G beta
# once per IPM iteration plus once at the end: 43 + 9 = 52.  The reference arm multiplies
# the oracle's measured time per product by it.
COLD_FP64_PRODUCTS_512 = 52


def _oracle_product_512_seconds():
    """The oracle's time for one product with M_perp^T M_perp at 512^3, extrapolated from
    one timed product at 256^3 (direct DFT along each axis: cost n (N0 + N1 + N2), 16x
    from 256^3 to 512^3).  Returns (seconds at 512^3, seconds measured at 256^3)."""
    from paper_2502_04217_gb300.synth import make_problem
    t = _oracle_g_seconds(make_problem("3d"))
    return 16.0 * t, t


def run_warm512(args):
    """Default line: the 512^3 learned-warm-start mixed-precision solve to a 1e-6 gap
    (network inference included), against the cold FP64 plain solve of the same instance."""
    import numpy as np
    import torch

    from paper_2502_04217_gb300 import binding
    from paper_2502_04217_gb300 import warmstart as wsm
    from paper_2502_04217_gb300.synth import make_problem

    ws_n, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load()
    stream = torch.cuda.current_stream()
    w = make_problem("3d512", index=rank)
    net = wsm.load(stream=stream.cuda_stream)
    graph = 0 if args.host_loop else 1
    o64 = _options(binding, precision=binding.IPM_FP64, gap_tol=GAP_TOL, lambda_relative=1, use_graph=graph)
    o32 = _options(binding, precision=binding.IPM_MIXED, gap_tol=GAP_TOL, lambda_relative=1, use_graph=graph)
    mask_d = torch.from_numpy(np.ascontiguousarray(w.mask)).cuda()
    y_d = torch.from_numpy(np.ascontiguousarray(w.y)).cuda()
    h64 = binding.ipm_create(w.dims, mask_d, y_d, w.lam_rel, o64, stream=stream.cuda_stream)
    h32 = binding.ipm_create(w.dims, mask_d, y_d, w.lam_rel, o32, stream=stream.cuda_stream)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    def warm():
        binding.ws_predict(net, h32, wsm.MU_SCALE)
        return binding.ipm_solve(h32)

    for _ in range(args.warmup):
        warm()
    # ---- timed region: K warm-start solves ------------------------------------------
    binding.ipm_profile_enable(h32, False)        # resets the device launch counter
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wt, rw = [], None
    torch.cuda.nvtx.range_push("solve")          # lets ncu select exactly the timed solves
    for _ in range(args.steps):
        t, rw = timed(warm)
        wt.append(t)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches, _ = binding.ipm_profile_get(h32, 5)
    launches += 6 * args.steps                     # features, 4 convolutions, start point per step
    total = sum(wt)
    if dist:
        tt = torch.tensor([total], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total = tt.item()
    value = total / (args.steps * ws_n)

    # ---- the plain method on the same instance: cold FP64 (and cold mixed) -------------
    binding.ipm_solve(h64)
    c64 = [timed(lambda: binding.ipm_solve(h64)) for _ in range(2)]
    t64, r64 = sum(t for t, _ in c64) / len(c64), c64[-1][1]
    tcold32, rc32 = timed(lambda: binding.ipm_solve(h32))
    t_inf = timed(lambda: binding.ws_forward(net, h32, None))[0]

    # ---- per-launch CUDA events of one warm solve: classes and the dominant one --------
    binding.ipm_profile_enable(h32, True)
    binding.ws_predict(net, h32, wsm.MU_SCALE)
    rp = dict(binding.ipm_solve(h32), warm_start=True)
    breakdown = _breakdown(binding, h32)
    binding.ipm_profile_enable(h32, False)
    roofline = _roofline_line(w.dims, "mixed", rp, breakdown, 1, "warm512", o32)

    # ---- KKT products at 512^3 (this instance, Sigma of the last iterate) and 256^3 ------
    kkt512 = _kkt_throughput(binding, torch, np, reps=10, h=h32, label="3d 512^3 mixed (FP32 FFT, FP64 diagonal)")

    # ---- end to end: problem from pinned host buffers, spectrum back to the host -------
    mask_h = mask_d.cpu().pin_memory()
    y_h = y_d.cpu().pin_memory()
    H, n = binding.ipm_sizes(h32)
    spec_h = torch.empty(2 * H, dtype=torch.float64).pin_memory()
    e2e_steps = min(args.steps, 5)
    e2e_t = []
    split = [0.0, 0.0, 0.0]
    for i in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        binding.ipm_set_problem(h32, mask_h, y_h, w.lam_rel)      # returns after its work (reads lambda_max)
        ta = time.perf_counter()
        warm()
        torch.cuda.synchronize()
        tb = time.perf_counter()
        binding.ipm_get_spectrum(h32, spec_h)
        t1 = time.perf_counter()
        if i > 0:
            e2e_t.append(t1 - t0)
            split = [split[0] + ta - t0, split[1] + tb - ta, split[2] + t1 - tb]
    e2e = {"value": sum(e2e_t) / len(e2e_t), "unit": "s", "h2d_bytes_per_step": int(mask_h.numel() + y_h.numel() * 8),
           "d2h_bytes_per_step": int(spec_h.numel() * 8), "steps": e2e_steps,
           "split_s": {"set_problem": split[0] / e2e_steps, "predict_and_solve": split[1] / e2e_steps,
                       "get_spectrum": split[2] / e2e_steps},
           "path": "ipm_set_problem (pinned host mask and signal) + ws_predict + ipm_solve + ipm_get_spectrum "
                   "(pinned host), wall clock"}
    binding.ipm_destroy(h64)
    binding.ipm_destroy(h32)
    binding.ws_destroy(net)
    del mask_d, y_d
    torch.cuda.empty_cache()
    kkt256 = _kkt_throughput(binding, torch, np, reps=20)

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        t512, t256 = _oracle_product_512_seconds()
        cpu = {"value": t512 * rw["kkt_products"], "unit": "s", "cores": _cores(), "kind": "oracle",
               "extrapolated": True,
               "sample": f"one oracle product with M_perp^T M_perp at 256^3 ({t256:.2f} s, numpy FP64 direct DFT), "
                         f"scaled by n (N0 + N1 + N2) to 512^3 (x16) and by the {rw['kkt_products']} products of "
                         "the warm solve"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32+f64", "data": "synthetic",
            "config": {"workload": _workload_desc("warm512"), "dims": list(w.dims), "gap_tol": GAP_TOL,
                       "network": "4-layer 3x3x3 conv, 32 channels, BF16, trained on 128^3 instances (weights file)",
                       "mu_scale": wsm.MU_SCALE, "l2": "inputs far larger than L2 (512^3 state: 25 GB)",
                       "parallelism": "replicas (one instance per rank)" if ws_n > 1 else "single GPU",
                       "launch": "network kernels + " + ("host-driven loops" if args.host_loop else
                                                          "one CUDA graph per solve")},
            "vs_fp64_plain": value / t64, "cold_fp64_s": t64, "cold_mixed_s": tcold32, "inference_s": t_inf,
            "solve": {"warm_ipm_iters": rw["ipm_iters"], "warm_cg_iters": rw["cg_iters_total"],
                      "warm_kkt_products": rw["kkt_products"], "cold_fp64_ipm_iters": r64["ipm_iters"],
                      "cold_fp64_cg_iters": r64["cg_iters_total"], "cold_fp64_kkt_products": r64["kkt_products"],
                      "cold_mixed_ipm_iters": rc32["ipm_iters"], "cold_mixed_cg_iters": rc32["cg_iters_total"],
                      "warm_rel_gap": rw["rel_gap"], "cold_fp64_rel_gap": r64["rel_gap"],
                      "objective_rel_diff": abs(rw["primal"] - r64["primal"]) / abs(r64["primal"]),
                      "step_s": [round(x, 4) for x in wt]},
            "clocks": clk, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "kkt_matvec": {"512^3": kkt512, "256^3": kkt256},
            "fp64_2d": _fp64_2d_extra(binding, torch),
        }))
    if dist:
        dist.destroy_process_group()
    return 0


def _oracle_layers(binding, net):
    """The network's parameters in the oracle's layout: [(W (3,3,3,cin,cout), b)] over real channels."""
    import numpy as np
    from paper_2502_04217_gb300 import warmstart as wsm
    p = np.empty(binding.ws_num_params(net), dtype=np.float32)
    binding.ws_get_params(net, p)
    out, o = [], 0
    for cin, cout, cir, cor in wsm.LAYERS:
        W = p[o:o + 27 * cout * cin].reshape(3, 3, 3, cout, cin).transpose(0, 1, 2, 4, 3)
        o += 27 * cout * cin
        b = p[o:o + cout]
        o += cout
        out.append((W[:, :, :, :cir, :cor].astype(np.float64).copy(), b[:cor].astype(np.float64)))
    return out


def run_kkt256(args):
    """Products with K at 256^3 in mixed precision: time per product, HBM roofline over its compulsory bytes."""
    import numpy as np
    import torch

    from paper_2502_04217_gb300 import binding
    from paper_2502_04217_gb300.synth import make_problem

    ws_n, rank, local = _dist()
    torch.cuda.set_device(local)
    binding.load()
    w = make_problem("3d", index=rank)
    clocks = ClockSampler(local)
    clocks.start()
    k = _kkt_throughput(binding, torch, np, reps=max(args.steps, 5), w=w)
    clk = clocks.stop()
    value = k["ms_per_matvec"] / 1e3
    peak = k["hbm_peak_gbs"]
    roofline = {"bound": "hbm", "achieved": k["algorithmic_gbs"], "peak": peak, "unit": "GB/s",
                "frac": k["frac_of_hbm"], "traffic": _traffic("kkt_apply (5 passes)", "kkt256"),
                "kernel": "kkt_apply: row(inv) -> col(inv) -> middle -> col(fwd) -> row(fwd, K diagonal)",
                "algorithmic_bytes": k["algorithmic_bytes"],
                "how": "achieved = compulsory bytes of one product over the stream time per call (CUDA events "
                       "around back-to-back calls); the five passes' own per-launch event times sum to "
                       "kkt_matvec.kernel_ms_per_matvec, about the same (the per-launch events stop the passes "
                       "from overlapping their launches)",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        t_g = _oracle_g_seconds(w)
        cpu = {"value": t_g, "unit": "s", "cores": _cores(), "kind": "oracle",
               "sample": "one oracle product with M_perp^T M_perp at 256^3 (direct DFT), the dominant part of a "
                         "product with K"}
    if rank == 0:
        print(json.dumps({
            "metric": "KKT matvec time (256^3, mixed precision)", "value": value, "unit": "s", "n_gpus": ws_n,
            "steps": max(args.steps, 5), "warmup": 3, "ms_per_step": 1e3 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": _workload_desc("kkt256"), "dims": list(w.dims),
                       "l2": "p, q, Lambda (1.35 GB per product) far larger than L2"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "gpu_launches": 5 * max(args.steps, 5),
            "clocks": clk, "kkt_matvec": k,
            "e2e_note": "kkt_apply works on device vectors; the solve lines carry the host path",
        }))
    return 0


def _conv_layer_roofline(binding, torch, D, reps, timed):
    """Per-launch time of one 32 -> 32 tcgen05 convolution on grid D and its tensor roofline."""
    V = D[0] * D[1] * D[2]
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(V * 32, device="cuda", generator=g).to(torch.bfloat16)
    wt = (0.05 * torch.randn(27 * 32 * 32, device="cuda", generator=g)).to(torch.bfloat16)
    bias = torch.zeros(32, device="cuda")
    yb = torch.empty(V * 32, device="cuda")
    layer = lambda: binding.ws_conv_forward(32, 32, D, x.view(torch.int16), wt.view(torch.int16), bias, 1, None, yb)
    for _ in range(3):
        timed(layer)
    lt = [timed(layer) for _ in range(reps)]
    t_layer = sum(lt) / len(lt)
    flops = 2.0 * V * 27 * 32 * 32
    peak = _peaks().get("bf16_tflops", 1900.0)
    achieved = flops / t_layer / 1e12
    del x, yb
    return ({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
             "traffic": _traffic("conv_tc_kernel<32,32>", "conv256"),
             "kernel": "conv_tc_kernel<32,32>: one 32->32 layer, tcgen05.mma M=128 N=32 K=16, FP32 output",
             "per_launch_us": 1e6 * t_layer, "algorithmic_flops": flops,
             "algorithmic_bytes": V * 32 * 2 + V * 32 * 4 + 27 * 32 * 32 * 2,
             "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; of measured)"}, lt)


def run_conv256(args):
    """One 32 -> 32 convolution layer on the 129 x 256 x 256 grid (tcgen05 kernel alone)."""
    import torch

    from paper_2502_04217_gb300 import binding

    ws_n, rank, local = _dist()
    torch.cuda.set_device(local)
    binding.load()
    stream = torch.cuda.current_stream()
    D = (129, 256, 256)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    clocks = ClockSampler(local)
    clocks.start()
    roofline, lt = _conv_layer_roofline(binding, torch, D, args.steps, timed)
    clk = clocks.stop()
    value = sum(lt) / len(lt)
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        import numpy as np
        from oracle import warmstart as ows
        rng = np.random.default_rng(0)
        sub = (8, 32, 32)
        xs, Ws = rng.standard_normal(sub + (32,)), 0.05 * rng.standard_normal((3, 3, 3, 32, 32))
        t0 = time.perf_counter()
        ows.conv3d(xs, Ws, np.zeros(32))
        t_s = time.perf_counter() - t0
        vs, V = sub[0] * sub[1] * sub[2], D[0] * D[1] * D[2]
        cpu = {"value": t_s * V / vs, "unit": "s", "cores": _cores(), "kind": "oracle", "extrapolated": True,
               "sample": f"oracle conv3d (numpy FP64) on an 8x32x32 block ({t_s:.3f} s), scaled by voxel count"}
    if rank == 0:
        print(json.dumps({
            "metric": "3x3x3 convolution layer time (32->32 channels)", "value": value, "unit": "s", "n_gpus": ws_n,
            "steps": args.steps, "warmup": 3, "ms_per_step": 1e3 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": _workload_desc("conv256"), "grid": list(D),
                       "l2": "input 541 MB and output 1.08 GB, both larger than L2"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "gpu_launches": args.steps + 3, "clocks": clk,
            "e2e_note": "a single layer works on device buffers only; the network line (infer256) has the host path",
            "layer_s": [round(t, 6) for t in lt],
        }))
    return 0


def run_infer256(args):
    """The warm-start network forward on the 256^3 slot grid; roofline of the 32->32 tcgen05 convolution."""
    import numpy as np
    import torch

    from paper_2502_04217_gb300 import binding
    from paper_2502_04217_gb300 import warmstart as wsm
    from paper_2502_04217_gb300.synth import make_problem

    ws_n, rank, local = _dist()
    torch.cuda.set_device(local)
    binding.load()
    stream = torch.cuda.current_stream()
    w = make_problem("3d", index=rank)
    opt = _options(binding, precision=binding.IPM_MIXED, gap_tol=GAP_TOL, lambda_relative=1)
    h = binding.ipm_create(w.dims, w.mask, w.y, w.lam_rel, opt, stream=stream.cuda_stream)
    net = wsm.load(stream=stream.cuda_stream)
    H, n = binding.ipm_sizes(h)
    V = H                                   # one voxel per half-spectrum slot
    D = (w.dims[-1] // 2 + 1, w.dims[0], w.dims[1])
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 512 MB > L2

    def timed(fn):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    fwd = lambda: binding.ws_forward(net, h, None)
    for _ in range(args.warmup):
        timed(fwd)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    ts = [timed(fwd) for _ in range(args.steps)]
    clk = clocks.stop()
    value = sum(ts) / len(ts)
    net_flops = 2.0 * V * 27 * sum(cir * cor for _, _, cir, cor in wsm.LAYERS)

    # dominant kernel: one 32 -> 32 layer (bias, ReLU) on the same grid, per-launch events
    roofline, lt = _conv_layer_roofline(binding, torch, D, max(5, args.steps), timed)
    roofline["network_tflops"] = net_flops / value / 1e12

    # end to end: problem from pinned host buffers, prediction back to the host
    mask_h = torch.from_numpy(np.ascontiguousarray(w.mask)).pin_memory()
    y_h = torch.from_numpy(np.ascontiguousarray(w.y)).pin_memory()
    out_h = torch.empty(V * 8, dtype=torch.float32).pin_memory()
    e2e_t = []
    for i in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        binding.ipm_set_problem(h, mask_h, y_h, w.lam_rel)
        binding.ws_forward(net, h, out_h)
        t1 = time.perf_counter()
        if i > 0:
            e2e_t.append(t1 - t0)
    e2e = {"value": sum(e2e_t) / len(e2e_t), "unit": "s", "h2d_bytes_per_step": int(mask_h.numel() + y_h.numel() * 8),
           "d2h_bytes_per_step": int(out_h.numel() * 4)}

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        from oracle import warmstart as ows
        layers = _oracle_layers(binding, net)
        sub = (8, 32, 32)
        xs = np.random.default_rng(0).standard_normal(sub + (8,))
        t0 = time.perf_counter()
        ows.forward(xs, layers)
        t_s = time.perf_counter() - t0
        vs = sub[0] * sub[1] * sub[2]
        cpu = {"value": t_s * V / vs, "unit": "s", "cores": _cores(), "kind": "oracle", "extrapolated": True,
               "sample": f"oracle network forward (numpy FP64) on an {sub[0]}x{sub[1]}x{sub[2]} block of random "
                         f"features ({t_s:.2f} s), scaled by voxel count to the {D[0]}x{D[1]}x{D[2]} grid"}
    binding.ws_destroy(net)
    binding.ipm_destroy(h)
    if rank == 0:
        print(json.dumps({
            "metric": "warm-start network inference time (features + 4 convolutions)", "value": value, "unit": "s",
            "n_gpus": ws_n, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * value,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": _workload_desc("infer256"), "grid": list(D),
                       "l2": "flushed between steps (512 MB write outside the timed events)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 5 * args.steps, "clocks": clk,
            "step_s": [round(t, 5) for t in ts], "layer_s": [round(t, 5) for t in lt],
        }))
    return 0


def main():
    args = _args()
    if args.sigma_rule is not None:
        _OPT_OVERRIDES["sigma_rule"] = args.sigma_rule
    if args.sigma_min is not None:
        _OPT_OVERRIDES["sigma_min"] = args.sigma_min
    if args.exact_residual is not None:
        _OPT_OVERRIDES["exact_residual"] = args.exact_residual
    if args.cg_tol is not None:
        _OPT_OVERRIDES["cg_tol"] = args.cg_tol
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "warm512":
        return run_warm512(args)
    if args.workload == "infer256":
        return run_infer256(args)
    if args.workload == "conv256":
        return run_conv256(args)
    if args.workload == "kkt256":
        return run_kkt256(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
