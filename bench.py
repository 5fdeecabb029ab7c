"""Benchmark: theta-evaluations per second of the dense INLA hot path at n = 16384.

Workload: the Poisson spatial LGM with n = 16384 latent (intercept + 16383 points, dense
anisotropic exponential covariance with a folded iid term), m = 100000 observations,
theta of dimension 4, and the batch of 2*4+1 central finite-difference theta points of one
BFGS gradient.  A step = one batched evaluation of all 9 points: prior build and
inversion, Newton to the mode (Cholesky + solves per step), the final factorisation,
log pi~(theta|y) and the marginal variances diag(Q*^-1), all on the GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...     (the FP64 CPU oracle on the host cores)

One JSON line on stdout (rank 0).  `value` is the mixed-precision path (Ozaki-split BF16
tensor cores, double-float storage) with the model resident on the device; `e2e` goes
through the C ABI from host buffers (model upload, evaluation, results back) every step.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "θ-evals/sec at n=16384 (FP64 vs mixed @ stated err); % of FP64/TC roofline"
UNIT = "theta-evals/s"
WORKLOAD = "poisson_n16384_m100000_fd9"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for i, nm in enumerate(names):
                if len(s) > 5 + i and s[5 + i].strip().lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


BENCH_WORKLOAD = "poisson_n16384_m100000_fd9"
CAPTURE_WORKLOADS = ("poisson_n4096_m20000_fd7", "poisson_n256_m1000_5pts")
# DRAM traffic of the GEMM as a multiple of its compulsory bytes (slice planes read once, C
# written and read once), from one small ncu capture of the dominant shape (the trailing update
# C -= P P^T, 8192 x 8192 lower, K = 512, S = 4, three launches).  The step's traffic per launch
# is this ratio times the step's compulsory bytes per launch (counted by the library for every
# launch).  Set to None when the kernel changes, until the capture is taken again.
GEMM_TRAFFIC_RATIO = 0.985
GEMM_TRAFFIC_PROFILE = "profiles/k_ozaki_gemm_syrk_8192x512_s4_traffic.md"


def _workload(rank, workload=BENCH_WORKLOAD):
    """The n = 16384 workload is the benchmark; the smaller ones exist only for profiling
    captures (a few GB on the device)."""
    from paper_2311_08050_gb300 import synth
    spec, thetas = synth.WORKLOADS[workload]()
    if rank:  # weak scaling: every rank evaluates its own FD batch (shifted centre)
        thetas = thetas + 0.01 * rank
    return spec, thetas


def _h2d_bytes(spec, thetas):
    b = spec.A.rowptr.nbytes + spec.A.col.nbytes + spec.A.val.nbytes + spec.y.nbytes + thetas.nbytes
    for blk in spec.blocks:
        if blk.points is not None:
            b += blk.points.nbytes
    return int(b)


def _pinned_copy(spec, thetas):
    """The spec's observation arrays, design, points and the theta batch copied into pinned
    (page-locked) host buffers."""
    import dataclasses
    import torch

    def pin(a):
        a = np.ascontiguousarray(a)
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0].copy()).dtype, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    from paper_2311_08050_gb300.synth import CSR
    A = CSR(spec.A.nrows, spec.A.ncols, pin(spec.A.rowptr), pin(spec.A.col), pin(spec.A.val))
    blocks = [dataclasses.replace(b, points=pin(b.points)) if b.points is not None else b for b in spec.blocks]
    ps = dataclasses.replace(spec, A=A, y=pin(spec.y), blocks=blocks,
                             offset=pin(spec.offset) if spec.offset is not None else None)
    return ps, pin(thetas)


def run_reference(args):
    """The FP64 CPU oracle on the host cores, one theta per step (bounded by --ref-budget)."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    from oracle import inla_oracle as O
    spec, thetas = _workload(0, args.workload)
    times = []
    t_start = time.time()
    k = 0
    while k < max(1, args.steps):
        t0 = time.perf_counter()
        O.evaluate(spec, thetas[k % len(thetas)])
        times.append(time.perf_counter() - t0)
        k += 1
        if time.time() - t_start > args.ref_budget:
            break
    value = len(times) / sum(times)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": 0, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n": spec.n, "m": spec.m, "batch": len(thetas),
                                            "parallelism": "host cores (numpy/scipy LAPACK)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "full oracle evaluation of one FD theta point per step (n=16384)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2311_08050_gb300 import build as B
    from paper_2311_08050_gb300 import inla
    B.build()
    L = inla.lib()
    L.inla_test_stats_read.argtypes = [C.POINTER(C.c_double)]
    L.inla_test_launch_count.restype = C.c_int64
    spec, thetas = _workload(rank, args.workload)
    nb = len(thetas)
    model = inla.Model(spec)
    stream = torch.cuda.Stream()
    sptr = C.c_void_p(stream.cuda_stream)
    n = spec.n
    xbuf = torch.empty((nb, n), dtype=torch.float64, device="cuda")
    vbuf = torch.empty((nb, n), dtype=torch.float64, device="cuda")
    xp = [xbuf[b].data_ptr() for b in range(nb)]
    vp = [vbuf[b].data_ptr() for b in range(nb)]
    kw = dict(precision=args.precision, slices=args.slices, newton_slices=args.newton_slices, stream=sptr,
              device_out=True, x_out=xp, var_out=vp, prior_slices=args.prior_slices, reuse_below=args.reuse_below,
              reuse_shrink=args.reuse_shrink, var_slices=args.var_slices, gram_slices=args.gram_slices)

    def step():
        lp, st, _, _ = inla.eval_batch([model], thetas, **kw)
        return lp, st

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    tuned = None
    if args.precision == "mixed" and args.autotune:
        # precision rungs calibrated on the FD centre against the six-slice evaluation (warm-up)
        from paper_2311_08050_gb300 import tune
        tr = tune.tune_precision(model, thetas[0], stream=sptr)
        kw.update(tr.opts())
        args.slices, args.newton_slices, args.prior_slices = tr.slices, tr.newton_slices, tr.prior_slices
        args.var_slices, args.gram_slices = tr.var_slices, tr.gram_slices
        tuned = {"prior_slices": tr.prior_slices, "gram_slices": tr.gram_slices, "slices": tr.slices,
                 "newton_slices": tr.newton_slices, "var_slices": tr.var_slices,
                 "errors_vs_six_slices": tr.errors, "tuning_seconds": round(tr.seconds, 2),
                 "tried": [t["setting"] for t in tr.tried]}
    for _ in range(max(1, args.warmup)):
        lp, st = step()
    assert np.all(st == 0), f"warm-up statuses {st.tolist()}"
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    launches_before = int(L.inla_test_launch_count())  # tuning + warm-up launches (ncu -s for the timed region)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            lp, st = step()
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    timed_launches = int(L.inla_test_launch_count())
    ms = ev0.elapsed_time(ev1)
    t_local = ms / 1e3
    from paper_2311_08050_gb300 import replicas
    t_max = replicas.max_over_ranks(t_local, world)
    value = world * nb * args.steps / t_max
    # ---------------- roofline of the dominant kernel (instrumented extra step) ----------------
    L.inla_test_stats_enable(1)
    L.inla_test_profile_enable(1)
    step()
    torch.cuda.synchronize()
    L.inla_test_stats_enable(0)
    L.inla_test_profile_enable(0)
    stats = (C.c_double * 5)()
    L.inla_test_stats_read(stats)
    # the instrumented step's Newton iterations (leading points, then followers): the largest step
    # over the points still iterating and whether the factor was computed afresh
    tr_steps, tr_ref = (C.c_double * 64)(), (C.c_int32 * 64)()
    L.inla_test_newton_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
    n_tr = min(64, int(L.inla_test_newton_trace(tr_steps, tr_ref, 64)))
    newton_trace = [{"step": float("%.3g" % tr_steps[i]), "refactored": int(tr_ref[i])} for i in range(n_tr)]
    pbuf = C.create_string_buffer(1 << 18)
    L.inla_test_profile_read_by_phase(pbuf, 1 << 18)
    phbuf = C.create_string_buffer(1 << 12)
    L.inla_test_phase_read(phbuf, 1 << 12)
    phases = []
    for line in phbuf.value.decode().splitlines():
        name, cnt, tot = line.split()
        phases.append({"phase": name, "ms": round(float(tot), 3)})
    by_kernel, by_phase = {}, {}
    for line in pbuf.value.decode().splitlines():
        key, cnt, tot = line.split()
        phase, name = key.split("/", 1)
        k = by_kernel.setdefault(name, [0, 0.0])
        k[0] += int(cnt)
        k[1] += float(tot)
        by_phase.setdefault(phase, []).append({"kernel": name, "launches": int(cnt), "ms": round(float(tot), 3)})
    breakdown = sorted(({"kernel": k, "launches": v[0], "ms": round(v[1], 3)} for k, v in by_kernel.items()),
                       key=lambda b: -b["ms"])
    phase_kernels = {ph: sorted(v, key=lambda b: -b["ms"])[:6] for ph, v in by_phase.items()}
    step_ms_prof = sum(b["ms"] for b in breakdown) or 1.0
    for b in breakdown:
        b["share"] = round(b["ms"] / step_ms_prof, 4)
    launches, alg, tens, kms, alg_bytes = stats[0], stats[1], stats[2], stats[3], stats[4]
    peaks, psrc = _peaks()
    peak_tc = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    tens_rate = tens / (kms / 1e3) / 1e12 if kms > 0 else None
    alg_rate = alg / (kms / 1e3) / 1e12 if kms > 0 else None
    # DRAM bytes per GEMM launch: the compulsory bytes of this step's launches (counted per launch
    # by the library) times the traffic ratio of the small ncu capture of the dominant shape
    alg_bytes_per_launch = alg_bytes / launches if launches else None
    traffic = GEMM_TRAFFIC_RATIO * alg_bytes_per_launch if (GEMM_TRAFFIC_RATIO and alg_bytes_per_launch) else None
    n_pad = ((spec.n + 255) // 256) * 256
    outer_block = {f"slices{sl}": int(L.inla_test_outer_block(n_pad, sl)) for sl in (args.newton_slices, args.slices)}
    outer_block["inverse"] = {f"slices{sl}": int(L.inla_test_inverse_block(n_pad, sl))
                              for sl in sorted({args.prior_slices or args.slices, args.var_slices or args.slices})}
    # achieved = the method's flops (2 x needed output elements x K per GEMM launch, i.e. the
    # Cholesky / inverse / product work itself) per second of GEMM time; the BF16 slice passes
    # the tensor pipe runs for them are reported separately
    roofline = {"bound": "tensor", "kernel": "k_ozaki_gemm<S> (tcgen05 BF16 slices)",
                "achieved": alg_rate, "peak": peak_tc, "unit": "TFLOP/s",
                "frac": (alg_rate / peak_tc) if alg_rate else None,
                "frac_algorithmic": (alg_rate / peak_tc) if alg_rate else None,
                "traffic": traffic,
                "traffic_unit": "bytes per launch (dram read + write)" if traffic else None,
                "traffic_source": (f"{GEMM_TRAFFIC_RATIO:.3f} x compulsory bytes per launch "
                                   f"({alg_bytes_per_launch:.4g}); ratio from {GEMM_TRAFFIC_PROFILE}")
                if traffic else "no capture of the current kernel",
                "tensor_pipe_tflops": tens_rate, "frac_tensor_pipe": (tens_rate / peak_tc) if tens_rate else None,
                "passes_per_flop": round(tens / alg, 2) if alg else None,
                "launches_per_step": int(launches), "kernel_ms_per_step": kms,
                "compulsory_bytes_per_step": alg_bytes,
                "peak_source": f"{psrc} bf16 sustained (kernel timed inside a long step), of measured"
                if psrc == "measured" else "fallback bf16 sustained"}
    # FP64 pipe peak, measured here by the library's FMA probe (no device setting changed)
    fp64_peak = C.c_double(0.0)
    fp32_peak = C.c_double(0.0)
    L.inla_test_fma_peak.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_double)]
    L.inla_test_fma_peak(0, 3, C.byref(fp64_peak))
    L.inla_test_fma_peak(1, 3, C.byref(fp32_peak))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": f"bf16 Ozaki slices x{args.prior_slices or args.slices} (prior factor and inverse) / "
                    f"x{args.gram_slices or args.prior_slices or args.slices} (prior precision W^T W) / x{args.slices} (final factor) / "
                    f"x{args.var_slices or args.slices} (its inverse: variances) / x{args.newton_slices} (Newton), "
                    "exact fp32 accumulation + df64 storage and diagonal tiles"
           if args.precision == "mixed" else "f64",
           "data": "synthetic (seeded; stands in for the paper's Poisson spatial workloads)",
           "config": {"workload": args.workload, "n": n, "m": spec.m, "theta_dim": spec.theta_dim, "batch": nb,
                      "precision": args.precision, "slices": args.slices, "newton_slices": args.newton_slices,
                      "prior_slices": args.prior_slices or args.slices,
                      "var_slices": args.var_slices or args.slices,
                      "gram_slices": args.gram_slices or args.prior_slices or args.slices,
                      "reuse_below": args.reuse_below or 0.1, "reuse_shrink": args.reuse_shrink or 0.25,
                      "l2": "inputs larger than L2 (2 GiB double-float matrices per theta)",
                      "outer_block_tuned": outer_block, "precision_tuned": tuned,
                      "parallelism": f"{world} GPU(s), theta batches sharded across ranks"},
           "clocks": clk.summary(), "roofline": roofline, "gpu_launches": None,
           "kernel_breakdown": breakdown[:12], "phase_breakdown": phases, "phase_kernels": phase_kernels,
           "newton_trace": newton_trace}
    # ---------------- end to end from host buffers ----------------
    if not args.no_e2e:
        # the step's inputs (observations, design, points, theta batch) in pinned host memory;
        # every step uploads them through the C ABI and reads the results back to the host
        pspec, pthetas = _pinned_copy(spec, thetas)
        e2e_steps = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            m2 = inla.Model(pspec)
            lp2, st2, xs2, vs2 = inla.eval_batch([m2], pthetas, precision=args.precision, slices=args.slices,
                                                 newton_slices=args.newton_slices, prior_slices=args.prior_slices,
                                                 reuse_below=args.reuse_below, reuse_shrink=args.reuse_shrink,
                                                 var_slices=args.var_slices, gram_slices=args.gram_slices)
            m2.close()
        t_e2e = time.perf_counter() - t0
        out["e2e"] = {"value": nb * e2e_steps / t_e2e * world, "unit": UNIT,
                      "h2d_bytes_per_step": _h2d_bytes(spec, thetas),
                      "d2h_bytes_per_step": int(nb * (2 * n * 8 + 8 + 4)), "steps": e2e_steps}
    # ---------------- FP64 GPU path on one theta (comparison) ----------------
    if not args.no_fp64 and args.precision == "mixed":
        t0 = time.perf_counter()
        x64 = torch.empty((1, n), dtype=torch.float64, device="cuda")
        v64 = torch.empty((1, n), dtype=torch.float64, device="cuda")
        lp64, st64, _, _ = inla.eval_batch([model], thetas[:1], precision="fp64", stream=sptr, device_out=True,
                                           x_out=[x64[0].data_ptr()], var_out=[v64[0].data_ptr()])
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        # the FP64 path refactors at every Newton iteration: its algorithmic flops are the prior
        # inversion (Cholesky, triangular inverse, W^T W: n_c^3), one n^3/3 Cholesky per
        # iteration plus the final one, and the triangular inverse for the variances (n^3/3)
        L.inla_test_newton_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
        iters64 = int(L.inla_test_newton_trace(None, None, 0))
        n_c = sum(b.size for b in spec.blocks if b.kind == "dense_exp")
        f64_flops = float(n_c) ** 3 + (iters64 + 1) * n ** 3 / 3.0 + n ** 3 / 3.0
        f64_rate = f64_flops / t64 / 1e12
        out["fp64"] = {"value": 1.0 / t64, "unit": UNIT, "thetas_timed": 1, "seconds": t64,
                       "log_post_theta0": float(lp64[0]), "status": int(st64[0]),
                       "mixed_minus_fp64_log_post": float(lp[0] - lp64[0]), "newton_iterations": iters64,
                       "algorithmic_tflop": f64_flops / 1e12}
        roofline["fp64"] = {"bound": "fp64 alu", "achieved": f64_rate, "peak": fp64_peak.value, "unit": "TFLOP/s",
                            "frac": f64_rate / fp64_peak.value if fp64_peak.value > 0 else None,
                            "what": "FP64 GPU path, whole theta evaluation: algorithmic flops / wall time",
                            "peak_source": "measured in this run by the library's DFMA probe (inla_test_fma_peak)"}
    roofline["fp32_fma_peak_tflops"] = fp32_peak.value
    # ---------------- FP64 CPU oracle on the host cores (rank 0) ----------------
    if rank == 0 and not args.no_cpu:
        from oracle import inla_oracle as O
        t0 = time.perf_counter()
        r = O.evaluate(spec, thetas[0])
        tc = time.perf_counter() - t0
        x_mixed = xbuf[0].cpu().numpy()
        v_mixed = vbuf[0].cpu().numpy()
        out["cpu_baseline"] = {"value": 1.0 / tc, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                               "sample": "one full oracle evaluation (theta = FD centre) of the n=16384 workload"}
        out["error_vs_oracle"] = {"log_post_abs": abs(float(lp[0]) - r["log_post"]),
                                  "x_hat_rel": float(np.max(np.abs(x_mixed - r["x_hat"])) /
                                                     max(1.0, np.max(np.abs(r["x_hat"])))),
                                  "var_rel": float(np.max(np.abs(v_mixed / r["var"] - 1.0))),
                                  "theta": "FD centre", "tolerance": {"log_post_abs": 1e-3, "var_rel": 1e-4}}
    out["gpu_launches"] = timed_launches
    out["config"]["launches_before_timed_region"] = launches_before
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_gemm(args):
    """Microbenchmark of the Ozaki GEMM alone (test hook): tensor-pipe and algorithmic rates
    for the shapes given as M,N,K,S[,lower] separated by ';'."""
    from paper_2311_08050_gb300 import build as B
    from paper_2311_08050_gb300 import inla
    B.build()
    L = inla.lib()
    P = C.POINTER(C.c_double)
    L.inla_test_ozaki_gemm.argtypes = [P, P, P] + [C.c_int32] * 8 + [C.c_double, C.c_double]
    L.inla_test_stats_read.argtypes = [C.POINTER(C.c_double)]
    peaks, _ = _peaks()
    rng = np.random.default_rng(0)
    res = []
    for spec in args.gemm.split(";"):
        f = [int(x) for x in spec.split(",")]
        M, N, K, S = f[:4]
        lower = f[4] if len(f) > 4 else 0
        accumulate = f[5] if len(f) > 5 else 0    # C = C - A B^T instead of C = A B^T
        A = rng.standard_normal((M, K))
        Bm = rng.standard_normal((N, K))
        Cm = np.zeros((M, N))
        for rep in range(3):
            L.inla_test_stats_enable(1 if rep == 2 else 0)
            rc = L.inla_test_ozaki_gemm(A.ctypes.data_as(P), Bm.ctypes.data_as(P), Cm.ctypes.data_as(P), M, N, K, S,
                                        0, 0, lower, 0, 1.0 if accumulate else 0.0, -1.0 if accumulate else 1.0)
            assert rc == 0
        L.inla_test_stats_enable(0)
        st = (C.c_double * 5)()
        L.inla_test_stats_read(st)
        ms = st[3]
        tens = st[2] / (ms / 1e3) / 1e12
        alg_t = st[1] / (ms / 1e3) / 1e12
        res.append({"M": M, "N": N, "K": K, "S": S, "lower": lower, "accumulate": accumulate, "ms": ms,
                    "alg_tflops": alg_t, "frac_algorithmic_bf16_burst": alg_t / peaks["bf16_tflops"],
                    "tensor_tflops": tens, "frac_tensor_pipe_bf16_burst": tens / peaks["bf16_tflops"],
                    "compulsory_bytes": st[4], "compulsory_gbs": st[4] / (ms / 1e3) / 1e9})
    print(json.dumps({"gemm_microbench": res}), flush=True)


def run_surrogate(args):
    """The learned-surrogate experiment on the n = 16384 model (surrogate.experiment): exact
    FD-BFGS on the mixed path against the surrogate trained on --train exact mixed evaluations,
    every exact evaluation counted; the FP64 path's time to the mode is estimated from one
    measured FP64 evaluation times the points the exact search needed."""
    import torch
    from paper_2311_08050_gb300 import build as B
    from paper_2311_08050_gb300 import inla, surrogate, synth
    B.build()
    torch.cuda.set_device(0)
    spec, _ = synth.WORKLOADS[args.workload]()
    th_true = synth.poisson_n16384_theta_true() if args.workload == BENCH_WORKLOAD else _[0]
    model = inla.Model(spec)
    chunk = args.surrogate_batch

    def exact_eval(thetas):
        out = []
        for c in range(0, len(thetas), chunk):
            lp, st, _, _ = inla.eval_batch([model], thetas[c:c + chunk], want_x=False, want_var=False,
                                           precision="mixed")
            out.append(np.where(np.asarray(st) == 0, lp, -np.inf))
        return np.concatenate(out)

    exact_eval(th_true[None, :])  # warm-up (tuner, graphs)
    th0 = th_true + np.array([0.6, -0.5, 0.4, -0.6])[:len(th_true)]
    res = surrogate.experiment(exact_eval, th_true, th0, n_train=args.train, n_holdout=args.holdout)
    t0 = time.perf_counter()
    lp64, st64, _, _ = inla.eval_batch([model], th_true[None, :], want_x=False, want_var=False, precision="fp64")
    t64 = time.perf_counter() - t0
    res["fp64"] = {"seconds_per_theta": t64, "status": int(st64[0]),
                   "time_to_mode_estimated_s": t64 * res["exact_search"]["points"],
                   "how": "one FP64 evaluation timed here x the exact points of the FD-BFGS search"}
    res["config"] = {"workload": args.workload, "n": spec.n, "m": spec.m, "theta_dim": spec.theta_dim,
                     "train": args.train, "holdout": args.holdout, "batch": chunk, "precision": "mixed (5/4 slices)",
                     "start": "theta_true + (0.6, -0.5, 0.4, -0.6)"}
    print(json.dumps({"surrogate_experiment": res}), flush=True)


_ORACLE_TIMER = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
from paper_2311_08050_gb300 import synth
from oracle import inla_oracle as O
w = synth.WORKLOADS[sys.argv[2]]()
specs, thetas = w
if not isinstance(specs, list):
    specs = [specs] * len(thetas)
k = int(sys.argv[3])
t0 = time.perf_counter()
for b in range(k):
    O.evaluate(specs[b], thetas[b])
print(json.dumps({"seconds": time.perf_counter() - t0, "points": k}))
"""


def _time_oracle(workload, points, cores):
    """The oracle on `points` theta points of a workload in a child process limited to `cores`
    BLAS / OpenMP threads (None: all host cores)."""
    env = dict(os.environ)
    if cores:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[v] = str(cores)
    r = subprocess.run([sys.executable, "-c", _ORACLE_TIMER, ROOT, workload, str(points)], capture_output=True,
                       text=True, env=env, timeout=3600)
    if r.returncode != 0:
        return {"error": r.stderr.strip()[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"theta_evals_per_s": d["points"] / d["seconds"], "points": d["points"], "seconds": d["seconds"],
            "cores": cores or os.cpu_count()}


def run_configs(args):
    """theta-evals/s of every workload of the scope table: the GPU mixed path (precision tuned
    per workload) and FP64 path on the whole batch (or the first points at n >= 8192), and the
    FP64 oracle on the host cores (all cores; one core where a point takes at most a minute)."""
    import torch
    from paper_2311_08050_gb300 import build as B
    from paper_2311_08050_gb300 import inla, synth, tune
    B.build()
    torch.cuda.set_device(0)
    rows = []
    plan = [("poisson_n256_m1000_5pts", 5, 5, 5, 5), ("poisson_n4096_m20000_fd7", 7, 7, 2, 1),
            ("spacetime_n8149_m8000_fd13", 13, 1, 1, 0), ("gaussian_64_models_n512_4096", 64, 64, 8, 4),
            ("poisson_n16384_m100000_fd9", 9, 1, 1, 0)]
    for name, n_mixed, n_fp64, n_orc, n_orc1 in plan:
        specs, thetas = synth.WORKLOADS[name]()
        multi = isinstance(specs, list)
        models = [inla.Model(s) for s in specs] if multi else [inla.Model(specs)]
        mot = np.arange(len(models), dtype=np.int32) if multi else None

        def run(k, **kw):
            sub = thetas[:k]
            return inla.eval_batch(models, sub, model_of_theta=None if mot is None else mot[:k], **kw)

        row = {"workload": name, "batch": len(thetas)}
        tuned = tune.tune_precision(models[0], thetas[0]) if not multi else None
        kw = tuned.opts() if tuned else {}
        run(n_mixed, precision="mixed", **kw)  # warm-up (outer-block tuner, graphs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lp, st, _, _ = run(n_mixed, precision="mixed", **kw)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        row["gpu_mixed"] = {"theta_evals_per_s": n_mixed / tm, "points": n_mixed, "seconds": tm,
                            "statuses_ok": bool(np.all(st == 0)),
                            "slices": tuned.opts() if tuned else "5/5/4 (default; 64 models, not tuned)"}
        if n_fp64 > 1:
            run(min(n_fp64, 2), precision="fp64")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lp64, st64, _, _ = run(n_fp64, precision="fp64")
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        row["gpu_fp64"] = {"theta_evals_per_s": n_fp64 / t64, "points": n_fp64, "seconds": t64,
                           "statuses_ok": bool(np.all(st64 == 0))}
        row["mixed_minus_fp64_log_post_max"] = float(np.max(np.abs(lp[:n_fp64] - lp64))) if n_fp64 <= n_mixed else None
        row["oracle_all_cores"] = _time_oracle(name, n_orc, None)
        if n_orc1:
            row["oracle_one_core"] = _time_oracle(name, n_orc1, 1)
        for m in models:
            m.close()
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"configs": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--slices", type=int, default=5, help="slices of the factor at the mode")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the given slice counts instead of the autotuned rungs")
    ap.add_argument("--newton-slices", type=int, default=4, help="slices of the Newton-step factorisations")
    ap.add_argument("--prior-slices", type=int, default=0, help="slices of the prior inversion (0: --slices)")
    ap.add_argument("--gram-slices", type=int, default=0,
                    help="slices of the prior precision W^T W (0: --prior-slices)")
    ap.add_argument("--var-slices", type=int, default=0,
                    help="slices of the inverse of the factor at the mode, for the variances (0: --slices)")
    ap.add_argument("--reuse-below", type=float, default=0.0, help="modified Newton: reuse a factor once steps are "
                    "below this (0: library default)")
    ap.add_argument("--reuse-shrink", type=float, default=0.0, help="modified Newton: keep a factor while steps "
                    "shrink at least by this ratio (0: library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=150.0)
    ap.add_argument("--workload", default=BENCH_WORKLOAD, choices=(BENCH_WORKLOAD,) + CAPTURE_WORKLOADS,
                    help="the benchmark workload (default) or a smaller case for profiling captures")
    ap.add_argument("--gemm", default=None, help="microbenchmark the Ozaki GEMM: 'M,N,K,S[,lower[,accumulate]];...'")
    ap.add_argument("--surrogate", action="store_true", help="the learned-surrogate experiment (time to the mode)")
    ap.add_argument("--configs", action="store_true", help="theta-evals/s of every workload: GPU mixed, GPU FP64, "
                    "oracle on all host cores and on one")
    ap.add_argument("--train", type=int, default=2000, help="--surrogate: exact training evaluations")
    ap.add_argument("--holdout", type=int, default=200, help="--surrogate: held-out exact evaluations")
    ap.add_argument("--surrogate-batch", type=int, default=16, help="--surrogate: points per batched call")
    args = ap.parse_args()
    if args.gemm:
        run_gemm(args)
        return
    if args.surrogate:
        run_surrogate(args)
        return
    if args.configs:
        run_configs(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
