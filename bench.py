"""Benchmark of the FDM layer-case time step on GB300 (cell-steps/s).

Workload (default): coupled FDM under loading on a 2048 x 2048 periodic grid -- seeded
zero-mean Gaussian random U13 field (correlation length 16 cells, RMS |alpha| 0.1),
stress-driven velocity with M = 1, E = 1, nu = 0.3, macroscopic shear strain ramped by 1e-4
per step, adaptive CFL 0.4 time step, minmod limiter.  One "step" = static FFT solve +
celerity + time-step reduction + KNP transport update (the whole hot path).

Timing: inputs resident in HBM; the L2 is flushed (256 MiB write) before every timed step
and each step is timed with CUDA events on the library's stream, phase by phase, so the
dominant kernel's duration is measured in the same run.  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n 2048] [--precision fp64|mixed]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDM cell-steps/s (FFT stress + Godunov transport), %HBM roofline; p50/p99 serve"
UNIT = "cell-steps/s"
PHASES = ["row_forward", "col_pass", "row_inverse", "knp_step"]
FALLBACK_HBM_GBS = 6800.0
FP64_HBM_TARGET_FRAC = 0.6   # target fraction of the HBM roofline for the FP64 path at 2048^2


def workload_params(n, precision):
    from paper_1911_03225_gb300.binding import Params, V_STRESS, LOAD_STRAIN_RAMP, FP64, MIXED, DF64
    return Params(n1=n, n2=n, velocity_mode=V_STRESS, mobility=1.0, loading_mode=LOAD_STRAIN_RAMP,
                  eps_bar13_rate=1e-4, cfl=0.4, theta=1.0, E=1.0, nu=0.3,
                  precision={"mixed": MIXED, "df64": DF64}.get(precision, FP64))


def workload_input(n, seed):
    from paper_1911_03225_gb300 import inputs
    return inputs.random_up(n, seed=seed, ell=16.0, rms_alpha=0.1)


def bytes_per_cell(elt, pair=False):
    """Algorithmic HBM bytes per cell and launch of each kernel (one read + one write of
    every array the kernel must touch; halo re-reads and tables excluded).  `pair`: the
    state is a pair of FP32 words (mixed precision), read and written whole by the stencil."""
    w = 2 if pair else 1
    return {"row_forward": 2 * elt,           # read U13 (high word), write half spectrum
            "col_pass": 2 * elt,              # read + write the half spectrum in place
            "row_inverse": 2 * elt,           # read half spectrum, write tau13
            "knp_step": (2 * w + 1) * elt}    # read U13 and tau13, write U13^{n+1}


# Algorithmic floating-point operations per node of the KNP update (Steps 1-4 as knp_node in
# fdm_device.cuh evaluates them; add, subtract and multiply 1, multiply-add 2, reciprocal
# and reciprocal square root 1; comparisons, min, max and sign flips 0):
#   first differences 8; limited second differences 20; one-sided derivatives 8;
#   one-sided speeds (three |(p,q)|^-1 and four products) 19; projection weights 4;
#   v0 dt and v0 dt / 2 2; the row and column quadratics of the two sides 20 + 20;
#   four corners of 36 (mixed difference 3, value 5, gradient 4, midpoint predictor 15,
#   |grad| 5, Psi and its weight 4) 144; projection 5.  Total 250, of which 11 reciprocal
#   square roots and one reciprocal.
KNP_FLOPS_PER_CELL = 250


KERNEL_SOURCES = ["fdm_kernels.cu", "fdm_device.cuh", "fdm_df.cuh", "fdm_internal.h"]


def kernel_source_hash():
    """sha256 (first 16 hex) of the step kernels' CUDA sources; profile figures are valid
    only for it."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1911_03225_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, precision, n):
    """DRAM bytes per launch of `kernel` from the committed ncu summaries under profiles/,
    or None when absent or taken on different kernel sources."""
    import glob
    sha = kernel_source_hash()
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(f):
            if not line.startswith("traffic:"):
                continue
            kv = dict(x.split("=", 1) for x in line.split()[1:])
            if (kv.get("kernel") == kernel and kv.get("precision") == precision and int(kv.get("n", 0)) == n
                    and kv.get("source") == sha):
                return int(kv["bytes"])
    return None


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_bandwidth_gbs", "copy_gbs"):
                if k in d:
                    return float(d[k]), "measured (MEASURED_PEAKS.json %s)" % k
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def measured_arith_peaks(local):
    """FP64, FP32 and double-word multiply-add rates of this GPU, measured now by the
    library's FMA-chain kernel (fdm_measure_arith_rate), with the SM clock sampled meanwhile."""
    from paper_1911_03225_gb300 import binding as B
    with ClockSampler(local) as clk:
        out = {"fp64": B.measure_arith_rate(B.FP64), "fp32": B.measure_arith_rate(B.MIXED),
               "df64": B.measure_arith_rate(B.DF64)}
    out = {k: round(v, 1) for k, v in out.items()}
    out["unit"] = "GFLOP/s (multiply-add = 2)"
    out["clocks"] = clk.summary()
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    from paper_1911_03225_gb300.replicas import init_replicas
    return init_replicas()


def max_over_ranks(x, world):
    from paper_1911_03225_gb300.replicas import max_over_ranks as mor
    return mor(x, world)


def barrier(world):
    from paper_1911_03225_gb300.replicas import barrier as bar
    bar(world)


def build_once(rank, world):
    """Rank 0 builds the library first; the others then find it up to date."""
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    __graft_entry__.build()


def time_steps(sim, steps, flush, stream):
    """Whole steps through the library's step call (one replay of the captured step per step),
    CUDA events around each step on the library's stream, L2 flushed before each step."""
    import torch
    evs = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.enqueue_steps(1)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    sim.sync()
    return sum(a.elapsed_time(b) for a, b in evs)


def time_device(sim, steps, flush, stream):
    """Per-step, per-phase CUDA-event timing with an L2 flush before each step (the kernels
    are enqueued one by one, an event between each two)."""
    import torch
    evs = []
    torch.cuda.nvtx.range_push("fdm_timed")   # lets ncu capture exactly the timed launches
    for _ in range(steps):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(len(PHASES) + 1)]
        e[0].record(stream)
        for ph in range(len(PHASES)):
            sim.enqueue_phase(ph)
            e[ph + 1].record(stream)
        evs.append(e)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    sim.sync()
    per_phase = {p: [] for p in PHASES}
    total = 0.0
    for e in evs:
        total += e[0].elapsed_time(e[-1])
        for i, p in enumerate(PHASES):
            per_phase[p].append(e[i].elapsed_time(e[i + 1]))
    return total, per_phase


def run_ours(args, world, rank, local):
    import torch
    import __graft_entry__
    from paper_1911_03225_gb300 import FDM

    build_once(rank, world)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n, K, W = args.n, args.steps, args.warmup
    cells = n * n
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    hbm_peak, peak_src = read_peaks()
    peaks = measured_arith_peaks(local)
    up0 = workload_input(n, seed=rank)

    results = {}
    for prec in ([args.precision] if args.precision != "all" else ["fp64", "df64", "mixed"]):
        p = workload_params(n, prec)
        sim = FDM(p, stream=stream.cuda_stream)
        sim.set_plastic_distortion(up0)
        for _ in range(W):
            flush.zero_()
            sim.enqueue_steps(1)
        sim.sync()
        barrier(world)
        with ClockSampler(local) as clk:
            barrier(world)
            total_ms = time_steps(sim, K, flush, stream)
            barrier(world)
            phased_ms, per_phase = time_device(sim, K, flush, stream)
            barrier(world)
        info = sim.info()
        t_max = max_over_ranks(total_ms, world)
        elt = 4 if prec == "mixed" else 8
        phase_mean = {ph: sum(v) / len(v) for ph, v in per_phase.items()}
        dom = max(phase_mean, key=phase_mean.get)
        bpc = bytes_per_cell(elt, pair=(prec == "mixed"))
        results[prec] = {"total_ms": t_max, "phased_ms": phased_ms, "phase_ms": phase_mean, "dominant": dom,
                         "clocks": clk.summary(), "info": info, "bpc": bpc, "sim": sim,
                         "launch": sim.launch_config()}

    primary = args.precision if args.precision != "all" else "fp64"
    r = results[primary]
    value = cells * K * world / (r["total_ms"] / 1e3)

    def roofline(prec, rr):
        """Roofline of the step's dominant kernel: the stencil against the measured multiply-add
        rate of its arithmetic (it is bound by arithmetic, not by HBM), the transforms
        against the HBM peak."""
        d = rr["dominant"]
        d_ms = rr["phase_ms"][d]
        hbm_gbs = rr["bpc"][d] * cells / (d_ms / 1e3) / 1e9
        if d == "knp_step":
            key = {"fp64": "fp64", "df64": "df64", "mixed": "fp32"}[prec]
            rl = {"bound": "alu", "achieved": KNP_FLOPS_PER_CELL * cells / (d_ms / 1e3) / 1e9, "peak": peaks[key],
                  "unit": "GFLOP/s", "flops_per_cell": KNP_FLOPS_PER_CELL,
                  "peak_source": "measured in this run (of measured): %s multiply-add chains on every SM, "
                                 "fdm_measure_arith_rate, SM clock %s MHz" % (
                                     {"fp64": "FP64", "fp32": "FP32", "df64": "double-word"}[key],
                                     peaks["clocks"].get("sm_mhz"))}
        else:
            rl = {"bound": "hbm", "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "peak_source": peak_src}
        rl["frac"] = rl["achieved"] / rl["peak"]
        rl["kernel"] = d
        rl["traffic"] = profiled_traffic(d, prec, n)
        rl["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, from the committed "
                                "profile summary (profiles/*.md) taken on the same kernel sources; not measured "
                                "in this run" if rl["traffic"] is not None else
                                "no committed profile of the current kernel sources")
        rl["algorithmic_bytes"] = rr["bpc"][d] * cells
        rl["hbm_GBs"] = hbm_gbs
        rl["hbm_frac"] = hbm_gbs / hbm_peak
        step_gbs = sum(rr["bpc"].values()) * cells / (rr["total_ms"] / K / 1e3) / 1e9
        rl["hbm_frac_of_step"] = step_gbs / hbm_peak
        return rl

    roof = roofline(primary, r)
    if primary == "fp64":
        roof["fp64_hbm_target"] = {
            "target_frac": FP64_HBM_TARGET_FRAC, "achieved_frac": roof["hbm_frac_of_step"],
            "met": roof["hbm_frac_of_step"] >= FP64_HBM_TARGET_FRAC,
            "why": "the FP64 step is bound by the FP64 pipe, not by HBM: its %d B per cell take %.0f us of HBM "
                   "time at the peak, its stencil alone %.0f us of FP64 multiply-adds at the measured rate" % (
                       sum(r["bpc"].values()), sum(r["bpc"].values()) * cells / hbm_peak / 1e3,
                       KNP_FLOPS_PER_CELL * cells / peaks["fp64"] / 1e3)}

    # end to end through the public API with host buffers in pinned memory (rank-local)
    sim = r["sim"]
    up_host = torch.empty(up0.shape, dtype=torch.float64, pin_memory=True).numpy()
    up_host[...] = up0
    out_host = {"up13": torch.empty(up0.shape, dtype=torch.float64, pin_memory=True).numpy()}
    barrier(world)
    t0 = time.perf_counter()
    sim.set_plastic_distortion(up_host)
    for _ in range(K):
        sim.step(1, info=True)
    out = sim.read_fields("up13", out=out_host)
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, world)
    e2e = {"value": cells * K * world / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": cells * 8 / K, "d2h_bytes_per_step": 104 + cells * 8 / K,
           "note": "per step: fdm_step(1) with the step's scalars read back; the initial U13 upload and "
                   "final U13 download (pinned host arrays) are amortised over the K steps"}
    assert np.isfinite(out["up13"]).all()

    extra = {}
    for prec, rr in results.items():
        extra[prec] = {"value": cells * K * world / (rr["total_ms"] / 1e3),
                       "ms_per_step": rr["total_ms"] / K,
                       "ms_per_step_phased": rr["phased_ms"] / K,
                       "phase_ms": {k: round(v, 5) for k, v in rr["phase_ms"].items()},
                       "roofline": roofline(prec, rr), "launch": rr["launch"],
                       "t_end": rr["info"].t, "clocks": rr["clocks"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": r["total_ms"] / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if primary == "fp64" else "f32 (FP64 scalars)",
            "data": "synthetic (seeded random U13 field; no dataset in the paper)",
            "config": {"workload": "coupled FDM under loading, %dx%d periodic layer, random field l=16 "
                                   "RMS|alpha|=0.1, M=1, E=1, nu=0.3, strain ramp 1e-4/step, CFL 0.4, "
                                   "minmod" % (n, n),
                       "n": n, "precision": primary, "l2": "flushed (256 MiB write) before every timed step",
                       "timing": "ms_per_step: K whole steps through fdm_enqueue_steps(1) (the captured step "
                                 "replayed), CUDA events around each step; phase_ms: a second pass of K steps "
                                 "with the four kernels enqueued one by one and an event between each two "
                                 "(ms_per_step_phased)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "launch": r["launch"]},
            "roofline": roof,
            "clocks": r["clocks"],
            "e2e": e2e,
            "gpu_launches": len(PHASES) * K,
            "precisions": extra,
        }
        import torch
        line["fft_comparison"] = {
            "note": "static solve (rows, K multiply with the xi = 0 loading, inverse) of this library vs the same "
                    "transform pair through cuFFT (torch.fft.rfft2 / irfft2 with one multiply), both L2-cold; "
                    "cuFFT is a timing comparison only",
            "ours_ms": {p_: round(sum(v["phase_ms"][k_] for k_ in PHASES[:3]), 5) for p_, v in extra.items()},
            "cufft_ms": {"fp64": round(cufft_static_solve_ms(n, torch.float64), 5),
                         "mixed": round(cufft_static_solve_ms(n, torch.float32), 5)}}
        # the mixed path's iterates stop improving at FP32 rounding (~1e-7)
        line["hetero_static"] = {"fp64": hetero_static(n, "fp64", tol=1e-12),
                                 "mixed": hetero_static(n, "mixed", tol=1e-6),
                                 "fp64_thin_layer": hetero_layer_static(512)}
    for rr in results.values():
        rr["sim"].close()
    if args.sub_records:
        # configurations 4 and 5 on the same GPU, in the same run (every rank, weak scaling)
        batched = batched_record(world, rank, local, args.instances, max(K, 100), W)
        served = serve_record(world, rank, local, args.sub_serve_requests, 100, args.sub_serve_max_steps,
                              args.serve_slots, args.serve_tick)
    if rank == 0:
        if args.sub_records:
            line["batched"] = batched
            line["serve"] = served
        if args.cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)


def hetero_static(n, precision, tol=1e-12, contrast=4.0):
    """Heterogeneous static problem (shear-modulus field of the given contrast, plastic layer
    filling the cell, stress control) on the n x n random field: iterations to the tolerance
    and wall time of one converged solve through the public call (after one untimed solve).
    One iteration moves 32 field words per cell, 33 with the mixed path's low words
    (polarisation 6, four transforms 16, Green operator 4, update 6): 256 B in FP64."""
    import torch
    from paper_1911_03225_gb300 import FDM, inputs
    from paper_1911_03225_gb300 import binding as B
    p = B.Params(n1=n, n2=n, nz=8, nh=8, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.01,
                 precision={"fp64": B.FP64, "mixed": B.MIXED}[precision])
    up0 = inputs.random_up(n, seed=0, ell=16.0, rms_alpha=0.1)
    f = inputs.modulus_factor(n, n, seed=1, lo=1.0 / contrast, hi=1.0, ell=24.0)
    def timed(**kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = sim.static_solve_heterogeneous(f, **kw)
        return (time.perf_counter() - t0) * 1e3, out

    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        sim.static_solve_heterogeneous(f, tol=tol, max_iter=400)
        ms, (_, _, it, res) = timed(tol=tol, max_iter=400)
        # one iteration alone: the difference of two fixed-length solves (the modulus upload,
        # validation and the field's moments are per solve)
        t10, _ = timed(tol=0.0, max_iter=10)
        t30, _ = timed(tol=0.0, max_iter=30)
    per_it = (t30 - t10) / 20.0
    bpc = 8 * 32 if precision == "fp64" else 4 * 33
    return {"n": n, "contrast": contrast, "tol": tol, "iterations": it,
            "residual": res, "ms": round(ms, 3), "ms_per_iteration": round(per_it, 4),
            "bytes_per_cell_iteration": bpc,
            "achieved_GBs_per_iteration": round(float(bpc) * n * n / (per_it / 1e3) / 1e9, 1)}


def cufft_static_solve_ms(n, dtype, reps=20):
    """Timing comparison only (never on the result path): the same static solve -- real 2-D
    FFT, multiply by a real symbol, inverse -- through torch.fft (cuFFT) on an n x n field of
    `dtype`, with the L2 flushed before each repetition like the timed steps."""
    import torch
    dev = torch.device("cuda")
    u = torch.randn(n, n, dtype=dtype, device=dev)
    k = torch.rand(n, n // 2 + 1, dtype=dtype, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        torch.fft.irfft2(torch.fft.rfft2(u) * k, s=(n, n))
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        torch.fft.irfft2(torch.fft.rfft2(u) * k, s=(n, n))
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def oracle_sample(seconds, threads, n=512, steps=None):
    """The FP64 oracle as it stands on a bounded sample of the workload: the same coupled
    configuration on an n x n grid (the layer-kernel precompute excluded), stepped until
    about `seconds` of wall time have passed (or exactly `steps` steps), its loops over
    independent rows and nodes on `threads` host threads (< 1: every core; the results are
    the same for every count).  Returns (cell-steps/s, steps, seconds, threads used)."""
    import oracle
    prev = oracle.threads()
    used = oracle.set_threads(threads)
    try:
        p = workload_params(n, "fp64")
        op = oracle.Params(**{k: getattr(p, k) for k in oracle.Params.__dataclass_fields__})
        K = oracle.kernel_table(n, n, n, p.nh, p.E / (2 * (1 + p.nu)), p.nu)
        st = oracle.State(up13=workload_input(n, seed=0).copy())
        t0 = time.perf_counter()
        k = 0
        while (steps is None and (time.perf_counter() - t0 < seconds or k < 2)) or (steps is not None and k < steps):
            st, rc = oracle.run(op, None, 1, K=K, state=st)
            k += 1
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(prev)
    return n * n * k / dt, k, dt, used


def cpu_baseline(seconds):
    """The oracle timed on the host's cores (every core, and one thread), a reported
    baseline beside the GPU numbers."""
    v_all, k_all, t_all, used = oracle_sample(seconds, 0)
    v_one, k_one, t_one, _ = oracle_sample(seconds, 1)
    return {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle", "nproc": os.cpu_count(),
            "sample": "coupled random-field workload on a 512x512 grid (bounded sample of the 2048x2048 workload), "
                      "%d steps (%.1f s) on %d threads, layer-kernel precompute excluded" % (k_all, t_all, used),
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": "the same, %d steps (%.1f s) on one thread" % (k_one, t_one)}}


def batched_workload(count=256, rank=0):
    """Configuration 4: `count` independent coupled instances, side drawn per seed from
    {64, 128, 256, 512}, random field (l = 16, RMS |alpha| = 0.1) with the instance's seed;
    each rank gets its own seeds."""
    from paper_1911_03225_gb300.replicas import instance_seeds
    sizes = [64, 128, 256, 512]
    out = []
    for i in instance_seeds(count, rank):
        n = sizes[int(np.random.default_rng(i).integers(4))]
        out.append((n, workload_input(n, seed=i)))
    return out


def batched_record(world, rank, local, count, K, W):
    """Configuration 4 measured: `count` instances in one batch (mixed precision, one launch
    per kernel and size class, steps replayed from CUDA graphs), K timed steps after W; then
    the plain per-instance FP64 form of a sample of the same instances on the same GPU, and
    the mixed results' error against it."""
    import torch
    from paper_1911_03225_gb300 import Batch, FDM
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    inst = batched_workload(count, rank)
    cells = sum(n * n for n, _ in inst)
    params = [workload_params(n, "mixed") for n, _ in inst]
    with Batch(params, stream=stream.cuda_stream) as b:
        for i, (n, up) in enumerate(inst):
            b.set_plastic_distortion(i, up)
            b.set_budget(i, W + K)
        b.enqueue_steps(W)
        b.sync()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            barrier(world)
            torch.cuda.nvtx.range_push("fdm_timed")
            e0.record(stream)
            b.enqueue_steps(K)
            e1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            barrier(world)
        left = b.sync()
        assert (left == 0).all()
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        launches = b.launches_per_step() * K
        sample = list(range(0, len(inst), max(1, len(inst) // 8)))[:8]
        mixed_out = {i: b.read_fields(i, "up13")["up13"] for i in sample}
        # trial: the same steps as one persistent cooperative launch (all phases of all size
        # classes, grid barriers between phases) against the graph-replayed launches above
        for i in range(len(inst)):
            b.set_budget(i, W + K)
        b.enqueue_steps_persistent(W)
        b.sync()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        b.enqueue_steps_persistent(K)
        p1.record(stream)
        torch.cuda.synchronize()
        assert (b.sync() == 0).all()
        ms_persist = max_over_ranks(p0.elapsed_time(p1), world)
    # the plain per-instance FP64 form on the same GPU: one handle per instance, stepped alone
    fp64_cells, fp64_ms, errs = 0, 0.0, []
    for i in sample:
        n, up = inst[i]
        with FDM(workload_params(n, "fp64"), stream=stream.cuda_stream) as sim:
            sim.set_plastic_distortion(up)
            sim.enqueue_steps(W)
            sim.sync()
            e0.record(stream)
            sim.enqueue_steps(K)
            e1.record(stream)
            sim.sync()
            fp64_ms += e0.elapsed_time(e1)
            fp64_cells += n * n
            ref = sim.read_fields("up13")["up13"]
        errs.append(float(np.linalg.norm(mixed_out[i] - ref) / np.linalg.norm(ref)))
    value = cells * K * world / (ms / 1e3)
    plain = fp64_cells * K / (fp64_ms / 1e3)
    return {"value": value, "unit": UNIT, "steps": K, "warmup": W, "ms_per_step": ms / K,
            "workload": "batched uneven instances: %d coupled simulations, side per seed in {64,128,256,512}, "
                        "mixed precision, one batched launch per kernel and size class, CUDA-graph steps" % len(inst),
            "instances": len(inst), "cells_per_step": cells,
            "l2": "working set %.0f MB > L2" % (cells * 4 * 5 / 1e6),
            "gpu_launches": launches, "clocks": clk.summary(),
            "plain_fp64_per_instance": {"value": plain, "unit": UNIT, "sample_instances": len(sample)},
            "persistent_trial": {"ms_per_step": ms_persist / K, "value": cells * K * world / (ms_persist / 1e3),
                                 "over_graph": ms / ms_persist, "launches": 1,
                                 "form": "one cooperative launch for all K steps: the four phases of every size "
                                         "class, grid barriers between phases (fdm_batch_enqueue_steps_persistent)"},
            "batched_mixed_over_plain_fp64": value / world / plain,
            "mixed_vs_fp64_rel_l2": {"max": max(errs), "mean": sum(errs) / len(errs), "after_steps": W + K,
                                     "stated_tolerance": 1e-5}}


def run_batched(args, world, rank, local):
    build_once(rank, world)
    rec = batched_record(world, rank, local, args.instances, args.steps, args.warmup)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 scalars)", "data": "synthetic (seeded random U13 fields)",
            "config": {"workload": rec["workload"], "cells_per_step": rec["cells_per_step"], "l2": rec["l2"]},
            "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
            "plain_fp64_per_instance": rec["plain_fp64_per_instance"],
            "mixed_vs_fp64_rel_l2": rec["mixed_vs_fp64_rel_l2"],
            "persistent_trial": rec["persistent_trial"],
        }), flush=True)


def serve_record(world, rank, local, R, min_steps, max_steps, slots, tick, group_size=8):
    """Configuration 5 measured: R Poisson arrivals (200 req/s, seeded), side uniform in
    {64, ..., 1024}, steps uniform in [min_steps, max_steps], half FP64 and half mixed, served
    under a 150 GB HBM budget with `slots` resident simulations per class at most."""
    import torch
    from paper_1911_03225_gb300.binding import FP64, MIXED
    from paper_1911_03225_gb300.serve import Request, Server, poisson_arrivals
    torch.cuda.set_device(local)
    rng = np.random.default_rng(1234 + rank)
    sizes = [64, 128, 256, 512, 1024]
    arr = poisson_arrivals(200.0, R, seed=77 + rank)
    reqs = []
    for k in range(R):
        n = int(rng.choice(sizes))
        steps = int(rng.integers(min_steps, max_steps + 1))
        prec = FP64 if rng.random() < 0.5 else MIXED
        reqs.append(Request(k, n, steps, prec, float(arr[k]), workload_input(n, seed=10_000 + k)))
    classes = {(n, p): slots for n in sizes for p in (FP64, MIXED)}
    srv = Server(workload_params(64, "fp64"), classes, hbm_budget=150e9, tick_steps=tick, keep_fields=False,
                 group_size=group_size)
    warmed = srv.warm()
    barrier(world)
    with ClockSampler(local) as clk:
        results, st = srv.run(reqs)
    srv.close()
    value = max_over_ranks(st["elapsed_s"], world)
    st = dict(st)
    st["warm_groups"] = warmed
    return {"value": st["cell_steps"] * world / value, "unit": UNIT,
            "workload": "served request mix: Poisson 200 req/s, side in {64..1024}, steps U[%d,%d], 50%% FP64 / "
                        "50%% mixed, 150 GB HBM budget, %d requests%s" % (
                            min_steps, max_steps, R, "" if R >= 2000 else " (window scaled down from 2000)"),
            "slots_per_class": slots, "group_size": group_size, "tick_steps": tick,
            "serve": st, "gpu_launches": st["launches"], "clocks": clk.summary()}


def run_serve(args, world, rank, local):
    build_once(rank, world)
    rec = serve_record(world, rank, local, args.serve_requests, args.serve_min_steps, args.serve_max_steps,
                       args.serve_slots, args.serve_tick)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 and f32 mix",
            "data": "synthetic (Poisson arrivals, seeded fields)",
            "config": {"workload": rec["workload"], "slots_per_class": rec["slots_per_class"],
                       "group_size": rec["group_size"], "tick_steps": rec["tick_steps"]},
            "serve": rec["serve"], "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
        }), flush=True)


def hetero_layer_static(n, nz=16, nh=4, tol=1e-10, contrast=4.0):
    """Heterogeneous static problem of a plastic layer thinner than the cell (nh of nz planes,
    moduli scaled by a contrast-4 field uniform through the depth, stress control), FP64: a
    converged solve and the time of one iteration (difference of two fixed-length solves)."""
    import torch
    from paper_1911_03225_gb300 import FDM, inputs
    from paper_1911_03225_gb300 import binding as B
    p = B.Params(n1=n, n2=n, nz=nz, nh=nh, velocity_mode=B.V_STRESS, loading_mode=B.LOAD_STRESS, sigma_bar13=0.01)
    up0 = inputs.random_up(n, seed=0, ell=16.0, rms_alpha=0.1)
    f = inputs.modulus_factor(n, n, seed=1, lo=1.0 / contrast, hi=1.0, ell=24.0)

    def timed(**kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = sim.static_solve_heterogeneous_layer(f, **kw)
        return (time.perf_counter() - t0) * 1e3, out

    with FDM(p) as sim:
        sim.set_plastic_distortion(up0)
        ms, (_, _, it, res) = timed(tol=tol, max_iter=400)
        t5, _ = timed(tol=0.0, max_iter=5)
        t15, _ = timed(tol=0.0, max_iter=15)
    per_it = (t15 - t5) / 10.0
    fields = 12 * (nz // 2 + 1)
    return {"n": n, "nz": nz, "nh": nh, "contrast": contrast, "tol": tol, "iterations": it, "residual": res,
            "ms": round(ms, 3), "ms_per_iteration": round(per_it, 4), "real_2d_fields": fields,
            "note": "the x3 modes of the depth-uniform medium iterate together: %d real n x n fields, each "
                    "transformed forward and back per iteration" % fields}


def run_hetero(args, world, rank, local):
    """The heterogeneous static problems alone (shear-modulus contrast 4, n x n): a layer filling
    the cell per precision, and a layer thinner than the cell (FP64)."""
    import torch
    build_once(rank, world)
    torch.cuda.set_device(local)
    if rank == 0:
        out = {"fp64": hetero_static(args.n, "fp64", tol=1e-12), "mixed": hetero_static(args.n, "mixed", tol=1e-6)}
        layer = hetero_layer_static(min(args.n, 512))
        print(json.dumps({"workload": "heterogeneous static problem, %dx%d, contrast 4, stress control" % (args.n, args.n),
                          "hetero_static": out, "hetero_layer_static": layer}), flush=True)


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle on the host's cores (the paper publishes no code or
    timings), each step a bounded sample of the workload (the coupled configuration at 512^2)."""
    if rank != 0:
        return
    oracle_sample(0.0, 0, steps=args.warmup)
    v, k, dt, used = oracle_sample(0.0, 0, steps=args.steps)
    sample = ("coupled random-field workload on a 512x512 grid (bounded sample of the %dx%d workload), "
              "%d steps on %d threads, layer-kernel precompute excluded" % (args.n, args.n, k, used))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "coupled FDM under loading (oracle sample)", "n": 512},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--precision", default="all", choices=["fp64", "df64", "mixed", "all"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-sub-records", dest="sub_records", action="store_false",
                    help="leave the batched and served configurations out of the default line")
    ap.add_argument("--sub-serve-requests", type=int, default=48)
    ap.add_argument("--sub-serve-max-steps", type=int, default=600)
    ap.add_argument("--workload", default="coupled", choices=["coupled", "batched", "serve", "hetero"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--serve-min-steps", type=int, default=100)
    ap.add_argument("--serve-max-steps", type=int, default=5000)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-tick", type=int, default=16)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "hetero":
        run_hetero(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    from paper_1911_03225_gb300.replicas import finalize
    finalize(world)


if __name__ == "__main__":
    main()
