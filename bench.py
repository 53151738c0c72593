"""Benchmark of the fused ADMM iteration on one GB300.

Workload: one 128x128x512 confocal scene (16 ps bins, 1 m wall) scanned on a
32x32 sub-grid (stride 4), reconstructed with Algorithm 1 (object-domain
curvature ADMM); a step is one ADMM iteration.  The scene is a seeded
synthetic stand-in (3-5 tilted / curved patches), its measurement the GPU
forward model with Poisson noise (peak 50, background 2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same
workload (rank 0 only).  Under torchrun every rank runs an independent
replica (scenes do not shard: replicas only) and rank 0 reports the sum of
iterations over the max time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "headline_128x128x512"
METRIC = "ADMM iter/s (Algorithm 1, 128x128x512 volume, 32x32 sampled scan)"
PAPER_ITER_PER_S = 1.0 / 0.1   # about 0.1 s per iteration at 128x128x512 on a TITAN RTX (Sec. 4.2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400,
                    help="timed iterations, split into 5 timed regions (median reported)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-system", action="store_true",
                    help="skip the short batched and served runs of the default line's `system` key")
    ap.add_argument("--ops", action="store_true",
                    help="only apply the forward and adjoint operators --steps times (for profiler captures)")
    ap.add_argument("--lateral", type=int, default=0,
                    help="lateral stage of the plan (0 FFT kernels, 1 split-BF16 tensor-core DFT products, "
                         "2 BF16 hi-only ones)")
    ap.add_argument("--workload", default="headline", choices=["headline", "batch16", "serve"],
                    help="headline: one 128x128x512 scene; batch16: 16 mixed scenes batched vs one by one; "
                         "serve: Poisson-arrival stream through the server")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrivals per second")
    ap.add_argument("--budget-gb", type=float, default=0.0, help="serve: HBM budget (0 = 80 percent of free)")
    ap.add_argument("--slots", type=int, default=4, help="serve: jobs running at once")
    ap.add_argument("--prewarm", type=int, default=2,
                    help="serve: job contexts per (grid, sampling, model) prepared before the arrivals start")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs(seed):
    cfg = synth.CONFIGS[WORKLOAD]
    vol = synth.make_volume(cfg, seed)
    mask = synth.make_mask(cfg)
    return cfg, vol, mask


# ---------------------------------------------------------------------------
# clocks (nvidia-smi sampled during the timed region)
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping (algorithmic work per launch of each kernel)
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tflops(sm_mhz, sms):
    # FP32 lanes: SMs x 128 lanes, 2 flops per FMA
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def algorithmic(cat, nx, nt, ncols):
    """(kind, amount per launch) for a timing category of the Algorithm-1 step."""
    S = (nt + 1) * nx * nx * 8
    Sc = (nt + 1) * ncols * 8
    K = (nt + 1) * (nx + 1) * (nx + 1) * 8
    F = nx * nx * nt * 4
    Fc = ncols * nt * 4
    Sp = (nt // 2 + 1) * nx * nx * 8
    if cat == "k_conv":
        # 60 N^2 log2 N nominal FFT flops per kt plane (12 N transforms of length N, 5 N log2 N each)
        return "flops", (nt + 1) * 60.0 * nx * nx * np.log2(nx), S + Sc + K
    if cat == "k_tfwd":   # average of the R_z pass (F -> S) and the R_t^T pass (3 Fc -> Sc)
        return "bytes", 0.5 * ((F + S) + (3 * Fc + Sc)), None
    if cat == "k_tinv":   # Sc -> Fc plus the three compact fit inputs
        return "bytes", Sc + 4 * Fc, None
    if cat == "k_tadj":   # S in, u-bar and reg in, periodic spectrum out
        return "bytes", S + 2 * F + Sp, None
    if cat == "k_sxy":
        return "bytes", 2 * Sp, None
    if cat == "k_sinv":   # spectrum in, u+ out, u-bar in (||d||^2)
        return "bytes", Sp + 2 * F, None
    if cat == "k_pre":    # u-bar, Lambda (3), phi in; reg out
        return "bytes", 6 * F, None
    if cat == "k_post":   # fused post and pre step: u+, u^k, u-bar, Lambda (3), phi in;
        return "bytes", 13 * F, None   # Lambda (3), phi, u-bar', reg out
    return "bytes", 0.0, None


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (replicas: every rank runs its own scene)
# ---------------------------------------------------------------------------
def max_over_ranks(value, world, device):
    """The largest value over all ranks (the job's time is its slowest rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, t_ms_max):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / (t_ms_max / 1e3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def source_digest(*rel):
    """First 16 hex digits of the SHA-256 of the named source files (together)."""
    import hashlib
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes per launch of the lateral pass k_conv4 from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, mean of the forward launch of
# A_D on the lattice of sampled rows, 135.64 + 1.47 MB, and the adjoint one,
# 72.58 + 24.95 MB) at 128x128x512 with 32x32 sampled columns, valid for the
# sources with this digest; any change to them makes the figure stale (null).
CONV4_TRAFFIC = {"bytes": 117.32e6, "workload": (128, 128, 512, 1024),
                 "sources": ("paper_2301_00406_gb300/csrc/conv4.cu", "paper_2301_00406_gb300/csrc/fft.cuh"),
                 "digest": "a364346b7731e3005ecf0a438cf84ec2"}


TUNE_KINDS = ["tfwd_rz", "tfwd_rtt", "tinv_store", "tinv_fit", "tadj_store", "tadj_solve", "sfwd", "sinv",
              "sinv_rz", "lateral_solve"]


def tuning_choices(nt, nx, columns=None):
    """The plan tuner's recorded choices for this geometry (t-pass launch
    shapes per kind and launch column count, restricted to `columns` when
    given; the lateral solve's kernel), read back from the library's tuning
    file; None where there is no file."""
    path = os.environ.get("NLOS_TUNE_CACHE")
    if path is None:
        base = os.environ.get("XDG_CACHE_HOME") or (os.path.join(os.environ["HOME"], ".cache")
                                                     if os.environ.get("HOME") else None)
        path = os.path.join(base, "nlos-gb300", "tpass_tuning") if base else None
    if not path or path == "off" or not os.path.exists(path):
        return None
    out = {"tpass": [], "lateral_solve": None}
    with open(path) as fh:
        for line in fh.read().splitlines()[2:]:
            f = line.split()
            if len(f) != 4:
                continue
            kind, knt, ncols, v = map(int, f)
            if knt != nt or not 0 <= kind < len(TUNE_KINDS):
                continue
            if TUNE_KINDS[kind] == "lateral_solve":
                if ncols == nx:
                    out["lateral_solve"] = {1: "shared-memory passes", 2: "half-warp transforms"}.get(v, v)
            elif columns is None or ncols in columns:
                out["tpass"].append({"kind": TUNE_KINDS[kind], "columns": ncols, "cols_per_cta": v & 255,
                                     "batched_halves": bool(v >> 8)})
    return out


def conv4_traffic(nx, ny, nt, ncols):
    t = CONV4_TRAFFIC
    if (nx, ny, nt, ncols) != t["workload"]:
        return None
    digest = "".join(source_digest(s) for s in t["sources"])
    return t["bytes"] if digest == t["digest"] else None


REGIONS = 5   # timed regions per measurement; the line reports their median


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2301_00406_gb300 import nlos
    cfg, vol, mask = make_inputs(seed=rank)
    nx, ny, nt = cfg["nx"], cfg["ny"], cfg["nt"]
    plan = nlos.Plan(nx, ny, nt, cfg["bin_width_s"], mask=mask)
    stream = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # measurement: GPU forward model + seeded Poisson noise
    u_true = torch.tensor(vol, dtype=torch.float32, device="cuda")
    sig = nlos.forward_t(plan, u_true, apply_mask=True).cpu().numpy()
    tau0_h = synth.poisson_measurement(sig, mask, cfg["peak"], cfg["background"], seed=100 + rank)
    tau0 = torch.tensor(tau0_h, dtype=torch.float32, device="cuda")
    u_out = torch.empty_like(tau0)
    if args.lateral:
        plan.set_lateral(args.lateral)

    p = nlos.params_default(1)
    p.a, p.b, p.mu = cfg["a"], cfg["b"], cfg["mu"]

    def recon(iters, tau_ptr=None, out_ptr=None, params=p):
        params.iters = iters
        return plan.reconstruct(params, tau_ptr or tau0.data_ptr(), out_ptr or u_out.data_ptr(), 0, stream)

    def prepare(iters, tau_ptr=None, out_ptr=None, params=p):
        # capture the run's graph outside the timed region (no iterations run)
        params.iters = iters
        return plan.reconstruct_prepare(params, tau_ptr or tau0.data_ptr(), out_ptr or u_out.data_ptr(), 0, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fn, regions):
        """CUDA-event times (ms) of `regions` calls of fn, each bracketed by a
        barrier and a device synchronisation on both sides."""
        out = []
        for _ in range(regions):
            barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            barrier()
            out.append(e0.elapsed_time(e1))
        return out

    recon(args.warmup)                       # warm-up (also computes ||A_D||^2 once)
    norm2 = plan.norm2(True)
    # the K timed steps are split into REGIONS reconstructions of K / REGIONS iterations
    per = max(1, args.steps // REGIONS)
    steps = per * REGIONS
    graphed = prepare(per)
    torch.cuda.synchronize()
    stats = {}
    with ClockSampler(local) as clk:
        reg_ms = timed(lambda: stats.update(recon(per)), REGIONS)
    clocks = clk.summary()
    t_ms = max_over_ranks(statistics.median(reg_ms), world, "cuda")   # median region, slowest rank
    value = job_rate(per, world, t_ms)

    # reconstructions of exactly 50 iterations (the recon/s metric)
    prepare(50)
    rec_ms = timed(lambda: recon(50), REGIONS)
    rec50 = job_rate(1, world, max_over_ranks(statistics.median(rec_ms), world, "cuda"))

    # per-kernel timing over one reconstruction of K iterations (NVTX range
    # "alg1_iterations" lets a profiler restrict itself to these launches)
    plan.timing_enable(True)
    torch.cuda.nvtx.range_push("alg1_iterations")
    recon(steps)
    torch.cuda.nvtx.range_pop()
    kt = plan.timing_read()
    plan.timing_enable(False)
    launches = sum(c for _, c in kt.values())

    # end to end through the C ABI from host memory (nlos_reconstruct_host):
    # pinned tau0 -> device, the iterations of one region, u -> pinned host,
    # host wall time of the whole call (it synchronises)
    tau0_pin = torch.tensor(tau0_h, dtype=torch.float32).pin_memory()
    u_pin = torch.empty_like(tau0_pin).pin_memory()
    p.iters = per
    plan.reconstruct_host(p, tau0_pin.data_ptr(), u_pin.data_ptr(), 0, stream)   # warm-up: buffers, graph
    e2e_s = []
    for _ in range(REGIONS):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.reconstruct_host(p, tau0_pin.data_ptr(), u_pin.data_ptr(), 0, stream)
        e2e_s.append(time.perf_counter() - t0)
        barrier()
    e2e_ms = max_over_ranks(1e3 * statistics.median(e2e_s), world, "cuda")
    nbytes = tau0_pin.numel() * 4

    # backtracking live: L0 = 1e-3 ||A_D||^2, the u-step repeats until the
    # FP64 test accepts (about ten rejections in the first iteration), and L
    # stays below the bound above which the test is skipped, so every
    # iteration evaluates the test's FP64 reductions; steady-state rate from
    # runs of per + 1 and 1 iterations
    pb = nlos.params_default(1)
    pb.a, pb.b, pb.mu = cfg["a"], cfg["b"], cfg["mu"]
    pb.L0 = 1e-3 * norm2
    prepare(per + 1, params=pb)
    prepare(1, params=pb)
    bt_stats = recon(per + 1, params=pb)
    t_long = statistics.median(timed(lambda: recon(per + 1, params=pb), 3))
    t_one = statistics.median(timed(lambda: recon(1, params=pb), 3))
    bt_rate = per / ((t_long - t_one) / 1e3)

    # Algorithm 2 on the same scene (secondary line)
    p2 = nlos.params_default(2)
    for k in ("a_u", "b_u", "a_tau", "b_tau", "mu1", "mu2", "mu3"):
        setattr(p2, k, cfg[k])
    p2.lambda_ = cfg["lam"]
    p2.iters = args.warmup
    tau_out = torch.empty_like(tau0)
    plan.reconstruct(p2, tau0.data_ptr(), u_out.data_ptr(), tau_out.data_ptr(), stream)
    torch.cuda.synchronize()
    p2.iters = per
    plan.reconstruct_prepare(p2, tau0.data_ptr(), u_out.data_ptr(), tau_out.data_ptr(), stream)
    alg2_ms = statistics.median(timed(
        lambda: plan.reconstruct(p2, tau0.data_ptr(), u_out.data_ptr(), tau_out.data_ptr(), stream), REGIONS))
    # per-kernel timing of Algorithm 2 (a second, host-stepped run; NVTX range
    # "alg2_iterations" for profilers)
    plan.timing_enable(True)
    torch.cuda.nvtx.range_push("alg2_iterations")
    plan.reconstruct(p2, tau0.data_ptr(), u_out.data_ptr(), tau_out.data_ptr(), stream)
    torch.cuda.nvtx.range_pop()
    kt2 = plan.timing_read()
    plan.timing_enable(False)

    if rank != 0:
        return None

    # roofline of the dominant kernel
    peaks, src = measured_peaks()
    ncols = int(mask.sum())
    dom = max((k for k in kt if k != "small"), key=lambda k: kt[k][0])
    tot_ms, nl = kt[dom]
    avg_s = tot_ms / max(nl, 1) / 1e3
    kind, amount, bytes_alg = algorithmic(dom, nx, nt, ncols)
    if kind == "flops":
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = alu_peak_tflops(sm_mhz, sms)
        ach = amount / avg_s / 1e12
        traffic = conv4_traffic(nx, ny, nt, ncols) if dom == "k_conv" and not args.lateral else None
        roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                "traffic": round(traffic) if traffic else None,
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (derived)",
                "algorithmic_hbm_gbs": round(bytes_alg / avg_s / 1e9, 1)}
    else:
        peak = peaks["hbm_gbs"]
        ach = amount / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": None, "peak_source": f"hbm_gbs ({src})"}
    step_ms = t_ms / per
    # whole-iteration HBM model: compulsory bytes of one Algorithm-1 iteration
    # (each state field read and written once, spectra written and read once,
    # the kernel spectrum read by both lateral passes)
    full = nx * ny
    s_frac = ncols / full
    F = full * nt * 4
    S = (nt + 1) * full * 8
    Sp = (nt // 2 + 1) * full * 8
    K = (nt + 1) * (nx + 1) * (ny + 1) * 8
    b_iter = (14 + s_frac) * F + 4 * S + 4 * s_frac * S + 4 * Sp + 2 * K
    it_gbs = b_iter / (step_ms / 1e3) / 1e9
    iter_roof = {"bytes_per_iter": round(b_iter), "achieved": round(it_gbs, 1), "peak": peaks["hbm_gbs"],
                 "unit": "GB/s", "frac": round(it_gbs / peaks["hbm_gbs"], 4),
                 "note": "model bytes (14+s)F + 4S + 4sS + 4S' + 2K over the measured iteration time"}
    kernels = {k: {"ms_per_step": round(v[0] / steps, 4), "launches_per_step": round(v[1] / steps, 2)}
               for k, v in kt.items() if v[1] > 0}

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "iter/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": round(value / PAPER_ITER_PER_S, 1), "dtype": "f32", "data": "synthetic",
        "config": {"workload": "alg1_128x128x512_16ps_32x32_sampled", "nx": nx, "ny": ny, "nt": nt,
                   "sampled_columns": ncols, "model": "object-domain curvature ADMM (Algorithm 1)",
                   "timed_regions": f"{REGIONS} reconstructions of {per} iterations each; value from the median "
                                    f"region (max over ranks)",
                   "region_ms": [round(x, 3) for x in reg_ms], "sm_count": sms,
                   "lateral_stage": {0: "FP32 FFT kernels", 1: "split-BF16 tcgen05", 2: "BF16 tcgen05"}[args.lateral],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set ~0.7 GB > 129 MB L2; no flush needed",
                   "graph": "whole reconstruction captured before the timed region" if graphed else "no graph",
                   "tuning": tuning_choices(nt, nx, (nx * ny, ncols))},
        "clocks": clocks,
        "e2e": {"value": round(job_rate(per, world, e2e_ms), 2), "unit": "iter/s",
                "h2d_bytes_per_step": nbytes / per, "d2h_bytes_per_step": nbytes / per,
                "note": f"nlos_reconstruct_host (C ABI, host buffers): pinned tau0 copied in, {per} iterations, "
                        f"u copied out, host wall time of the synchronising call; median of {REGIONS}"},
        "gpu_launches": launches,
        "roofline": roof,
        "iteration_roofline": iter_roof,
        "kernels": kernels,
        "secondary": {"alg2_iter_per_s": round(per / (alg2_ms / 1e3), 2),
                      "alg2_kernels_ms_per_step": {k: round(v[0] / per, 4) for k, v in kt2.items() if v[1]},
                      "recon_per_s_at_50_iters": round(rec50, 3),
                      "recon_50_ms": [round(x, 3) for x in rec_ms],
                      "alg1_backtracking_live": {
                          "iter_per_s": round(bt_rate, 2), "L0": "1e-3 ||A_D||^2",
                          "backtracks_in_first_run": bt_stats["backtracks"],
                          "final_L_over_norm2": round(bt_stats["L"] / norm2, 4),
                          "note": "steady state (runs of K/5 + 1 and 1 iterations); every iteration computes the "
                                  "FP64 backtracking-test terms"},
                      "alg1_energy_last": stats.get("energy")},
    }
    if world == 1 and not args.no_system:
        out["system"] = system_summary(args)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, tau0_h, mask, 2.0 * norm2, samples=3)
    return out


def system_summary(args):
    """The batched and served forms beside the one-scene numbers: the 16-scene
    batch against its sequential run, and 10 s of Poisson arrivals at 20 jobs/s
    through the server (4 jobs at once, contexts prepared before the arrivals).
    A failure here is reported in the line, not raised."""
    res = {}
    try:
        b = run_batch16(args)
        res["batch16"] = {k: b[k] for k in ("value", "unit", "batched_s", "sequential_s", "speedup_vs_sequential",
                                            "results_identical_to_sequential")}
    except Exception as e:  # noqa: BLE001
        res["batch16"] = {"error": f"{type(e).__name__}: {e}"}
    try:
        sa = argparse.Namespace(**vars(args))
        sa.duration, sa.rate, sa.slots, sa.prewarm, sa.budget_gb = 10.0, 20.0, 4, 2, 0.0
        v = run_serve(sa)
        res["serve"] = {k: v[k] for k in ("p50_s", "p99_s", "max_s", "mean_queue_s", "jobs", "throughput_jobs_per_s",
                                          "prewarm")}
        res["serve"]["config"] = "10 s of Poisson arrivals at 20/s, 64^2 or 128^2 x 512 grids, 3 samplings, " \
                                 "Algorithm 1 or 2, 50 iterations, 4 jobs at once"
    except Exception as e:  # noqa: BLE001
        res["serve"] = {"error": f"{type(e).__name__}: {e}"}
    return res


# ---------------------------------------------------------------------------
# the oracle (FP64 NumPy, one thread) on the same workload
# ---------------------------------------------------------------------------
def cpu_baseline(cfg, tau0_h, mask, L0, samples=3, warmup=0, budget_s=None):
    """The FP64 oracle's Algorithm 1 at the GPU arm's L0 = 2 ||A_D||^2, timed
    one iteration per sample (each from the zero start, one trial: the test
    cannot reject at that L0); median seconds per iteration."""
    from oracle import admm, lct
    g = lct.Geometry(cfg["nx"], cfg["ny"], cfg["nt"], cfg["bin_width_s"])
    op = lct.Operator(g, mask)
    for _ in range(warmup):  # bounded warm-up steps: one adjoint operator application each
        op.adjoint_d(tau0_h)
    times, trials = [], []
    t_start = time.perf_counter()
    while len(times) < samples:
        t0 = time.perf_counter()
        _, hist = admm.alg1(tau0_h, mask, g, cfg["a"], cfg["b"], cfg["mu"], 1, L0=L0, op=op)
        times.append(time.perf_counter() - t0)
        trials.append(1 + int(sum(hist["backtracks"])))
        if budget_s is not None and time.perf_counter() - t_start + times[-1] > budget_s:
            break
    per = statistics.median(times)
    return {"value": round(1.0 / per, 5), "unit": "iter/s", "cores": 1, "kind": "oracle",
            "samples": len(times), "seconds": [round(t, 2) for t in times],
            "sample": f"{len(times)} Algorithm-1 iteration(s) of the FP64 NumPy oracle at 128x128x512, 32x32 sampled "
                      f"(median {per:.1f} s each; L0 = {L0:.6g} = 2 ||A_D||^2 as on the GPU, "
                      f"u-step trials per iteration {trials}: the same work per iteration as the GPU arm's; "
                      f"numpy.fft single-threaded) after {warmup} warm-up step(s) of one adjoint operator "
                      f"application each; host cores available: {os.cpu_count()}"}


GOLDEN_ALG1 = os.path.join(ROOT, "tests", "golden", "headline_alg1_128x128x512.npz")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    cfg, vol, mask = make_inputs(seed=0)
    from oracle import lct
    g = lct.Geometry(cfg["nx"], cfg["ny"], cfg["nt"], cfg["bin_width_s"])
    sig = lct.Operator(g, mask).forward_d(vol)
    tau0_h = synth.poisson_measurement(sig, mask, cfg["peak"], cfg["background"], seed=100)
    # L0 = 2 ||A_D||^2 of this geometry and mask, as the oracle's own power
    # iteration gave it in the stored FP64 run (the first entry of its L history)
    L0 = float(np.load(GOLDEN_ALG1)["L"][0])
    cb = cpu_baseline(cfg, tau0_h, mask, L0, samples=max(1, args.steps), warmup=args.warmup, budget_s=150.0)
    steps = cb["samples"]
    value = cb["value"]
    return {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 / value, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": round(value / PAPER_ITER_PER_S, 4), "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "alg1_128x128x512_16ps_32x32_sampled", "nx": cfg["nx"], "ny": cfg["ny"],
                       "nt": cfg["nt"], "model": "object-domain curvature ADMM (Algorithm 1)"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": cb["sample"], "value": value, "unit": "iter/s"},
            "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ops(args):
    """Forward and adjoint operator applications only (few launches), then the
    time of the unmasked forward operator A and of its lateral stage (CUDA
    events: 3 warm-up calls, 10 timed; then 10 calls with per-kernel timing),
    with the plan's lateral stage set by --lateral."""
    import torch
    from paper_2301_00406_gb300 import nlos
    cfg, vol, mask = make_inputs(seed=0)
    plan = nlos.Plan(cfg["nx"], cfg["ny"], cfg["nt"], cfg["bin_width_s"], mask=mask)
    if args.lateral:
        plan.set_lateral(args.lateral)
    u = torch.tensor(vol, dtype=torch.float32, device="cuda")
    for _ in range(args.steps):
        tau = nlos.forward_t(plan, u, apply_mask=True)
        u = nlos.adjoint_t(plan, tau, apply_mask=True)
    torch.cuda.synchronize()
    x = torch.tensor(vol, dtype=torch.float32, device="cuda")
    for _ in range(3):
        nlos.forward_t(plan, x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        nlos.forward_t(plan, x)
    e1.record()
    torch.cuda.synchronize()
    plan.timing_enable(True)
    for _ in range(10):
        nlos.forward_t(plan, x)
    kt = plan.timing_read()
    plan.timing_enable(False)
    return {"ops": args.steps, "checksum": float(u.double().sum().item()), "lateral_mode": args.lateral,
            "forward_ms": round(e0.elapsed_time(e1) / 10, 4), "lateral_stage_ms": round(kt["k_conv"][0] / 10, 4)}


# ---------------------------------------------------------------------------
# batching (16 mixed scenes) and serving (Poisson arrivals)
# ---------------------------------------------------------------------------
BATCH16 = [(32, 256, 32e-12)] * 6 + [(64, 512, 16e-12)] * 6 + [(128, 512, 16e-12)] * 4


def _scene_inputs(nlos, n, nt, bw, mask, seed, model):
    import torch
    plan = nlos.Plan(n, n, nt, bw, mask=mask)
    vol = synth.scene_patches(n, n, nt, seed) if model == 2 else synth.scene_planes_glyph(n, n, nt, seed)
    sig = nlos.forward_t(plan, torch.tensor(vol, dtype=torch.float32, device="cuda"), apply_mask=True).cpu().numpy()
    tau0 = synth.poisson_measurement(sig, mask, 50.0, 2.0, seed + 1000).astype(np.float32)
    return plan, tau0


def _params(nlos, model, iters):
    cfg = synth.CONFIGS["headline_128x128x512"]
    p = nlos.params_default(model)
    if model == 1:
        p.a, p.b, p.mu = cfg["a"], cfg["b"], cfg["mu"]
    p.iters = iters
    return p


def run_batch16(args):
    """16 scenes of mixed size, random 25 % masks, models alternating, 50 iterations:
    one nlos_reconstruct_batch call vs 16 nlos_reconstruct calls in sequence."""
    import torch
    from paper_2301_00406_gb300 import nlos
    iters = 50
    plans, params, taus, outs = [], [], [], []
    for i, (n, nt, bw) in enumerate(BATCH16):
        model = 1 if i % 2 == 0 else 2
        mask = synth.random_mask(n, n, 0.25, 500 + i)
        plan, tau0 = _scene_inputs(nlos, n, nt, bw, mask, i, model)
        plans.append(plan)
        params.append(_params(nlos, model, iters))
        taus.append(torch.tensor(tau0, device="cuda"))
        outs.append(torch.empty_like(taus[-1]))
    stream = torch.cuda.current_stream().cuda_stream

    def sequential():
        for pl, pa, t, o in zip(plans, params, taus, outs):
            pl.reconstruct(pa, t.data_ptr(), o.data_ptr(), 0, stream)

    def batched():
        nlos.reconstruct_batch(plans, params, [t.data_ptr() for t in taus], [o.data_ptr() for o in outs],
                               stream=stream)

    for f in (sequential, batched):        # warm-up (plans compute their norms here)
        f()
    torch.cuda.synchronize()
    times = {}
    for name, f in (("sequential", sequential), ("batched", batched)):
        reps = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            f()
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t0)
        times[name] = statistics.median(reps)
    seq = [o.clone() for o in outs]
    batched()
    torch.cuda.synchronize()
    same = all(torch.equal(a, b) for a, b in zip(seq, outs))
    total_iters = iters * len(BATCH16)
    return {"metric": "batched reconstructions/s (16 mixed scenes, 50 iterations each)",
            "value": round(len(BATCH16) / times["batched"], 3), "unit": "recon/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch16_mixed", "scenes": "6x 32x32x256, 6x 64x64x512, 4x 128x128x512",
                       "masks": "random 25 %", "models": "alternating 1/2", "iters": iters},
            "batched_s": round(times["batched"], 4), "sequential_s": round(times["sequential"], 4),
            "speedup_vs_sequential": round(times["sequential"] / times["batched"], 3),
            "batched_iter_per_s": round(total_iters / times["batched"], 1),
            "results_identical_to_sequential": bool(same)}


def run_serve(args):
    """Poisson arrivals (mean --rate per second) for --duration seconds through nlos_server."""
    import torch
    from paper_2301_00406_gb300 import nlos
    rng = np.random.default_rng(7)
    grids = [(64, 512, 16e-12), (128, 512, 16e-12)]
    samplings = [8, 16, 32]          # sampled points per side
    pool = {}
    for n, nt, bw in grids:          # a few seeded measurements per (grid, sampling, model)
        for side in samplings:
            mask = synth.stride_mask(n, n, n // side)
            for model in (1, 2):
                plan, tau0 = _scene_inputs(nlos, n, nt, bw, mask, len(pool), model)
                plan.close()
                pool[(n, nt, bw, side, model)] = (mask, tau0)
    free, total = torch.cuda.mem_get_info()
    budget = int(args.budget_gb * (1 << 30)) if args.budget_gb > 0 else int(0.8 * free)
    srv = nlos.Server(hbm_budget_bytes=budget, max_slots=args.slots)
    t_warm = time.perf_counter()
    warmed = 0
    if args.prewarm > 0:                 # plans, contexts and graphs built before traffic
        for (n, nt, bw, side, model), (mask, _) in pool.items():
            warmed += srv.prepare(n, n, nt, bw, _params(nlos, model, 50), contexts=args.prewarm, mask=mask)
    t_warm = time.perf_counter() - t_warm
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=int(args.rate * args.duration * 2)))
    arrivals = arrivals[arrivals < args.duration]
    keys = list(pool.keys())
    choice = rng.integers(0, len(keys), size=len(arrivals))
    jobs = []
    t_start = time.perf_counter()
    for t_arr, ci in zip(arrivals, choice):
        while time.perf_counter() - t_start < t_arr:
            time.sleep(0.0005)
        n, nt, bw, side, model = keys[ci]
        mask, tau0 = pool[keys[ci]]
        out = np.empty_like(tau0)
        jid = srv.submit(n, n, nt, bw, _params(nlos, model, 50), tau0, out, mask=mask)
        jobs.append((jid, out, keys[ci]))
    lat, queued = [], []
    for jid, _, _ in jobs:
        st = srv.wait(jid, timeout_s=600.0)
        assert st is not None and st["status"] == 0
        q, tot = srv.job_times(jid)
        lat.append(tot)
        queued.append(q)
    t_end = time.perf_counter()
    info = srv.info()
    srv.close()
    lat = np.array(lat)
    late = lat[arrivals[:len(lat)] >= min(10.0, args.duration / 2)]   # arrivals after the first 10 s
    return {"metric": "served reconstruction latency p50/p99 (Poisson arrivals)",
            "value": round(float(np.percentile(lat, 50)), 4), "unit": "s", "higher_is_better": False,
            "p50_s": round(float(np.percentile(lat, 50)), 4), "p99_s": round(float(np.percentile(lat, 99)), 4),
            "mean_queue_s": round(float(np.mean(queued)), 4), "jobs": len(jobs),
            "p99_after_10s_s": round(float(np.percentile(late, 99)), 4) if len(late) else None,
            "max_s": round(float(lat.max()), 4),
            "prewarm": {"contexts_per_kind": args.prewarm, "contexts_ready": warmed, "seconds": round(t_warm, 3)},
            "throughput_jobs_per_s": round(len(jobs) / (t_end - t_start), 3),
            "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve_poisson", "rate_per_s": args.rate, "duration_s": args.duration,
                       "grids": "64x64x512, 128x128x512 (16 ps)", "sampling": "8x8, 16x16, 32x32 strides",
                       "models": "1 or 2 at random", "iters": 50, "budget_bytes": budget, "slots": args.slots},
            "server": info}


def main():
    args = parse()
    if args.workload == "batch16":
        print(json.dumps(run_batch16(args)))
        return
    if args.workload == "serve":
        print(json.dumps(run_serve(args)))
        return
    if args.ops:
        print(json.dumps(run_ops(args)))
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
