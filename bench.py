"""Benchmark of the MOT-JVIE march on GB300.

Workload (default): dielectric sphere eps_r = 12 voxelised in a 104^3 grid
(1,124,864 voxels of the bounding grid, 589,344 inside, 3 components), c dt = h,
FIR3 regularisation (Eq. FIR3) with delta = 1e-7 * 104^3, single x-polarised +z
modulated-Gaussian plane wave (the pulse peaks inside the timed window).

Variants: FP32-history and FP64 with the blocked temporal scheme (block B = 8, levels
of length 8, 16, 32, 64 over lags [S, 2S) and one of length 64 over lags 128..191,
the last fitted to ell = 182), and the plain FP64 direct march for comparison.  A bench
"step" is one pass of every row of the hot path: for the blocked scheme 128 time steps
(two periods of the block schedule, in each of which every level fires), for the
direct scheme one time step.  Each time step runs the forward FFT of J_{n-1}, the far-lag block products due
at that step, the near-lag MAC, the inverse FFT, the FIR epilogue and the Z_0 solve.

Metric: voxel-timesteps/s = (bounding-grid voxels) x (time steps) / march time.
The headline value is the first variant (FP32-history, blocked).  Inputs (the
excitation of every timed time step) are resident in HBM before the timed region; the
spectral ring (tens of GB) is far larger than L2, so no flush is needed.

Besides the contract's keys, each variant reports its phase times (CUDA events on the
march stream), the roofline of its dominant history kernel, and a timing-only
comparison of its forward FFT phase with cuFFT (torch.fft.rfftn) on the full padded
grid.  `e2e` marches one bench step from pinned host excitation to pinned host J
through the library's overlapped transfers (timed after one untimed call through the
same buffers).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

CONFIG_NAME = "sphere104"
REF_SAMPLE_N = 10          # oracle sample grid (its direct sum is O(M^2) per step)
REF_STEPS_PER_BENCH_STEP = 24   # oracle time steps per bench step (~3 s of CPU work)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp32_history", "fp64"])
    ap.add_argument("--config", default=CONFIG_NAME)
    ap.add_argument("--scheme", default="blocked",
                    choices=["blocked", "blocked_doubling", "direct"])
    ap.add_argument("--block", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[3], 16) if parts[3].startswith("0x") else int(parts[3])
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def geometry(ctx):
    Pu, Pv, Pw = ctx.P
    Hu, Hv, Hw = Pu // 2 + 1, Pv // 2 + 1, Pw // 2 + 1
    return Hu * Hv * Hw, Pw * Pv * Hu


def workload_text(name, shape):
    """What a named workload is, with its sizes (grid [W][V][U])."""
    W, V, U = shape
    M = W * V * U
    if name.startswith("box"):
        return ("eps_r=12 block filling a %d x %d x %d grid (W x V x U, %d voxels), c dt = h, "
                "FIR3 delta=1e-7*M, +x y-polarised modulated Gaussian plane wave" % (W, V, U, M))
    if name.startswith("sphere"):
        return ("sphere eps_r=12, %d^3 voxels (%d), c dt = h, FIR3 delta=1e-7*M, +z "
                "x-polarised modulated Gaussian plane wave" % (U, M))
    return "%s, %d x %d x %d voxels (W x V x U), c dt = h" % (name, W, V, U)


def mac_bytes_per_launch(ctx, precision, lags, n_levels):
    """Algorithmic bytes of one lag-MAC launch over `lags` lags: every lag reads the real
    kernel spectrum once per octant bin (6 values) and the three complex spectra of J
    at every rfft bin; the result (3 complex) is written once per rfft bin; with the
    blocked scheme each far level's accumulator entry of the step is read (3 complex)."""
    s = 8 if precision == "fp64" else 4
    noct, nbins = geometry(ctx)
    return lags * (6 * s * noct + 6 * s * nbins) + 6 * s * nbins * (1 + n_levels)


def far_bytes_per_period(ctx, precision):
    """Algorithmic bytes of every block Toeplitz launch of one period (each level S
    fires period / S times): the past spectra of its window that some output uses
    (lags a .. a + S - 1 of outputs n0 .. n0 + S - 1 reach back to n0 - a - S + 1, and
    nothing older than n0 - ell is used: min(2S - 1, ell - a + S) times, 3 complex per
    bin), the level's temporal kernel spectra (S + 1 frequencies x 6 complex per octant
    bin), and the S future accumulators it writes (3 complex per bin)."""
    c = 16 if precision == "fp64" else 8
    noct, nbins = geometry(ctx)
    levels, lags = ctx.levels, ctx.level_lags
    if not levels:
        return 0, 0
    period = max(levels)
    total, launches = 0, 0
    for S, a in zip(levels, lags):
        live = min(2 * S - 1, ctx.ell - a + S)
        per = 3 * c * nbins * live + (S + 1) * 6 * c * noct + S * 3 * c * nbins
        total += per * (period // S)
        launches += period // S
    return total, launches


def far_flops_per_period(ctx):
    """Floating-point operations of every block Toeplitz launch of one period, counted
    per rfft bin and firing as 3 forward and 3 inverse complex FFTs of length 2S
    (5 N log2 N each) and the 3x3 complex symmetric product at each of the 2S
    frequencies (72)."""
    import math
    _, nbins = geometry(ctx)
    levels = ctx.levels
    if not levels:
        return 0, 0
    period = max(levels)
    total, launches = 0.0, 0
    for S in levels:
        n = 2 * S
        per = nbins * (2 * 3 * 5 * n * math.log2(n) + 72 * n)
        total += per * (period // S)
        launches += period // S
    return total, launches


def mac_flops_per_launch(ctx, lags):
    """Floating-point operations of one lag-MAC launch: a real symmetric 3x3 times a
    complex 3-vector (36) per rfft bin and lag."""
    _, nbins = geometry(ctx)
    return 36.0 * nbins * lags


def fma_peaks():
    """Sustained FP64 and FP32 FMA rates of this GPU (FLOP/s), measured now by the
    library's FMA-chain kernel, with the SM clock sampled during the FP64 launch."""
    from paper_2407_03323_gb300.mot import fma_peak
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    with ClockSampler(dev) as clk:
        f64 = fma_peak(True, target_ms=400.0)
    f32 = fma_peak(False, target_ms=200.0)
    return {"fp64_tflops": f64 / 1e12, "fp32_tflops": f32 / 1e12, "clocks_fp64": clk.summary(),
            "how": "mot_fma_peak: 8 independent FMA chains per thread, occupancy-filled "
                   "grid, one launch of ~0.4 s (FP64) / 0.2 s (FP32), CUDA events"}


def profile_traffic(config, precision, scheme, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if recorded
    for this workload, precision and history scheme."""
    p = os.path.join(ROOT, "profiles", "%s_%s.txt" % (kernel, config))
    if not os.path.exists(p):
        return None
    key = "traffic_bytes_per_launch_%s_%s:" % (precision, scheme)
    for line in open(p):
        if line.startswith(key):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


# ------------------------------------------------------------------ replicas

def max_over_ranks(x, world):
    """The largest of the ranks' values (each rank times its own replica between
    barriers; the slowest one bounds the job).  Works on any initialised process group:
    NCCL reduces a device tensor, gloo a host one."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world):
    """Whole-job rate: every rank marches the same workload (weak scaling, replicas),
    so the job processes world * units in the slowest rank's time."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ our arm

def cufft_comparison(P, U, V, W, dtype_name):
    """Time of one library FFT (cuFFT through torch.fft.rfftn) of the same zero-padded
    three-component grid that the forward FFT phase transforms, for comparison only: it
    transforms the full padded cube (no pruning of the zero padding).  Returns ms per
    transform, or None if it cannot run."""
    try:
        import torch
        dt = torch.float32 if dtype_name == "fp32_history" else torch.float64
        x = torch.zeros((3, P[2], P[1], P[0]), dtype=dt, device="cuda")
        x[:, :W, :V, :U] = torch.rand((3, W, V, U), dtype=dt, device="cuda")
        for _ in range(3):
            torch.fft.rfftn(x, dim=(1, 2, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n = 20
        e0.record()
        for _ in range(n):
            torch.fft.rfftn(x, dim=(1, 2, 3))
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n
    except Exception:
        return None


def march_timed(ctx, torch, stream, E, n_steps, dev, world):
    """Time n_steps of mot_march (excitation staged from the device tensor E)."""
    ctx.set_excitation(E, stream=stream)
    ctx.set_profiling(True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        ctx.march(n_steps, out=None, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    return ms, clk.summary()


def run_variant(args, cfg, prec, scheme, block, dev, world, steps, warmup, want_e2e,
                peaks=None):
    import torch
    from paper_2407_03323_gb300 import Context
    eps, taps, p = cfg["eps_r"], cfg["taps"], cfg["pulse"]
    M = eps.size
    t_setup = time.time()
    ctx = Context(eps, taps, precision=prec, scheme=scheme, block=block)
    setup_s = time.time() - t_setup
    stream = torch.cuda.current_stream()
    # a bench step: one time step (direct); 128 time steps, whole periods of the block
    # schedule (every level fires in each), for the blocked scheme
    per = ctx.period * max(1, 128 // ctx.period) if scheme.startswith("blocked") else 1
    n_warm, n_time = warmup * per, steps * per
    # warm-up marches the pulse's leading edge; the timed steps get the pulse itself
    Ew = torch.zeros((min(n_warm, per), M, 3), dtype=torch.float64, device="cuda")
    done = 0
    while done < n_warm:
        k = min(per, n_warm - done)
        ctx.set_excitation(Ew[:k], stream=stream)
        ctx.march(k, out=None, stream=stream)
        done += k
    del Ew
    E = torch.empty((n_time, M, 3), dtype=torch.float64, device="cuda")
    t0 = p["t0"] + n_warm           # the pulse enters at the start of the timed window
    ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], t0, n_warm + 1, n_time,
                   out=E, stream=stream)
    torch.cuda.synchronize()
    ms, clocks = march_timed(ctx, torch, stream, E, n_time, dev, world)
    st = ctx.stats()
    info = ctx.info()
    peak, peak_kind = measured_peaks()
    # dominant kernel of the history evaluation
    mac_lags = min(block - 1, ctx.ell) if scheme.startswith("blocked") else ctx.ell
    mac_b = mac_bytes_per_launch(ctx, prec, mac_lags,
                                 len(ctx.levels) if scheme.startswith("blocked") else 0)
    mac_ms = st["ms_mac"] / max(st["mac_launches"], 1)
    cands = [("k_mac", mac_b, mac_ms, st["ms_mac"])]
    if scheme.startswith("blocked") and st["far_launches"]:
        fb, fl = far_bytes_per_period(ctx, prec)
        periods = st["far_launches"] / max(fl, 1)
        far_bytes_launch = fb / max(fl, 1)
        far_ms = st["ms_far"] / max(st["far_launches"], 1)
        cands.append(("k_far", far_bytes_launch, far_ms, st["ms_far"]))
    name, b_launch, ms_launch, _ = max(cands, key=lambda x: x[3])
    achieved = b_launch / (ms_launch * 1e-3) / 1e9
    hist_ms = st["ms_fft_fwd"] + st["ms_far"] + st["ms_mac"] + st["ms_fft_inv"]
    traffic = profile_traffic(args.config, prec, scheme, name)
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
            "algorithmic_bytes_per_launch": b_launch}
    if traffic:   # the same fraction from the profiled DRAM bytes instead of the model
        roof["frac_from_traffic"] = traffic / (ms_launch * 1e-3) / 1e9 / peak
    if prec == "fp64" and peaks:
        # FP64 kernels are bound by FP64 arithmetic here: report against the FP64 rate
        if name == "k_far":
            ff, fl = far_flops_per_period(ctx)
            f_launch = ff / max(fl, 1)
        else:
            f_launch = mac_flops_per_launch(ctx, mac_lags)
        ach = f_launch / (ms_launch * 1e-3) / 1e12
        roof = {"bound": "fp64", "kernel": name, "achieved": ach,
                "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                "frac": ach / peaks["fp64_tflops"],
                "peak_kind": "measured in this run (mot_fma_peak, FP64 FMA chains)",
                "traffic": roof["traffic"], "algorithmic_flops_per_launch": f_launch,
                "algorithmic_bytes_per_launch": b_launch,
                "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_kind": peak_kind}}
    out = {
        "scheme": scheme, "block": block if scheme.startswith("blocked") else None,
        "time_steps_per_bench_step": per,
        "value": job_throughput(M * n_time, ms * 1e-3, world),
        "ms_per_step": ms / steps, "ms_per_time_step": ms / n_time,
        "setup_s": setup_s, "launches": st["launches"],
        "cg_inner_iters_per_time_step": st["cg_iters"] / max(st["steps"], 1),
        "phase_ms_per_time_step": {k: st["ms_" + k] / max(st["steps"], 1)
                                   for k in ("fft_fwd", "far", "mac", "fft_inv", "solve")},
        "history_ms_per_time_step": hist_ms / max(st["steps"], 1),
        "roofline": roof,
        "clocks": clocks, "ell": info["ell"], "P": list(info["P"]), "levels": ctx.levels,
        "level_lags": ctx.level_lags,
    }
    W_, V_, U_ = eps.shape
    out["fft_comparison"] = {
        "ours_forward_fft_ms": st["ms_fft_fwd"] / max(st["steps"], 1),
        "cufft_rfftn_full_padded_ms": cufft_comparison(info["P"], U_, V_, W_, prec),
        "note": "timing comparison only; cuFFT transforms the full padded grid"}
    e2e = None
    if want_e2e:
        k = per                                  # one bench step through host buffers
        Eh = torch.empty((k, M, 3), dtype=torch.float64).pin_memory()
        Eh.copy_(E[:k].cpu())
        Jh = torch.empty((k, M, 3), dtype=torch.float64).pin_memory()
        del E
        # one untimed call through the same host buffers first (first touch of the
        # pinned pages by the copy engines), then the timed one
        ctx.set_excitation(Eh, stream=stream)
        ctx.march(k, out=Jh, stream=stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t_0 = time.perf_counter()
        ctx.set_excitation(Eh, stream=stream)
        ctx.march(k, out=Jh, stream=stream)
        torch.cuda.synchronize()
        sec = max_over_ranks(time.perf_counter() - t_0, world)
        e2e = {"value": job_throughput(M * k, sec, world), "unit": "voxel-timesteps/s",
               "h2d_bytes_per_step": M * 3 * 8 * per, "d2h_bytes_per_step": M * 3 * 8 * per,
               "variant": "%s/%s" % (prec, scheme)}
    ctx.close()
    torch.cuda.empty_cache()
    return out, e2e


def run_ours(args, rank, world):
    import torch
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = wl.config(args.config)
    variants = []
    precs = ["fp32_history", "fp64"] if args.precision == "both" else [args.precision]
    for prec in precs:
        variants.append((prec, args.scheme, args.block))
    if args.precision == "both" and args.scheme.startswith("blocked"):
        variants.append(("fp64", "direct", 0))     # the plain FP64 march, for comparison
    results, e2e = {}, None
    peaks = fma_peaks() if any(v[0] == "fp64" for v in variants) else None
    for prec, scheme, block in variants:
        # the plain direct FP64 march is slow: time a few single steps
        steps, warm = (args.steps, args.warmup)
        if scheme == "direct" and args.scheme.startswith("blocked"):
            steps, warm = 8, 3
        r, e = run_variant(args, cfg, prec, scheme, block, dev, world, steps, warm,
                           want_e2e=(e2e is None and not args.no_e2e), peaks=peaks)
        results["%s/%s" % (prec, scheme)] = r
        e2e = e2e or e
    return results, e2e, peaks


# ------------------------------------------------------------------ oracle arm

def oracle_sample(steps, warmup):
    """The CPU oracle's direct-sum march (Eqs. PnMOT + dense LU solve) on a bounded
    sample of the workload: the same sphere (eps_r = 12, FIR3, plane wave) at
    10^3 voxels; table and factorisation are setup and not timed."""
    from oracle import excitation, kernel_table, march
    from oracle.spline import num_lags
    N = REF_SAMPLE_N
    cfg = wl.config("sphere%d" % N)
    eps, taps, p = cfg["eps_r"], cfg["taps"], cfg["pulse"]
    G, _, _ = kernel_table.octant_table(N, num_lags(N, N, N) + 1)
    E = excitation.tested_excitation(eps, p, warmup + steps)
    march.march(G, eps, taps, E[:max(warmup, 1)])
    t0 = time.perf_counter()
    march.march(G, eps, taps, E[:steps])
    sec = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except ImportError:
        cores = os.cpu_count()
    return {"value": eps.size * steps / sec, "unit": "voxel-timesteps/s", "cores": cores,
            "kind": "oracle",
            "sample": "direct-sum oracle march, sphere eps_r=12 in a %d^3 grid (FIR3), "
                      "%d steps (element table and LU setup untimed)" % (N, steps)}


def run_batched_bench(args, world):
    """Config of uneven scatterers x excitations (workloads.batched_instances): the
    marches of every scatterer and excitation, FP32-history, blocked scheme with B and
    the FFT length strategy tuned per size bucket; a bench step = 128 time steps of every march.  Setup and
    tuning (which also warms every kernel variant up) are outside the timed region."""
    import torch
    from paper_2407_03323_gb300.batch import BlockTuner, run_batched
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    inst = wl.batched_instances()
    tuner = BlockTuner("fp32_history")
    n_steps = 128 * args.steps
    res = run_batched(inst, n_steps, tuner=tuner)
    value = world * res["value"]
    return {"metric": "voxel-timesteps/s", "value": value, "unit": "voxel-timesteps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * res["march_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 history + double-float CG residual + f64 state", "data": "synthetic",
            "config": {"workload": "%d scatterers (sides %d..%d, sphere/cube, eps_r 2..30) x %d "
                                   "plane waves, FIR3, %d time steps"
                                   % (len(inst), min(x["N"] for x in inst),
                                      max(x["N"] for x in inst), len(inst[0]["waves"]), n_steps),
                       "blocks": res["blocks"], "fft_lengths": res["fft_lengths"],
                       "memory_waves": res["waves"],
                       "setup_s": res["setup_s"], "tuning_s_per_step": res["tuning"],
                       "warmup": "tuning marches (block length x FFT length strategy) of every bucket",
                       "parallelism": "replicas" if world > 1 else "1 GPU"}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl != "reference" and args.config.startswith("batched"):
        line = run_batched_bench(args, world)
        if rank == 0:
            print(json.dumps(line))
        return
    if args.impl == "reference":
        if rank != 0:
            return
        ref = oracle_sample(REF_STEPS_PER_BENCH_STEP * max(args.steps, 1), args.warmup)
        line = {"impl": "reference", "metric": "voxel-timesteps/s", "value": ref["value"],
                "unit": "voxel-timesteps/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": "%s (oracle sample: %d^3)" % (args.config, REF_SAMPLE_N)},
                "cpu_baseline": ref,
                "e2e": {"value": ref["value"], "unit": "voxel-timesteps/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    results, e2e, peaks = run_ours(args, rank, world)
    head_key = next(iter(results))
    head = results[head_key]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(4 * REF_STEPS_PER_BENCH_STEP, 2)   # ~10 s of CPU work
    if rank != 0:
        return
    prec = head_key.split("/")[0]
    line = {
        "metric": "voxel-timesteps/s", "value": head["value"], "unit": "voxel-timesteps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 history (FFT, spectra, lag products, inner CG) + double-float CG "
                 "residual + f64 (elements, FIR, state J)" if prec == "fp32_history" else "f64",
        "data": "synthetic",
        "config": {"workload": workload_text(args.config, wl.config(args.config)["eps_r"].shape),
                   "variant": head_key,
                   "step": ("%d time steps (whole periods of the block schedule)"
                            % head["time_steps_per_bench_step"])
                           if head["time_steps_per_bench_step"] > 1 else "one time step",
                   "levels": head["levels"], "level_lags": head["level_lags"],
                   "P": head["P"], "ell": head["ell"],
                   "l2_flush": "inputs larger than L2 (spectral ring)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        "gpu_launches": head["launches"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "variants": results,
        "fma_peaks": peaks,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
