"""Benchmark of the MOT-JVIE march on GB300.

Workload (default): dielectric sphere eps_r = 12 voxelised in a 104^3 grid
(1,124,864 voxels of the bounding grid, 589,344 inside, 3 components), c dt = h,
9-tap linear-phase high-pass FIR regularisation with delta = 1e-7 * 104^3, single
x-polarised +z modulated-Gaussian plane wave.  A "step" is one time step of the march:
the forward FFT of J_{n-1}, the lag multiply-accumulate over the spectral ring, the
inverse FFT, the FIR epilogue and the CG solve of Z_0.

Metric: voxel-timesteps/s = (bounding-grid voxels) x (time steps) / march time.
The headline value is the FP32-history march; the FP64 march is reported alongside.
Inputs (the excitation of every timed step) are resident in HBM before the timed
region; the spectral ring (tens of GB) is far larger than L2, so no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
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

import workloads as wl  # noqa: E402

CONFIG_NAME = "sphere104"
REF_SAMPLE_N = 10          # oracle sample grid (its direct sum is O(M^2) per step)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both", choices=["both", "fp32_history", "fp64"])
    ap.add_argument("--config", default=CONFIG_NAME)
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


def mac_bytes_per_launch(ctx, precision):
    """Algorithmic bytes of one direct lag-MAC launch: every lag reads the real kernel
    spectrum once per octant bin (6 values) and the three complex spectra of J at every
    rfft bin; the result is written once per rfft bin (3 complex values)."""
    s = 8 if precision == "fp64" else 4
    Pu, Pv, Pw = ctx.P
    Hu, Hv, Hw = Pu // 2 + 1, Pv // 2 + 1, Pw // 2 + 1
    noct = Hu * Hv * Hw
    nbins = Pw * Pv * Hu
    L = ctx.ell
    return L * (6 * s * noct + 6 * s * nbins) + 6 * s * nbins


def profile_traffic(precision):
    """DRAM bytes per k_mac launch from the committed ncu summary, if recorded."""
    p = os.path.join(ROOT, "profiles", "k_mac_sphere104.txt")
    if not os.path.exists(p):
        return None
    key = "traffic_bytes_per_launch_%s:" % precision
    for line in open(p):
        if line.startswith(key):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world):
    import torch
    from paper_2407_03323_gb300 import Context
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    cfg = wl.config(args.config)
    eps, taps, p = cfg["eps_r"], cfg["taps"], cfg["pulse"]
    M = eps.size
    precisions = ["fp32_history", "fp64"] if args.precision == "both" else [args.precision]
    results = {}
    e2e = None
    for prec in precisions:
        t_setup = time.time()
        ctx = Context(eps, taps, precision=prec)
        setup_s = time.time() - t_setup
        stream = torch.cuda.current_stream()
        W, K = args.warmup, args.steps
        E = torch.empty((W + K, M, 3), dtype=torch.float64, device="cuda")
        ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"], 1, W + K, out=E,
                       stream=stream)
        ctx.set_excitation(E, stream=stream)
        torch.cuda.synchronize()
        ctx.march(W, out=None, stream=stream)
        torch.cuda.synchronize()
        ctx.set_profiling(True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            ev0.record(stream)
            ctx.march(K, out=None, stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        st = ctx.stats()
        info = ctx.info()
        mac_ms = st["ms_mac"] / max(st["mac_launches"], 1)
        bytes_mac = mac_bytes_per_launch(ctx, prec)
        peak, peak_kind = measured_peaks()
        achieved = bytes_mac / (mac_ms * 1e-3) / 1e9
        results[prec] = {
            "value": world * M * K / (ms * 1e-3),
            "ms_per_step": ms / K,
            "setup_s": setup_s,
            "launches": st["launches"],
            "cg_iters_per_step": st["cg_iters"] / max(st["steps"], 1),
            "phase_ms_per_step": {k: st["ms_" + k] / max(st["steps"], 1)
                                  for k in ("fft_fwd", "mac", "fft_inv", "solve")},
            "roofline": {"bound": "hbm", "kernel": "k_mac", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": profile_traffic(prec),
                         "algorithmic_bytes_per_launch": bytes_mac},
            "clocks": clk.summary(),
            "ell": info["ell"], "P": list(info["P"]),
        }
        # end-to-end through the public API with host buffers (first precision only)
        if e2e is None and not args.no_e2e:
            Eh = torch.empty((K, M, 3), dtype=torch.float64).pin_memory()
            Eh.copy_(E[W:W + K].cpu())
            Jh = torch.empty((K, M, 3), dtype=torch.float64).pin_memory()
            del E
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            t0 = time.perf_counter()
            ctx.set_excitation(Eh, stream=stream)
            ctx.march(K, out=Jh, stream=stream)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            if world > 1:
                t = torch.tensor([sec], device="cuda")
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
                sec = float(t.item())
            e2e = {"value": world * M * K / sec, "unit": "voxel-timesteps/s",
                   "h2d_bytes_per_step": M * 3 * 8, "d2h_bytes_per_step": M * 3 * 8,
                   "precision": prec}
        ctx.close()
        torch.cuda.empty_cache()
    return results, e2e


# ------------------------------------------------------------------ oracle arm

def oracle_sample(steps, warmup):
    """The CPU oracle's direct-sum march (Eqs. PnMOT + dense LU solve) on a bounded
    sample of the workload: the same sphere (eps_r = 12, hp9 FIR, plane wave) at
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
            "sample": "direct-sum oracle march, sphere eps_r=12 in a %d^3 grid (hp9 FIR), "
                      "%d steps (element table and LU setup untimed)" % (N, steps)}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        ref = oracle_sample(max(args.steps, 8), args.warmup)
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
    results, e2e = run_ours(args, rank, world)
    head = results.get("fp32_history") or results.get("fp64")
    head_prec = "fp32_history" if "fp32_history" in results else "fp64"
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(24, 2)
    if rank != 0:
        return
    M = wl.config(args.config)["eps_r"].size
    line = {
        "metric": "voxel-timesteps/s", "value": head["value"], "unit": "voxel-timesteps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 history (FFT, spectra, lag MAC) + f64 (elements, FIR, CG)"
                 if head_prec == "fp32_history" else "f64",
        "data": "synthetic",
        "config": {"workload": "sphere eps_r=12, %d^3 voxels (%d), c dt = h, hp9 FIR "
                               "delta=1e-7*M, +z x-polarised modulated Gaussian plane wave"
                               % (round(M ** (1 / 3)), M),
                   "history": "direct spectral lag sum (all %d lags per step)" % head["ell"],
                   "P": head["P"], "l2_flush": "inputs larger than L2 (spectral ring)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        "gpu_launches": head["launches"],
        "e2e": e2e,
        "cpu_baseline": cpu,
        "precisions": results,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
