"""Diagnostics of the stabilisation study (Secs. 5.1, 6, 7): experiment drivers over
the library's entry points (argument marshalling and bookkeeping only; every operator
application, march step and transform runs in the library's kernels).

    python -m paper_2407_03323_gb300.diagnostics pdsa --sides 4,8,14,20,32
    python -m paper_2407_03323_gb300.diagnostics truncation
    python -m paper_2407_03323_gb300.diagnostics fir
    python -m paper_2407_03323_gb300.diagnostics sphere100
    python -m paper_2407_03323_gb300.diagnostics response
    python -m paper_2407_03323_gb300.diagnostics adjoint
    python -m paper_2407_03323_gb300.diagnostics stability

* pdsa        smallest eigenvalue of A_n = diag(1/chi) D_n / C(ell, n) (Eq. Dn) on
              cubes of growing side: Lanczos Ritz values (a negative one certifies that
              D_n is indefinite), the circulant bracket, and the PDSA-guided delta (the
              smallest delta that lifts the Ritz estimate of lambda_min(D_ell^delta) to
              zero: D_ell^delta = D_ell + delta I, so A_ell grows by delta / chi);
              optionally with every lag spectrum rounded to FP32 (the FP32-history
              store), and every n = 0..ell.
* truncation  the truncated MOT-JVIE of Sec. 6: elements of the history lags rounded
              to eps_trunc, the growth per step of the alternating (theta = pi) part of
              the solution, and lambda_min(A_ell) of the truncated table.
* fir         FIR2 / FIR3 / FIR4 at delta = 0.1 against the unregularised march on the
              eps_r = 12 cube (Sec. 6.2): difference normalised by the peak, late growth.
* sphere100   the eps_r = 100 sphere (Sec. 7.2 scale) with FIR3 delta = 1e-7 M: stable
              march, CG iterations and time per step.
* response    |H^alpha| with the 20 % cosine taper (Eq. Halpha, Sec. 7.1) at a probe of
              the eps_r = 12 cube after a FIR3 march.
* adjoint     gradient of the gated scattered-field energy at 64 probes around a
              heterogeneous 48^3 block (2048 steps, checkpoints every 64) against central
              differences at 32 voxels.
* stability   the 104^3 eps_r = 12 sphere marched 40,960 steps (10x the workload) in
              FP32-history: maxima of ||J_n|| over every 2048 steps.

Geometry as in the paper: the 0.2 m cube discretised by N^3 voxels with c0 dt = h,
probe r = (0.025, 0.075, 0.025) m -> voxel (N/8, 3N/8, N/8), the x-polarised Gaussian
plane wave travelling along -z, T = 100 light-metres = 500 N steps (shortened by
--steps).
"""
import argparse
import json
import math
import time

import numpy as np

from . import mot as _mot

import workloads as wl


def _growth_per_step(x, frac=0.3, win=16):
    """|lambda| of the dominant late theta = pi (per-step alternating) behaviour: the
    second difference (x_n - 2 x_{n-1} + x_{n-2}) / 4 keeps theta = pi with gain 1 and
    damps slow ringing by sin^2(pi f dt); over the last `frac` of the series the
    maxima of windows of `win` steps are fitted by a line in log scale, whose slope per
    step gives the growth factor."""
    x = np.asarray(x, float)
    d = np.abs(x[2:] - 2 * x[1:-1] + x[:-2]) / 4.0
    n0 = int(len(d) * (1 - frac))
    seg = d[n0:]
    nb = seg.size // win
    if nb < 4 or not np.all(np.isfinite(seg)):
        return float("nan")
    peaks = seg[:nb * win].reshape(nb, win).max(axis=1)
    if peaks.min() <= 0.0:
        return float("nan")
    t = win * np.arange(nb)
    slope = np.polyfit(t, np.log(peaks), 1)[0]
    return float(math.exp(slope))


def _probe_index(N, frac=(0.125, 0.375, 0.125)):
    u, v, w = (min(N - 1, int(math.floor(f * N))) for f in frac)
    return u + N * (v + N * w)


def _march_probe(ctx, wave, steps, probes, chunk=64):
    """March `steps` steps of the tested plane wave; returns (J at probes [steps][P][3],
    ||J_n|| per step, step of the first failure or 0)."""
    import torch
    M = ctx.M
    idx = torch.as_tensor(np.asarray(probes), device="cuda")
    Jc = torch.empty((chunk, M, 3), dtype=torch.float64, device="cuda")
    E = torch.empty((chunk, M, 3), dtype=torch.float64, device="cuda")
    out = np.zeros((steps, len(probes), 3))
    norms = np.zeros(steps)
    # the pulse peaks at t0 + r . k_hat; after t_end it is below exp(-32) everywhere and
    # the steps are marched with E = 0 (nothing staged)
    W, V, U = ctx.shape
    t_end = wave["t0"] + math.sqrt(U * U + V * V + W * W) + 8.0 * wave["sigma_t"]
    done, fail = 0, 0
    while done < steps:
        k = min(chunk, steps - done)
        if done + 1 <= t_end:
            ctx.plane_wave(wave["k_hat"], wave["p_hat"], wave["f_c"], wave["sigma_t"],
                           wave["t0"], done + 1, k, out=E[:k])
            ctx.set_excitation(E[:k])
        try:
            ctx.march(k, out=Jc[:k])
        except _mot.MotError:
            fail = ctx.info()["fail_step"] or done + 1
            out = out[:done]
            norms = norms[:done]
            break
        out[done:done + k] = Jc[:k][:, idx].cpu().numpy()
        norms[done:done + k] = torch.linalg.vector_norm(Jc[:k].reshape(k, -1), dim=1).cpu().numpy()
        done += k
    return out, norms, fail


def _paper_wave(N, eps_r):
    """x-polarised plane wave along -z; t0 = 6 sigma_t - min_box(r . k_hat) = 6 sigma_t
    + N, so the pulse (peak at t = t0 + r . k_hat) is still 6 sigma_t away from every
    voxel at t = 0."""
    p = wl.pulse(N, eps_r, k_hat=(0.0, 0.0, -1.0), p_hat=(1.0, 0.0, 0.0))
    p["t0"] = 6.0 * p["sigma_t"] + N
    return p


# ------------------------------------------------------------------------- PDSA
def pdsa_scan(sides, eps_r=12.0, k=20000, fp32_spectrum=False, all_n=False, k_n=2000, seed=1,
              taps=None):
    rows = []
    for N in sides:
        t0 = time.perf_counter()
        with _mot.Context(wl.cube(N, eps_r), taps) as ctx:
            ell = ctx.ell
            r = ctx.pdsa_lanczos(ell, k, seed=seed, fp32_spectrum=fp32_spectrum, n_out=4)
            b = ctx.pdsa_bounds(ell, fp32_spectrum=fp32_spectrum)
            row = {"N": N, "M": N ** 3, "ell": ell, "steps": r["steps"],
                   "theta_min": r["theta_min"], "resid_min": r["resid_min"],
                   "lowest_ritz": r["ritz"].tolist(),
                   "theta_max": r["theta_max"], "resid_max": r["resid_max"],
                   "bracket": [b["lo"], b["hi"]], "chi_max": b["chi_max"],
                   "fp32_spectrum": fp32_spectrum}
            if r["theta_min"] < -r["resid_min"]:
                row["status"] = "indefinite (negative Ritz value)"
            elif b["lo"] > 0.0:
                row["status"] = "positive definite (bracket)"
            elif r["resid_min"] < 0.01 * r["theta_min"]:
                row["status"] = "converged smallest Ritz value > 0"
            else:
                row["status"] = "not converged in %d steps" % r["steps"]
            # delta that lifts the estimate theta_min - resid_min of lambda_min to 0
            row["delta_guided"] = max(0.0, -(r["theta_min"] - r["resid_min"])) * b["chi_max"]
            row["delta_paper"] = 1e-7 * N ** 3
            if all_n:
                row["theta_min_n"] = [ctx.pdsa_lanczos(n, k_n, seed=seed,
                                                       fp32_spectrum=fp32_spectrum)["theta_min"]
                                      for n in range(ell + 1)]
        row["seconds"] = time.perf_counter() - t0
        rows.append(row)
    return rows


# ------------------------------------------------------------------- truncation
def truncation_experiment(N=20, eps_r=2.0, eps_list=(0.0, 1e-9, 1e-8, 1e-7, 1e-6, 1e-5),
                          steps=None, precision="fp64", scheme="direct", k=5000):
    steps = steps or 500 * N
    wave = _paper_wave(N, eps_r)
    probe = _probe_index(N)
    rows = []
    for q in eps_list:
        t0 = time.perf_counter()
        with _mot.Context(wl.cube(N, eps_r), precision="fp64", scheme="direct") as an:
            if q > 0:
                an.truncate_table(q)
            lz = an.pdsa_lanczos(an.ell, k, seed=1)
        with _mot.Context(wl.cube(N, eps_r), precision=precision, scheme=scheme,
                          block=8 if scheme == "blocked" else 0) as ctx:
            if q > 0:
                ctx.truncate_table(q)
            ctx.set_solver(growth_limit=1e30)
            J, norms, fail = _march_probe(ctx, wave, steps, [probe])
        jx = J[:, 0, 0]
        rows.append({"eps_trunc": q, "steps": len(jx), "fail_step": fail,
                     "growth_per_step": _growth_per_step(jx),
                     "late_over_peak": float(np.abs(jx[-len(jx) // 10:]).max() / np.abs(jx).max())
                     if len(jx) else float("nan"),
                     "theta_min_A_ell": lz["theta_min"], "resid": lz["resid_min"],
                     "seconds": time.perf_counter() - t0})
    return rows


# -------------------------------------------------------------------- FIR sweep
def fir_sweep(N=20, eps_r=12.0, delta=0.1, filters=("none", "fir2", "fir3", "fir4"),
              steps=None, precision="fp64", scheme="direct"):
    steps = steps or 500 * N
    wave = _paper_wave(N, eps_r)
    probe = _probe_index(N)
    series = {}
    info = {}
    for f in filters:
        taps = None if f == "none" else wl.fir_taps(f, delta)
        t0 = time.perf_counter()
        with _mot.Context(wl.cube(N, eps_r), taps, precision=precision, scheme=scheme,
                          block=8 if scheme == "blocked" else 0) as ctx:
            ctx.set_solver(growth_limit=1e30)
            J, norms, fail = _march_probe(ctx, wave, steps, [probe])
        series[f] = J[:, 0, 0]
        info[f] = {"fail_step": fail, "growth_per_step": _growth_per_step(J[:, 0, 0]),
                   "seconds": time.perf_counter() - t0}
    ref = series.get("none")
    for f in filters:
        x = series[f]
        info[f]["steps"] = len(x)
        info[f]["late_over_peak"] = (float(np.abs(x[-len(x) // 10:]).max() / np.abs(x).max())
                                     if len(x) else float("nan"))
    theta = np.linspace(0.0, math.pi, 9)
    for f in filters:
        if f != "none":
            info[f]["fir_magnitude"] = _mot.fir_magnitude(wl.fir_taps(f, delta), theta).tolist()
        if ref is not None and f != "none":
            n = min(len(ref), len(series[f]))
            peak = np.abs(ref[:n]).max()
            # difference over the first half (before any late unregularised growth)
            h = n // 2
            info[f]["max_diff_over_peak_first_half"] = float(np.abs(series[f][:h] - ref[:h]).max() / peak)
    return info


# ---------------------------------------------------------------- eps_r = 100
def sphere100(N=105, eps_r=100.0, steps=2000, precision="fp32_history", block=8):
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    wave = _paper_wave(N, eps_r)
    probe = [_probe_index(N, (0.5, 0.5, 0.5)), _probe_index(N, (0.3, 0.5, 0.7))]
    import torch
    with _mot.Context(wl.sphere(N, eps_r), taps, precision=precision, scheme="blocked",
                      block=block) as ctx:
        ctx.set_solver(growth_limit=1e30)
        ctx.set_profiling(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, norms, fail = _march_probe(ctx, wave, steps, probe)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = ctx.stats()
    ms = {k: st[k] / max(st["steps"], 1) for k in st if k.startswith("ms_")}
    return {"N": N, "eps_r": eps_r, "steps": len(norms), "fail_step": fail,
            "peak_norm": float(norms.max()) if len(norms) else None,
            "last_over_peak": float(norms[-1] / norms.max()) if len(norms) else None,
            "cg_iters_per_step": st["cg_iters"] / max(st["steps"], 1),
            "ms_per_step_phases": ms, "wall_s_incl_excitation": wall,
            "growth_per_step": _growth_per_step(J[:, 0, 0])}


# ------------------------------------------------------------ |H^alpha| (Eq. Halpha)
def response(N=20, eps_r=12.0, delta=0.1, steps=None, taper=0.2, n_freq=200):
    steps = steps or 500 * N
    wave = _paper_wave(N, eps_r)
    probe = _probe_index(N)
    with _mot.Context(wl.cube(N, eps_r), wl.fir_taps("fir3", delta), scheme="blocked",
                      block=8, precision="fp32_history") as ctx:
        J, norms, fail = _march_probe(ctx, wave, steps, [probe])
    fmax = 2.0 * wave["f_c"]
    freqs = np.linspace(fmax / n_freq, fmax, n_freq)
    H = _mot.frequency_response(J, 1.0, taper, [eps_r], wave["f_c"], wave["sigma_t"], freqs)
    Hx = H[:, 0, 0]
    top = np.argsort(Hx)[::-1][:5]
    return {"N": N, "steps": len(J), "fail_step": fail,
            "f_c": wave["f_c"], "freqs_at_top_Hx": freqs[top].tolist(),
            "top_Hx": Hx[top].tolist(),
            "Hx_at_fc": float(np.interp(wave["f_c"], freqs, Hx))}


def adjoint_probes(N=48, steps=2048, n_probes=64, checkpoint=64, n_fd=32, h=1e-4,
                   precision="fp64", scheme="blocked", block=8, seed=240703324):
    """The adjoint workload: gradient of the time-gated scattered-field energy at probes
    around a heterogeneous block with respect to every voxel's eps_r.

    eps_r = 1 + 11 x smoothed seeded noise on an N^3 block; the x-polarised +z plane wave
    for eps_r = 12; O = sum_{n >= N/2} sum_p |E^s_p(t_n)|^2 over a Fibonacci lattice of
    probes on the sphere of radius 2N; dO/deps_r by the probe field's transpose and the
    adjoint march with currents checkpointed every `checkpoint` steps
    (torch.autograd); checked by central differences of two forward marches at n_fd
    seeded voxels.  Returns the errors and the times."""
    import torch
    from .autograd import march, probe_field
    eps0 = wl.heterogeneous_block(N)
    taps = wl.fir_taps("none")
    p = wl.pulse(N, 12.0)
    wave = {k: p[k] for k in ("k_hat", "p_hat", "f_c", "sigma_t", "t0")}
    first = N // 2
    opts = {"precision": precision, "scheme": scheme, "block": block}
    probes = wl.fibonacci_probes(N, n_probes)
    t = time.time()
    pctx = _mot.Context(eps0, precision="fp32_history")
    pctx.probe_setup(probes)
    t_setup = time.time() - t

    def objective(J):
        return (probe_field(J, pctx)[first:] ** 2).sum()

    eps = torch.tensor(eps0, dtype=torch.float64, requires_grad=True)
    t = time.time()
    O = objective(march(eps, taps, wave, steps, checkpoint_every=checkpoint, **opts))
    O.backward()
    torch.cuda.synchronize()
    t_grad = time.time() - t
    grad = eps.grad.numpy().reshape(-1)
    gmax = float(np.abs(grad).max())

    def value(e):
        with torch.no_grad():
            return float(objective(march(torch.tensor(e), taps, wave, steps, **opts)))

    rng = np.random.default_rng(seed)
    voxels = rng.choice(eps0.size, n_fd, replace=False)
    rows, worst = [], 0.0
    t = time.time()
    for m in voxels:
        ep = eps0.copy().reshape(-1)
        em = eps0.copy().reshape(-1)
        ep[m] += h
        em[m] -= h
        fd = (value(ep.reshape(eps0.shape)) - value(em.reshape(eps0.shape))) / (2 * h)
        err = abs(fd - grad[m]) / max(abs(fd), 1e-2 * gmax)
        worst = max(worst, err)
        rows.append({"voxel": int(m), "eps_r": float(eps0.reshape(-1)[m]), "fd": fd,
                     "adjoint": float(grad[m]), "rel_err": err})
    t_fd = time.time() - t
    pctx.close()
    return {"N": N, "steps": steps, "probes": int(len(probes)), "gate_from_step": first + 1,
            "checkpoint_every": checkpoint, "objective": float(O.detach()), "grad_max": gmax,
            "fd_step": h, "max_rel_err": worst, "voxels": rows, "probe_setup_s": t_setup,
            "gradient_s": t_grad, "fd_s_per_march": t_fd / (2 * n_fd), **opts}


def stability(config="sphere104", steps=40960, window=2048, chunk=256,
              precision="fp32_history", scheme="blocked", block=8):
    """Late-time stability of a long march (Secs. 5.2, 6): the workload's pulse, then
    E = 0; ||J_n|| of every step (summed on the device), reported as the maximum over
    each window of `window` steps.  The FIR-regularised march is stable when these
    maxima never grow after the pulse."""
    import torch
    cfg = wl.config(config)
    eps, taps, p = cfg["eps_r"], cfg["taps"], cfg["pulse"]
    ctx = _mot.Context(eps, taps, precision=precision, scheme=scheme, block=block)
    M = ctx.M
    buf = torch.empty((chunk, M, 3), dtype=torch.float64, device="cuda")
    E = torch.empty((chunk, M, 3), dtype=torch.float64, device="cuda")
    norms = []
    t = time.time()
    for n0 in range(1, steps + 1, chunk):
        k = min(chunk, steps + 1 - n0)
        if n0 <= 2 * p["t0"]:                     # the pulse; E = 0 once it has passed
            ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"], n0, k,
                           out=E[:k])
            ctx.set_excitation(E[:k])
        ctx.march(k, out=buf[:k])
        norms.append(torch.linalg.vector_norm(buf[:k].reshape(k, -1), dim=1).cpu().numpy())
    torch.cuda.synchronize()
    wall = time.time() - t
    norms = np.concatenate(norms)
    ctx.close()
    wins = [float(norms[i:i + window].max()) for i in range(0, steps, window)]
    after = wins[1:]
    return {"config": config, "precision": precision, "scheme": scheme, "steps": steps,
            "finite": bool(np.all(np.isfinite(norms))), "peak": float(norms.max()),
            "window": window, "window_max": wins,
            "never_grows_after_first": bool(all(b <= a for a, b in zip(after, after[1:]))),
            "last_over_peak": wins[-1] / float(norms.max()), "wall_s": wall,
            "ms_per_step": 1e3 * wall / steps}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("what", choices=["pdsa", "truncation", "fir", "sphere100", "response",
                                     "adjoint", "stability"])
    ap.add_argument("--sides", default="4,6,8,10,12,14,16,20,24,32")
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--k", type=int, default=20000)
    ap.add_argument("--fp32-spectrum", action="store_true")
    ap.add_argument("--all-n", action="store_true")
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_history"])
    ap.add_argument("--scheme", default="direct", choices=["direct", "blocked", "blocked_doubling"])
    ap.add_argument("--filters", default="none,fir2,fir3,fir4")
    ap.add_argument("--delta", type=float, default=0.1)
    a = ap.parse_args(argv)
    if a.what == "pdsa":
        out = pdsa_scan([int(s) for s in a.sides.split(",")], eps_r=a.eps or 12.0, k=a.k,
                        fp32_spectrum=a.fp32_spectrum, all_n=a.all_n)
    elif a.what == "truncation":
        out = truncation_experiment(N=a.N or 20, eps_r=a.eps or 2.0, steps=a.steps)
    elif a.what == "fir":
        out = fir_sweep(N=a.N or 20, eps_r=a.eps or 12.0, steps=a.steps, delta=a.delta,
                        filters=tuple(a.filters.split(",")), precision=a.precision,
                        scheme=a.scheme)
    elif a.what == "sphere100":
        out = sphere100(N=a.N or 105, eps_r=a.eps or 100.0, steps=a.steps or 2000)
    elif a.what == "adjoint":
        out = adjoint_probes(N=a.N or 48, steps=a.steps or 2048)
    elif a.what == "stability":
        out = stability(steps=a.steps or 40960, precision=a.precision
                        if a.precision != "fp64" else "fp32_history")
    else:
        out = response(N=a.N or 20, eps_r=a.eps or 12.0, steps=a.steps)
    print(json.dumps(out, indent=1, default=float))


if __name__ == "__main__":
    main()
