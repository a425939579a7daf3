"""Parity with the oracle at the padded FFT lengths the full-size workloads run.

* Sparse-source histories (Eq. PnMOT): the history P_{n-1} of a past supported on a
  few source voxels, through the library's FFT / ring / MAC path (mot_eval_history),
  against the oracle's direct sum over those sources (element quadrature per offset,
  no FFT), at the sources and at sampled voxels.  Grids: 104^3 (padded length 210:
  the 14 x 15 four-step codelets of every pass), 48^3 (96 = 8 x 12), and 150 x 6 x 5
  (300 along x: the generic Stockham passes).  FP64 and FP32-history, direct and both
  blocked level plans (B = 8; doubling levels up to S = 128, or the last level fitted
  to ell; the longest lags are reached by sources in opposite corners).
* A 320-step FP64 march of a 16^3 sphere (padded 32) with the 9-tap FIR against the
  oracle's direct-sum march (C loops over voxel pairs and lags, dense LU of Z_0), in
  the direct and the blocked scheme, and the FP32-history march against it.

Tolerances.  FP64: the two sides' element quadratures agree to ~1e-12 of the largest
element at an offset and an FP64 FFT adds ~1e-15 of the global scale, so each sampled
component must agree to 1e-11 of max(|P| there, 1e-3 max |P|).  FP32-history: the
spectra, transforms and lag products carry FP32 rounding (unit 6e-8) through about
log2(P^3) ~ 23 butterfly levels in each direction, i.e. a few 1e-6 of the L2 norm of
the spectrum, spread over all voxels; every sampled component must agree to 2e-6 of
the largest |P| over the sampled voxels (which include the sources, where |P| peaks).
"""
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mot():
    from paper_2407_03323_gb300 import build, mot as m
    if not os.path.exists(m.LIB_PATH):
        build.build()
    m.load_library()
    return m


def _grid(name):
    rng = np.random.default_rng(240703323)
    if name == "cube104":
        eps = 2.0 + 10.0 * rng.uniform(size=(104, 104, 104))
    elif name == "block48":
        eps = wl.heterogeneous_block(48)
    else:                                            # "long150"
        eps = 2.0 + 10.0 * rng.uniform(size=(5, 6, 150))
        eps[2, 3, 40:44] = 1.0
    return eps


def _sources_and_targets(eps, rng, n_src=10, n_tgt=14):
    """Sources in opposite corners and on the faces (so that the largest offsets, and
    hence the longest lags and the last far level, are reached) plus random active
    voxels; targets = the sources plus random voxels (active and not)."""
    W, V, U = eps.shape
    e = eps.reshape(-1)
    corners = [(0, 0, 0), (U - 1, V - 1, W - 1), (U - 1, 0, W // 2), (0, V - 1, W - 1),
               (U // 2, V // 2, 0)]
    src = []
    for u, v, w in corners:
        m = u + U * (v + V * w)
        if e[m] > 1.0 and m not in src:
            src.append(m)
    active = np.nonzero(e > 1.0)[0]
    while len(src) < n_src:
        m = int(rng.choice(active))
        if m not in src:
            src.append(m)
    tgt = list(src)
    while len(tgt) < len(src) + n_tgt:
        m = int(rng.integers(0, e.size))
        if m not in tgt:
            tgt.append(m)
    return src, tgt


@pytest.mark.parametrize("name", ["cube104", "block48", "long150"])
def test_sparse_history_against_oracle_full_size(mot, name):
    from oracle import march as om
    eps = _grid(name)
    taps = wl.fir_taps("fir3", 1e-7 * eps.size)
    rng = np.random.default_rng(17)
    src, tgt = _sources_and_targets(eps, rng)
    W, V, U = eps.shape
    ell = int(np.floor(np.sqrt(U * U + V * V + W * W))) + 2
    Jsrc = rng.normal(size=(ell, len(src), 3))
    ref = om.history_sparse(eps, taps, src, Jsrc, tgt, ell + 1)
    scale = np.abs(ref).max()
    Jh = np.zeros((ell, eps.size, 3))
    Jh[:, src] = Jsrc
    # level plans (S, first lag) at ell = 182, 85, 152
    doubling = {"cube104": [8, 16, 32, 64, 128], "block48": [8, 16, 32, 64],
                "long150": [8, 16, 32, 64, 128]}[name]
    fitted = {"cube104": ([8, 16, 32, 64, 64], [8, 16, 32, 64, 128]),
              "block48": ([8, 16, 32, 32], [8, 16, 32, 64]),
              "long150": ([8, 16, 32, 64, 32], [8, 16, 32, 64, 128])}[name]
    for scheme in ("direct", "blocked", "blocked_doubling"):
        for prec in ("fp64", "fp32_history"):
            with mot.Context(eps, taps, precision=prec, scheme=scheme,
                             block=0 if scheme == "direct" else 8) as ctx:
                assert ctx.ell == ell
                if name == "cube104":
                    assert ctx.P == (210, 210, 210)
                elif name == "block48":
                    assert ctx.P == (96, 96, 96)
                else:
                    assert ctx.P[0] == 300
                if scheme == "blocked_doubling":
                    assert ctx.levels == doubling and ctx.level_lags == doubling
                elif scheme == "blocked":
                    assert (ctx.levels, ctx.level_lags) == fitted
                P = ctx.eval_history(Jh)[tgt]
            err = np.abs(P - ref)
            if prec == "fp64":
                local = np.maximum(np.abs(ref), 1e-3 * scale)
                worst = float((err / local).max())
                assert worst < 1e-11, (scheme, prec, worst)
            else:
                worst = float(err.max() / scale)
                assert worst < 2e-6, (scheme, prec, worst)


@pytest.fixture(scope="module")
def sphere16_oracle():
    from oracle import direct, excitation, kernel_table
    from oracle.spline import num_lags
    N = 16
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("hp9", 1e-7 * N ** 3)
    p = wl.pulse(N, 12.0, k_hat=(1.0, 2.0, 2.0), p_hat=(0.0, 1.0, -1.0))
    steps = 320
    n_first = int(p["t0"]) - 100               # start on the rising edge of the pulse
    G, _, _ = kernel_table.octant_table(N, num_lags(N, N, N) + 1)
    E = excitation.tested_excitation(eps, p, steps, n_first=n_first)
    J = direct.march(G, eps, taps, E)
    return {"eps": eps, "taps": taps, "p": p, "steps": steps, "n_first": n_first, "J": J}


@pytest.mark.parametrize("precision,scheme,tol", [("fp64", "direct", 1e-10),
                                                  ("fp64", "blocked", 1e-10),
                                                  ("fp32_history", "blocked", 1e-5)])
def test_long_march_sphere16_fir9_against_oracle(mot, sphere16_oracle, precision, scheme, tol):
    """320 steps of the 16^3 eps_r = 12 sphere with the 9-tap FIR, excitation computed
    on each side independently; blocked scheme B = 4 (levels 4, 8, 16 over ell = 29)."""
    o = sphere16_oracle
    p = o["p"]
    with mot.Context(o["eps"], o["taps"], precision=precision, scheme=scheme,
                     block=4 if scheme == "blocked" else 0) as ctx:
        assert ctx.P == (32, 32, 32)
        E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"],
                           o["n_first"], o["steps"])
        ctx.set_excitation(E)
        J = ctx.march(o["steps"])
    ref = o["J"]
    assert np.linalg.norm(ref[-1]) > 1e-3 * np.abs(ref).max()   # still ringing at the end
    rel = np.linalg.norm(J - ref) / np.linalg.norm(ref)
    assert rel < tol, rel
