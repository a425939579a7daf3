"""Truncated interaction table (mot_truncate_table) and the tapered frequency
response (mot_frequency_response) against the oracle (Secs. 6, 7.1)."""
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


@pytest.fixture(scope="module")
def trunc_case():
    """6^3 heterogeneous grid and a truncation step q chosen so that no oracle element
    of a history lag lies within 1e-10 of the largest element of a rounding midpoint:
    the two sides' tables agree to 1e-12 of the largest element, so both round every
    element to the same multiple of q."""
    from oracle import excitation, kernel_table, march
    from oracle.spline import num_lags
    N = 6
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    rng = np.random.default_rng(31)
    eps = 2.0 + 6.0 * rng.uniform(size=(N, N, N))
    taps = wl.fir_taps("fir3", 0.01)
    q = None
    for s in (1.0, 1.13, 1.37, 1.71, 1.93, 2.29, 2.71, 3.17):
        cand = 1e-6 * s
        r = G[1:] / cand
        if np.abs(r - np.floor(r) - 0.5).min() * cand > 1e-10 * np.abs(G).max():
            q = cand
            break
    assert q is not None
    Gt = G.copy()
    Gt[1:] = q * np.rint(G[1:] / q)
    p = wl.pulse(N, 8.0)
    E = excitation.tested_excitation(eps, p, 90)
    J = march.march(Gt, eps, taps, E)
    return {"N": N, "ell": ell, "eps": eps, "taps": taps, "q": q, "Gt": Gt, "E": E, "J": J}


def test_truncated_table_matches_oracle(mot, trunc_case):
    o = trunc_case
    with mot.Context(o["eps"], o["taps"]) as plain:
        g0 = plain.table(0, o["ell"] + 1)
    with mot.Context(o["eps"], o["taps"]) as ctx:
        ctx.truncate_table(o["q"])
        g = ctx.table(0, o["ell"] + 1)
    assert np.array_equal(g[0], g0[0])                      # lag 0 (the Z_0 stencil) kept
    assert np.array_equal(g[1:], o["Gt"][1:])               # same multiples of q as the oracle
    assert np.abs(g[1:] - g0[1:]).max() <= 0.5 * o["q"] * (1 + 1e-12)


@pytest.mark.parametrize("precision,scheme,tol", [("fp64", "direct", 1e-10),
                                                  ("fp64", "blocked", 1e-10),
                                                  ("fp32_history", "blocked", 5e-5)])
def test_truncated_march_matches_oracle(mot, trunc_case, precision, scheme, tol):
    o = trunc_case
    with mot.Context(o["eps"], o["taps"], precision=precision, scheme=scheme, block=4) as ctx:
        ctx.truncate_table(o["q"])
        ctx.set_excitation(o["E"])
        J = ctx.march(o["E"].shape[0])
    err = np.linalg.norm(J - o["J"]) / np.linalg.norm(o["J"])
    assert err < tol


def test_truncate_refuses_marched_or_shared(mot):
    with mot.Context(wl.cube(4, 4.0)) as ctx:
        s = ctx.share()
        with pytest.raises(mot.MotError, match="shared"):
            ctx.truncate_table(1e-6)
        s.close()
        ctx.march(2)
        with pytest.raises(mot.MotError, match="before the first step"):
            ctx.truncate_table(1e-6)


def test_frequency_response_matches_oracle(mot):
    torch = pytest.importorskip("torch")
    from oracle import response
    rng = np.random.default_rng(8)
    N, npr = 700, 5
    J = rng.normal(size=(N, npr, 3))
    eps_p = 2.0 + 10.0 * rng.uniform(size=npr)
    p = wl.pulse(20, 12.0)
    freqs = np.linspace(0.2, 2.0, 37) * p["f_c"]
    H, jh = mot.frequency_response(J, 1.0, 0.2, eps_p, p["f_c"], p["sigma_t"], freqs,
                                   with_spectrum=True)
    ref_j = response.tapered_dft(J, 1.0, 0.2, freqs)
    ref = response.frequency_response(J, 1.0, 0.2, eps_p, p["f_c"], p["sigma_t"], freqs)
    assert np.abs(jh - ref_j).max() <= 1e-12 * np.abs(ref_j).max()
    assert np.abs(H - ref).max() <= 1e-12 * np.abs(ref).max()
    Hd = mot.frequency_response(torch.tensor(J, device="cuda"), 1.0, 0.2, eps_p, p["f_c"],
                                p["sigma_t"], freqs)
    assert np.array_equal(Hd, H)


def test_experiment_drivers_run_small(mot):
    """The diagnostics drivers end to end on small grids (shapes and bookkeeping)."""
    from paper_2407_03323_gb300 import diagnostics as dg
    rows = dg.pdsa_scan([4, 6], k=400)
    assert [r["N"] for r in rows] == [4, 6] and all(r["steps"] >= 2 for r in rows)
    assert all(r["bracket"][0] <= r["theta_min"] <= r["theta_max"] <= r["bracket"][1]
               for r in rows)
    tr = dg.truncation_experiment(N=6, eps_list=(0.0, 1e-6), steps=160, k=200)
    assert len(tr) == 2 and tr[0]["steps"] == 160
    fs = dg.fir_sweep(N=6, steps=160)
    assert set(fs) == {"none", "fir2", "fir3", "fir4"} and "fir_magnitude" in fs["fir3"]
    sp = dg.sphere100(N=12, steps=96)
    assert sp["steps"] == 96 and sp["fail_step"] == 0
    rs = dg.response(N=8, steps=400, n_freq=40)
    assert rs["steps"] == 400 and len(rs["top_Hx"]) == 5
