"""Positive definite stability analysis on the device (mot_pdsa_apply, mot_pdsa_bounds,
mot_pdsa_lanczos; Sec. 5.1, Eq. Dn) against the oracle's dense
A_n = diag(1/chi) D_n / C(ell, n) on the active voxels and its circulant embedding.

Tolerances: the element tables of the two sides are independent FP64 quadratures that
agree to 1e-12 of the largest element, so products agree to ~1e-11 of max|y| and
eigenvalues to ~1e-10 of the operator's norm."""
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


def _case(N, seed, inactive=2):
    from oracle import kernel_table
    from oracle.spline import num_lags
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    rng = np.random.default_rng(seed)
    eps = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    eps[0, 0, :inactive] = 1.0
    return ell, G, eps


@pytest.fixture(scope="module")
def case6():
    ell, G, eps = _case(6, 21)
    return {"ell": ell, "G": G, "eps": eps, "taps": wl.fir_taps("fir3", 0.05)}


@pytest.mark.parametrize("fp32", [False, True])
def test_apply_matches_oracle(mot, case6, fp32):
    from oracle import pdsa
    o = case6
    x = np.random.default_rng(4).normal(size=(6 ** 3, 3))
    with mot.Context(o["eps"], o["taps"]) as ctx:
        assert ctx.ell == o["ell"]
        for n in (0, 1, 6, o["ell"]):
            y = ctx.pdsa_apply(n, x, fp32_spectrum=fp32)
            ref = pdsa.circulant_apply(o["G"], o["eps"], o["taps"], o["ell"], n, ctx.P, x,
                                       round32=fp32)
            assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max(), n
            if not fp32 and n in (0, o["ell"]):
                act = o["eps"].reshape(-1) > 1.0
                A = pdsa.scaled_pdsa_matrix(o["G"], o["eps"], o["taps"], o["ell"], n)
                yd = (A @ x[act].reshape(-1)).reshape(-1, 3)
                assert np.abs(y[act] - yd).max() <= 1e-11 * np.abs(yd).max()
                assert np.all(y[~act] == 0.0)


def test_apply_device_buffers(mot, case6):
    torch = pytest.importorskip("torch")
    o = case6
    x = np.random.default_rng(5).normal(size=(6 ** 3, 3))
    with mot.Context(o["eps"], o["taps"]) as ctx:
        yh = ctx.pdsa_apply(o["ell"], x)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        ctx.pdsa_apply(o["ell"], xd, out=yd)
        assert np.array_equal(yd.cpu().numpy(), yh)


def test_bounds_match_oracle(mot, case6):
    from oracle import pdsa
    o = case6
    with mot.Context(o["eps"], o["taps"]) as ctx:
        for n in (0, 6, o["ell"]):
            b = ctx.pdsa_bounds(n)
            lo, hi, smin, smax = pdsa.circulant_bounds(o["G"], o["eps"], o["taps"], o["ell"],
                                                       n, ctx.P)
            scale = max(abs(smin), abs(smax))
            for got, ref in ((b["lo"], lo), (b["hi"], hi), (b["symbol_min"], smin),
                             (b["symbol_max"], smax)):
                assert abs(got - ref) <= 1e-10 * scale, (n, got, ref)
            e = o["eps"][o["eps"] > 1.0]
            assert b["chi_max"] == pytest.approx(((e - 1) / e).max(), rel=1e-15)


def test_lanczos_full_dimension(mot):
    """Full reorthogonalisation with k = dim: the Ritz values are the eigenvalues
    (extremes to 1e-9 of ||A||)."""
    from oracle import pdsa
    ell, G, eps = _case(4, 22)
    taps = wl.fir_taps("fir3", 0.02)
    dim = 3 * int((eps > 1.0).sum())
    with mot.Context(eps, taps) as ctx:
        for n in (0, ell):
            lam = np.linalg.eigvalsh(pdsa.scaled_pdsa_matrix(G, eps, taps, ell, n))
            r = ctx.pdsa_lanczos(n, dim, seed=3, reorth=True, n_out=dim)
            th = r["ritz"]
            norm = np.abs(lam).max()
            assert r["steps"] <= dim and len(th) == r["steps"]
            assert abs(th[0] - lam[0]) <= 1e-9 * norm and th[0] == r["theta_min"]
            assert abs(r["theta_max"] - lam[-1]) <= 1e-9 * norm
            assert max(r["resid_min"], r["resid_max"]) <= 1e-8 * norm


def test_lanczos_cube8(mot):
    """eps_r = 12 cube, N = 8, D_ell without taps (the smallest eigenvalue, 6.2e-6 of a
    spectrum reaching 2.6, is three-fold): the plain recurrence run past the dimension
    converges to lambda_min; 150 reorthogonalised steps give an upper bound within its
    residual of an eigenvalue, inside the circulant bracket."""
    from oracle import pdsa
    ell, G, _ = _case(8, 0, inactive=0)
    eps = wl.cube(8, 12.0)
    lam = np.linalg.eigvalsh(pdsa.scaled_pdsa_matrix(G, eps, np.zeros(0), ell, ell))
    tol = 1e-10 * np.abs(lam).max()
    with mot.Context(eps) as ctx:
        plain = ctx.pdsa_lanczos(ell, 6000, seed=1)
        r = ctx.pdsa_lanczos(ell, 150, seed=1, reorth=True)
        b = ctx.pdsa_bounds(ell)
    assert abs(plain["theta_min"] - lam[0]) <= 1e-3 * lam[0]
    assert abs(plain["theta_max"] - lam[-1]) <= tol
    assert plain["ritz"][0] == plain["theta_min"] and np.all(np.diff(plain["ritz"]) >= 0)
    assert r["theta_min"] >= lam[0] - tol and r["theta_max"] <= lam[-1] + tol
    assert np.abs(lam - r["theta_min"]).min() <= r["resid_min"] + tol
    assert np.abs(lam - r["theta_max"]).min() <= r["resid_max"] + tol
    assert b["lo"] <= lam[0] and lam[-1] <= b["hi"]


def test_pdsa_needs_fp64_context(mot):
    with mot.Context(wl.cube(4, 4.0), precision="fp32_history") as ctx:
        with pytest.raises(mot.MotError, match="FP64"):
            ctx.pdsa_bounds(0)
