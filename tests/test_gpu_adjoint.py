"""Adjoint march (mot_adjoint) against the oracle's dense transposed march, the duality
<g, J> = <lambda, E>, and central finite differences of the forward march."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _hetero(N, seed):
    rng = np.random.default_rng(seed)
    eps = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    eps[0, 0, :2] = 1.0                      # two vacuum voxels (gradient defined as 0)
    return eps


def test_adjoint_matches_oracle(mot):
    from oracle import adjoint, excitation, kernel_table, march
    from oracle.spline import num_lags
    N, steps = 4, 60
    eps = _hetero(N, 21)
    taps = wl.fir_taps("fir3", 0.05)
    p = wl.pulse(N, 6.0, k_hat=(0.0, 1.0, 1.0), p_hat=(1.0, 0.0, 0.0))
    G, _, _ = kernel_table.octant_table(N, num_lags(N, N, N) + 1)
    E = excitation.tested_excitation(eps, p, steps)
    e_inc = excitation.tested_excitation(eps, p, steps, with_chi=False)
    Jref = march.march(G, eps, taps, E)
    g = np.random.default_rng(3).normal(size=Jref.shape)
    lam_ref = adjoint.adjoint(G, eps, taps, g)
    grad_ref = adjoint.gradient_eps(G, eps, taps, e_inc, Jref, lam_ref)
    with mot.Context(eps, taps) as ctx:
        ctx.set_excitation(E)
        J = ctx.march(steps)
        grad, lam = ctx.adjoint(J, g, want_lambda=True)
    assert rel_l2(J, Jref) < 1e-10
    assert rel_l2(lam, lam_ref) < 1e-10
    act = eps.reshape(-1) > 1.0
    gf = grad.reshape(-1)
    assert np.abs(gf[act] - grad_ref[act]).max() < 1e-9 * np.abs(grad_ref[act]).max()
    assert np.all(gf[~act] == 0.0)


@pytest.mark.parametrize("scheme,precision,tol", [("direct", "fp64", 1e-10),
                                                  ("blocked", "fp64", 1e-10),
                                                  ("blocked", "fp32_history", 1e-5)])
def test_adjoint_duality_16(mot, scheme, precision, tol):
    """<g, J> = <lambda, E> (Z J = E, Z^T lambda = g) on a 16^3 heterogeneous block."""
    N, steps = 16, 120
    eps = _hetero(N, 5)
    taps = wl.fir_taps("hp9", 1e-7 * N ** 3)
    p = wl.pulse(N, 6.0)
    g = np.random.default_rng(9).normal(size=(steps, N ** 3, 3))
    with mot.Context(eps, taps, precision=precision, scheme=scheme, block=4) as ctx:
        E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 60, 1, steps)
        ctx.set_excitation(E)
        J = ctx.march(steps)
        _, lam = ctx.adjoint(J, g, want_lambda=True)
    lhs, rhs = np.sum(g * J), np.sum(lam * E)
    assert abs(lhs - rhs) < tol * abs(lhs)


def test_adjoint_gradient_matches_finite_differences(mot):
    """O = sum_n <w_n, J_n>: dO/deps_m by the adjoint against central differences of two
    GPU forward marches (FP64, 10^3 heterogeneous block, 9-tap FIR)."""
    N, steps = 10, 100
    eps = _hetero(N, 8)
    taps = wl.fir_taps("hp9", 1e-7 * N ** 3)
    p = wl.pulse(N, 6.0)
    w = np.random.default_rng(1).normal(size=(steps, N ** 3, 3))

    def objective(e):
        with mot.Context(e, taps) as ctx:
            E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 50, 1,
                               steps)
            ctx.set_excitation(E)
            J = ctx.march(steps)
            return float(np.sum(w * J)), J

    O0, J = objective(eps)
    with mot.Context(eps, taps) as ctx:
        grad = ctx.adjoint(J, w).reshape(-1)
    # Each forward march meets the solver tolerance, not the exact solution, so the
    # difference quotient carries an absolute error of about |O| x (solve error) / h,
    # the same at every voxel: the bound's floor is a fraction of the largest gradient.
    h = 1e-4
    rng = np.random.default_rng(2)
    act = np.nonzero(eps.reshape(-1) > 1.0)[0]
    for m in rng.choice(act, 6, replace=False):
        ep = eps.copy().reshape(-1)
        em = eps.copy().reshape(-1)
        ep[m] += h
        em[m] -= h
        fd = (objective(ep.reshape(eps.shape))[0] - objective(em.reshape(eps.shape))[0]) / (2 * h)
        assert abs(fd - grad[m]) < 1e-6 * max(abs(fd), 1e-2 * np.abs(grad).max()), (m, fd, grad[m])
