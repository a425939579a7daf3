"""Restart from a saved history (mot_restart), the segmented adjoint
(mot_adjoint_begin/run/end) and the torch.autograd.Function over the march, with and
without checkpoint/recompute, against central differences of the forward march."""
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


def _hetero(N, seed):
    rng = np.random.default_rng(seed)
    eps = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    eps[0, 0, :2] = 1.0
    return eps


def _wave(N, shift):
    p = wl.pulse(N, 6.0)
    return {"k_hat": p["k_hat"], "p_hat": p["p_hat"], "f_c": p["f_c"], "sigma_t": p["sigma_t"],
            "t0": p["t0"] - shift}


def _march(ctx, w, n_first, n):
    E = ctx.plane_wave(w["k_hat"], w["p_hat"], w["f_c"], w["sigma_t"], w["t0"], n_first, n)
    ctx.set_excitation(E)
    return ctx.march(n)


@pytest.mark.parametrize("precision,scheme,tol", [("fp64", "blocked", 1e-12),
                                                  ("fp64", "direct", 1e-12),
                                                  ("fp32_history", "blocked", 1e-6)])
def test_restart_continues_the_march(mot, precision, scheme, tol):
    """March 70 + 60 steps straight, and 70 then a restart of a fresh context from the
    last ell currents (far levels S = 4..16 fire across the restart point)."""
    N = 10
    eps = _hetero(N, 3)
    taps = wl.fir_taps("fir3", 1e-3)
    w = _wave(N, 50.0)
    with mot.Context(eps, taps, precision=precision, scheme=scheme, block=4) as a:
        ref = np.concatenate([_march(a, w, 1, 70), _march(a, w, 71, 60)])
        ell = a.ell
    with mot.Context(eps, taps, precision=precision, scheme=scheme, block=4) as b:
        b.restart(70, ref[70 - ell:70])
        cont = _march(b, w, 71, 60)
    err = np.linalg.norm(cont - ref[70:]) / np.linalg.norm(ref[70:])
    assert err < tol


def test_segmented_adjoint_equals_one_shot(mot):
    """mot_adjoint against begin / run over three uneven segments (windows that hold
    only each segment and the L - 1 steps before it) / end."""
    N, steps = 8, 90
    eps = _hetero(N, 4)
    taps = wl.fir_taps("fir3", 0.01)
    w = _wave(N, 40.0)
    g = np.random.default_rng(6).normal(size=(steps, N ** 3, 3))
    with mot.Context(eps, taps) as ctx:
        J = _march(ctx, w, 1, steps)
        ref = ctx.adjoint(J, g)
        L = max(len(taps), 2)
        ctx.adjoint_begin(steps)
        hi = steps
        for cnt in (17, 40, 33):
            lo = hi - cnt + 1
            first = max(1, lo - L + 1)
            ctx.adjoint_run(cnt, J[first - 1:hi], first, g[lo - 1:hi])
            hi = lo - 1
        grad = ctx.adjoint_end()
    assert np.abs(grad - ref).max() <= 1e-13 * np.abs(ref).max()


def test_autograd_gradient_checkpointed_and_fd(mot):
    """O = time-gated energy of J at 48 probe voxels; d O / d eps_r through the
    autograd Function, all currents kept and checkpointed every 24 steps (recomputed
    from mot_restart), against each other and against central differences."""
    torch = pytest.importorskip("torch")
    from paper_2407_03323_gb300.autograd import march
    N, steps = 10, 100
    eps0 = _hetero(N, 8)
    taps = wl.fir_taps("fir3", 1e-3)
    w = _wave(N, 50.0)
    probes = np.random.default_rng(5).choice(N ** 3, 48, replace=False)
    gate = slice(40, steps)

    def objective(J):
        return (J[gate] ** 2).sum()

    grads = {}
    for K in (None, 24):
        eps = torch.tensor(eps0, dtype=torch.float64, requires_grad=True)
        O = objective(march(eps, taps, w, steps, probes=probes, checkpoint_every=K))
        O.backward()
        grads[K] = eps.grad.numpy().reshape(-1)
    gmax = np.abs(grads[None]).max()
    assert np.abs(grads[24] - grads[None]).max() < 1e-9 * gmax

    def value(e):
        with torch.no_grad():
            return float(objective(march(torch.tensor(e), taps, w, steps, probes=probes)))

    h = 1e-4
    act = np.nonzero(eps0.reshape(-1) > 1.0)[0]
    for m in np.random.default_rng(2).choice(act, 4, replace=False):
        ep = eps0.copy().reshape(-1)
        em = eps0.copy().reshape(-1)
        ep[m] += h
        em[m] -= h
        fd = (value(ep.reshape(eps0.shape)) - value(em.reshape(eps0.shape))) / (2 * h)
        assert abs(fd - grads[None][m]) < 1e-6 * max(abs(fd), 1e-2 * gmax), (m, fd, grads[None][m])
    assert np.all(grads[None][eps0.reshape(-1) == 1.0] == 0.0)
