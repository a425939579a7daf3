"""Several right-hand sides of one scatterer through one context (mot_set_excitation_rhs,
mot_march_rhs): the interleaved march of all of them gives, bitwise, what separate
contexts give for each excitation alone (same kernels, same arguments), with host and
device outputs and across calls; the number of right-hand sides is fixed once marching
has started; the solver settings reach every right-hand side."""
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


def _waves(N, eps, n):
    dirs = wl.random_directions(n, 11)
    return [wl.pulse(N, eps, k_hat=k, p_hat=p) for k, p in dirs]


def _excitations(ctx, waves, n_first, n):
    return np.stack([ctx.plane_wave(w["k_hat"], w["p_hat"], w["f_c"], w["sigma_t"], w["t0"],
                                    n_first, n) for w in waves])


@pytest.mark.parametrize("precision,scheme,block", [("fp32_history", "blocked", 4),
                                                    ("fp64", "direct", 0)])
def test_rhs_march_is_bitwise_the_separate_marches(mot, precision, scheme, block):
    torch = pytest.importorskip("torch")
    N = 10
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    waves = _waves(N, 12.0, 3)
    kw = dict(precision=precision, scheme=scheme, block=block)
    chunks = [35, 25]
    ref = []
    for w in waves:
        with mot.Context(eps, taps, **kw) as c:
            out, done = [], 0
            for k in chunks:
                c.set_excitation(_excitations(c, [w], done + 1, k)[0])
                out.append(c.march(k))
                done += k
            ref.append(np.concatenate(out))
    ref = np.stack(ref)
    with mot.Context(eps, taps, **kw) as c:
        done, host, dev = 0, [], []
        for j, k in enumerate(chunks):
            c.set_excitation_rhs(_excitations(c, waves, done + 1, k))
            if j == 0:
                host.append(c.march_rhs(k))
            else:
                J = torch.empty((3, k, c.M, 3), dtype=torch.float64, device="cuda")
                c.march_rhs(k, out=J)
                host.append(J.cpu().numpy())
            done += k
        got = np.concatenate(host, axis=1)
        for r in range(3):
            assert c.rhs(r).info()["n_done"] == sum(chunks)
    assert np.abs(ref).max() > 0
    assert np.array_equal(got, ref)


def test_rhs_count_is_fixed_once_marching(mot):
    N = 6
    eps = wl.cube(N, 4.0)
    waves = _waves(N, 4.0, 2)
    with mot.Context(eps, precision="fp32_history") as c:
        c.set_excitation_rhs(_excitations(c, waves, 1, 8))
        c.set_solver(tol=1e-9, max_iter=1)      # reaches both right-hand sides
        with pytest.raises(mot.MotError) as ei:
            c.march_rhs(8)
        assert ei.value.status == mot.MOT_ERR_NOT_CONVERGED
        c.set_solver(tol=1e-9, max_iter=200)
        c.set_excitation_rhs(_excitations(c, waves, 9, 8))
        c.march_rhs(8)
        with pytest.raises(mot.MotError) as ei:
            c.set_excitation_rhs(_excitations(c, waves + waves[:1], 17, 8))
        assert ei.value.status == mot.MOT_ERR_ARG
        with pytest.raises(mot.MotError):
            c.rhs(2)


def test_rhs_device_excitation_written_on_the_context_stream(mot):
    """Excitations generated on the device by the context (mot_plane_wave into a CUDA
    buffer, on the context's stream) and staged for all right-hand sides at once: each
    right-hand side's stream waits for the staging, so the march equals the separate
    marches bitwise."""
    torch = pytest.importorskip("torch")
    N = 8
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    waves = _waves(N, 12.0, 4)
    kw = dict(precision="fp32_history", scheme="blocked", block=4)
    n = 40
    ref = []
    for w in waves:
        with mot.Context(eps, taps, **kw) as c:
            c.set_excitation(_excitations(c, [w], 1, n)[0])
            ref.append(c.march(n))
    with mot.Context(eps, taps, **kw) as c:
        E = torch.empty((len(waves), n, c.M, 3), dtype=torch.float64, device="cuda")
        for r, w in enumerate(waves):
            c.plane_wave(w["k_hat"], w["p_hat"], w["f_c"], w["sigma_t"], w["t0"], 1, n, out=E[r])
        c.set_excitation_rhs(E)
        got = c.march_rhs(n)
    assert np.array_equal(got, np.stack(ref))
