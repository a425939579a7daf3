"""Zero-padded FFT lengths chosen by the caller (mot_create_padded): any length >= 2N - 1
per axis gives the same linear convolution of the history (App. A), so the march with
a longer or differently factored length equals the default one to rounding: FP64 to
1e-12 relative L2 (direct and blocked), FP32-history through a four-step codelet length
to 1e-5."""
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


def _march(mot, eps, taps, w, steps, **kw):
    with mot.Context(eps, taps, **kw) as c:
        E = c.plane_wave(w["k_hat"], w["p_hat"], w["f_c"], w["sigma_t"], w["t0"], 1, steps)
        c.set_excitation(E)
        return c.march(steps), c.P


@pytest.mark.parametrize("scheme,block", [("direct", 0), ("blocked", 4)])
def test_longer_fft_lengths_give_the_same_fp64_march(mot, scheme, block):
    N = 8
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    w = wl.pulse(N, 12.0)
    ref, P0 = _march(mot, eps, taps, w, 96, precision="fp64", scheme=scheme, block=block)
    got, P1 = _march(mot, eps, taps, w, 96, precision="fp64", scheme=scheme, block=block,
                     fft_len=(24, 20, 30))
    assert tuple(P0) == (16, 16, 16) and tuple(P1) == (24, 20, 30)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_codelet_length_fp32_history(mot):
    N = 24
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    w = wl.pulse(N, 12.0)
    kw = dict(scheme="blocked", block=8)
    ref, _ = _march(mot, eps, taps, w, 160, precision="fp64", **kw)
    got, P = _march(mot, eps, taps, w, 160, precision="fp32_history", fft_len=(64, 64, 64), **kw)
    assert tuple(P) == (64, 64, 64)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
