"""Degenerate grids through the C ABI: grids one voxel thick along some axes (no
neighbours there, padded lengths 2), a single voxel (Z_0 a multiple of the identity:
the Chebyshev interval collapses to one point), and a grid without dielectric (chi = 0
everywhere: J stays exactly zero, no solve runs)."""
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


@pytest.mark.parametrize("shape", [(1, 1, 5), (3, 1, 4), (1, 1, 1)])
def test_thin_grids_match_oracle(mot, shape):
    from oracle import excitation, kernel_table, march
    from oracle.spline import num_lags
    W, V, U = shape
    rng = np.random.default_rng(sum(shape))
    eps = 2.0 + 8.0 * rng.uniform(size=shape)
    taps = wl.fir_taps("fir3", 0.01)
    ell = num_lags(U, V, W)
    G, _, _ = kernel_table.octant_table(max(shape), ell + 1)
    p = wl.pulse(max(shape), 6.0, k_hat=(0.6, 0.0, 0.8), p_hat=(0.0, 1.0, 0.0))
    steps = 48
    E = excitation.tested_excitation(eps, p, steps)
    ref = march.march(G, eps, taps, E)
    with mot.Context(eps, taps) as ctx:
        assert ctx.ell == ell
        ctx.set_excitation(E)
        J = ctx.march(steps)
    assert np.linalg.norm(J - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision,scheme", [("fp64", "direct"), ("fp32_history", "blocked")])
def test_grid_without_dielectric(mot, precision, scheme):
    eps = np.ones((4, 5, 6))
    p = wl.pulse(6, 4.0)
    with mot.Context(eps, wl.fir_taps("fir3", 0.01), precision=precision, scheme=scheme,
                     block=4) as ctx:
        E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 30, 1, 40)
        assert np.all(E == 0.0)                 # E = chi e with chi = 0
        ctx.set_excitation(E)
        J = ctx.march(40)
    assert np.all(J == 0.0)
