"""mot_plane_wave_static (the allocation-free host-output plane wave) against
mot_plane_wave through the C ABI: two calls in a row, each equal to the allocating
entry point; requests beyond its fixed scratch are rejected with a clear error."""
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

SCRATCH_DOUBLES = 2 ** 21


@pytest.fixture(scope="module")
def mot():
    from paper_2407_03323_gb300 import build, mot as m
    if not os.path.exists(m.LIB_PATH):
        build.build()
    m.load_library()
    return m


def test_static_plane_wave_matches_allocating_entry_point(mot):
    N = 24
    eps = wl.sphere(N, 12.0)
    p = wl.pulse(N, 12.0, k_hat=(1.0, 2.0, 2.0), p_hat=(0.0, 1.0, -1.0))
    steps = SCRATCH_DOUBLES // (3 * N ** 3)          # the largest request that fits
    assert steps >= 2
    with mot.Context(eps) as ctx:
        for n_first in (1, 1 + steps):               # two calls in a row
            ref = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"],
                                 n_first, steps)
            got = ctx.plane_wave_static(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"],
                                        p["t0"], n_first, steps)
            assert np.abs(ref).max() > 0
            assert np.array_equal(got, ref)


def test_static_plane_wave_rejects_oversized_request(mot):
    N = 24
    with mot.Context(wl.cube(N, 4.0)) as ctx:
        steps = SCRATCH_DOUBLES // (3 * N ** 3) + 1
        with pytest.raises(mot.MotError) as e:
            ctx.plane_wave_static((0, 0, 1), (1, 0, 0), 0.05, 10.0, 30.0, 1, steps)
        assert "exceeds its fixed device scratch" in str(e.value)
        # the context stays usable
        E = ctx.plane_wave_static((0, 0, 1), (1, 0, 0), 0.05, 10.0, 30.0, 1, 2)
        assert E.shape == (2, N ** 3, 3)
