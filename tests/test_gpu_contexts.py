"""Several live contexts: different grids and FIR taps marched interleaved give each
one's own result (no state shared between contexts but read-only setup), and
contexts created with mot_create_shared march like independently created ones."""
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


def _run(ctx, pulse, n_first, n):
    E = ctx.plane_wave(pulse["k_hat"], pulse["p_hat"], pulse["f_c"], pulse["sigma_t"],
                       pulse["t0"] - 40.0, n_first, n)
    ctx.set_excitation(E)
    return ctx.march(n)


def test_interleaved_contexts_with_different_grids_and_taps(mot):
    cases = [(wl.sphere(9, 12.0), wl.fir_taps("fir3", 0.02), "fp64", "direct"),
             (wl.cube(6, 4.0), wl.fir_taps("hp9", 0.01), "fp32_history", "blocked"),
             (np.full((4, 7, 11), 6.0), wl.fir_taps("fir2", 0.05), "fp64", "blocked")]
    pulses = [wl.pulse(e.shape[0], 6.0) for e, _, _, _ in cases]
    alone = []
    for (eps, taps, prec, sch), p in zip(cases, pulses):
        with mot.Context(eps, taps, precision=prec, scheme=sch, block=4) as c:
            alone.append(np.concatenate([_run(c, p, 1, 30), _run(c, p, 31, 30)]))
    ctxs = [mot.Context(eps, taps, precision=prec, scheme=sch, block=4)
            for eps, taps, prec, sch in cases]
    try:
        parts = [[] for _ in ctxs]
        for k in range(2):
            for i, (c, p) in enumerate(zip(ctxs, pulses)):
                parts[i].append(_run(c, p, 1 + 30 * k, 30))
        for i in range(len(ctxs)):
            assert np.array_equal(np.concatenate(parts[i]), alone[i]), i
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("precision,scheme", [("fp64", "blocked"), ("fp32_history", "blocked"),
                                              ("fp64", "direct")])
def test_shared_contexts_march_like_fresh_ones(mot, precision, scheme):
    """Three excitations of one scatterer: the source and two shared contexts, marched
    interleaved, against three separately created contexts."""
    N = 10
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    dirs = wl.random_directions(3, 11)
    pulses = [wl.pulse(N, 12.0, k_hat=k, p_hat=p) for k, p in dirs]
    ref = []
    for p in pulses:
        with mot.Context(eps, taps, precision=precision, scheme=scheme, block=4) as c:
            ref.append(_run(c, p, 1, 80))
    src = mot.Context(eps, taps, precision=precision, scheme=scheme, block=4)
    ctxs = [src, src.share(), src.share()]
    try:
        with pytest.raises(RuntimeError):
            src.close()                       # shared contexts still use its setup
        out = [[] for _ in ctxs]
        for k in range(4):
            for i, (c, p) in enumerate(zip(ctxs, pulses)):
                out[i].append(_run(c, p, 1 + 20 * k, 20))
        for i in range(3):
            assert np.array_equal(np.concatenate(out[i]), ref[i]), i
    finally:
        for c in ctxs[1:]:
            c.close()
        src.close()
