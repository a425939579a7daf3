"""Whole periods of the march as CUDA graphs (mot_set_graph): the graph march gives the
same J, bitwise, as the step-by-step march (the same kernels with the same arguments),
in both precisions and both history schemes, including steps before the first whole
period and after the last; the executable graph is instantiated once and updated in
place for every later period; host outputs fall back to step-by-step launches."""
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


def _march(mot, eps, taps, wave, steps, graph, chunks, out_device=True, **kw):
    torch = pytest.importorskip("torch")
    with mot.Context(eps, taps, **kw) as c:
        if graph:
            c.set_graph(graph)
        c.set_profiling(False)
        out, done = [], 0
        for k in chunks:
            E = c.plane_wave(wave["k_hat"], wave["p_hat"], wave["f_c"], wave["sigma_t"],
                             wave["t0"], done + 1, k)
            c.set_excitation(E)
            if out_device:
                J = torch.empty((k, c.M, 3), dtype=torch.float64, device="cuda")
                c.march(k, out=J)
                out.append(J.cpu().numpy())
            else:
                out.append(c.march(k))
            done += k
        return np.concatenate(out), c.stats(), c.info()


@pytest.mark.parametrize("precision,scheme,block", [("fp32_history", "blocked", 4),
                                                    ("fp64", "blocked", 4),
                                                    ("fp32_history", "direct", 0)])
def test_graph_march_is_bitwise_the_step_march(mot, precision, scheme, block):
    N = 10
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("fir3", 1e-7 * N ** 3)
    w = wl.pulse(N, 12.0)
    kw = dict(precision=precision, scheme=scheme, block=block)
    with mot.Context(eps, taps, **kw) as c:
        Q = 2 * c.period if c.levels else 16
    chunks = [3 * Q + 5, 2 * Q + 7]          # whole periods, a ragged tail, a new call
    steps = sum(chunks)
    ref, st0, _ = _march(mot, eps, taps, w, steps, 0, chunks, **kw)
    got, st1, info = _march(mot, eps, taps, w, steps, Q, chunks, **kw)
    assert st0["graph_launches"] == 0
    assert st1["graph_launches"] >= 3 and st1["graph_instantiations"] == 1
    assert st1["launches"] == st0["launches"]
    assert np.abs(ref).max() > 0
    assert np.array_equal(got, ref)
    assert info["n_done"] == steps


def test_graph_with_host_outputs_marches_step_by_step(mot):
    N = 8
    eps = wl.cube(N, 4.0)
    w = wl.pulse(N, 4.0)
    kw = dict(precision="fp32_history", scheme="blocked", block=4)
    ref, _, _ = _march(mot, eps, None, w, 40, 0, [40], out_device=False, **kw)
    with mot.Context(eps, None, **kw) as c:
        Q = c.period
    got, st, _ = _march(mot, eps, None, w, 40, Q, [40], out_device=False, **kw)
    assert st["graph_launches"] == 0
    assert np.array_equal(got, ref)


def test_set_graph_rejects_periods_that_are_not_whole_level_periods(mot):
    with mot.Context(wl.cube(8, 4.0), precision="fp32_history", scheme="blocked", block=4) as c:
        S = c.period
        with pytest.raises(mot.MotError) as ei:
            c.set_graph(S + 1)
        assert ei.value.status == mot.MOT_ERR_ARG
        with pytest.raises(mot.MotError):
            c.set_graph(-1)
        c.set_graph(2 * S)
        c.set_graph(0)
