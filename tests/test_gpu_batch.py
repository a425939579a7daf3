"""Batched uneven scatterers x excitations (paper_2407_03323_gb300.batch): every march
of the batch ends where the same march run alone ends (bitwise), with the excitations
as separate contexts or as right-hand sides of one context per scatterer, and the
block-size tuner returns one of its candidates."""
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


@pytest.mark.parametrize("rhs", [False, True])
def test_batch_matches_individual_marches(mot, rhs):
    pytest.importorskip("torch")
    from paper_2407_03323_gb300.batch import BlockTuner, run_batched
    inst = wl.batched_instances(n_instances=3, n_rhs=2, seed=7, side_range=(8, 12))
    tuner = BlockTuner("fp32_history", candidates=(4, 8), buckets=(12,))
    res = run_batched(inst, 96, tuner=tuner, chunk=32, workers=8, rhs=rhs)
    assert set(res["blocks"]) <= {4, 8}
    for i, x in enumerate(inst):
        for j, w in enumerate(x["waves"]):
            with mot.Context(x["eps_r"], x["taps"], precision="fp32_history", scheme="blocked",
                             block=res["blocks"][i]) as c:
                for n0 in range(0, 96, 32):
                    E = c.plane_wave(w["k_hat"], w["p_hat"], w["f_c"], w["sigma_t"], w["t0"],
                                     n0 + 1, 32)
                    c.set_excitation(E)
                    c.march(32, out=None)
                assert c.info()["last_norm"] == res["last_norms"][(i, j)], (i, j)
    assert res["value"] > 0
