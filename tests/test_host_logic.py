"""Host-side logic that needs no GPU: the memory estimate and bucketing of the batched
driver, the seeded batched workload, the pulse parameters, and the diagnostics CLI."""
import math

import numpy as np
import pytest

import workloads as wl


def _pad(N):
    P = max(2 * N - 1, 2)
    while True:
        n = P
        for r in (2, 3, 5, 7):
            while n % r == 0:
                n //= r
        if n == 1 and P % 2 == 0:
            return P
        P += 1


def test_state_bytes_follows_the_padded_grid():
    """The per-march memory estimate uses the library's padding (smallest even 7-smooth
    P >= 2N - 1) and grows with N; FP64 rings cost twice the FP32 ones."""
    from paper_2407_03323_gb300.batch import _state_bytes
    assert [_pad(N) for N in (8, 32, 48, 104)] == [16, 64, 96, 210]
    prev = 0
    for N in (16, 24, 32, 40, 48):
        b32 = _state_bytes(N, "fp32_history", 8)
        b64 = _state_bytes(N, "fp64", 8)
        P = _pad(N)
        slot32 = 3 * P * P * (P // 2 + 1) * 8
        assert b32 % slot32 == (200 * N ** 3) % slot32
        assert b64 - 200 * N ** 3 == 2 * (b32 - 200 * N ** 3)
        assert b32 > prev
        prev = b32


def test_block_tuner_buckets():
    from paper_2407_03323_gb300.batch import BlockTuner
    t = BlockTuner()
    assert [t.bucket(N) for N in (16, 24, 25, 33, 48, 60)] == [24, 24, 32, 40, 48, 60]


def test_batched_instances_are_seeded_and_in_range():
    a = wl.batched_instances(n_instances=5, n_rhs=3, seed=11)
    b = wl.batched_instances(n_instances=5, n_rhs=3, seed=11)
    for x, y in zip(a, b):
        assert x["N"] == y["N"] and x["shape"] == y["shape"] and x["eps"] == y["eps"]
        assert np.array_equal(x["eps_r"], y["eps_r"])
        assert 16 <= x["N"] <= 48 and 2.0 <= x["eps"] <= 30.0
        assert x["eps_r"].shape == (x["N"],) * 3 and len(x["waves"]) == 3
        for w in x["waves"]:
            assert abs(np.linalg.norm(w["k_hat"]) - 1) < 1e-12
            assert abs(np.dot(w["k_hat"], w["p_hat"])) < 1e-12


def test_pulse_parameters():
    """f_c dt = 1/(10 sqrt(eps)) (10 voxels per wavelength inside), amplitude-spectrum
    FWHM 0.5 f_c, so sigma_t = 2 sqrt(2 ln 2) / (pi f_c)."""
    p = wl.pulse(32, 12.0)
    fc = 1.0 / (10.0 * math.sqrt(12.0))
    assert abs(p["f_c"] - fc) < 1e-15
    assert abs(p["sigma_t"] - 2.0 * math.sqrt(2.0 * math.log(2.0)) / (math.pi * fc)) < 1e-9


def test_diagnostics_cli_help():
    from paper_2407_03323_gb300 import diagnostics
    with pytest.raises(SystemExit) as e:
        diagnostics.main(["--help"])
    assert e.value.code == 0
