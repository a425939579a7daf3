"""Host-side logic that needs no GPU: the memory estimate and bucketing of the batched
driver, the seeded batched workload, the pulse parameters, the diagnostics CLI, and the
bench's algorithmic-byte model of the far levels."""
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


def test_far_level_byte_model_counts_the_live_window():
    """bench.py's algorithmic bytes of the far levels (the roofline's numerator): per
    firing, the past spectra that some output of the level uses (enumerated here over
    every output j < S and lag l in [a, a + S) with l <= ell), the level spectra and
    the S outputs; summed over the firings of one period of the plan."""
    import bench
    from paper_2407_03323_gb300 import mot

    class Ctx:
        pass

    for B, ell, P in ((8, 182, 210), (8, 165, 48), (4, 152, 300), (8, 85, 96), (2, 19, 20)):
        for scheme in ("blocked", "blocked_doubling"):
            plan = mot.level_plan(B, ell, scheme)
            ctx = Ctx()
            ctx.P, ctx.ell = (P, P, P), ell
            ctx.levels = [S for S, _ in plan]
            ctx.level_lags = [a for _, a in plan]
            noct, nbins = (P // 2 + 1) ** 3, P * P * (P // 2 + 1)
            period = max(ctx.levels)
            want, firings = 0, 0
            for S, a in plan:
                n0 = 10 ** 6
                live = {n0 + j - l for j in range(S) for l in range(a, a + S) if l <= ell}
                per = 3 * 8 * nbins * len(live) + (S + 1) * 6 * 8 * noct + S * 3 * 8 * nbins
                want += per * (period // S)
                firings += period // S
            got, launches = bench.far_bytes_per_period(ctx, "fp32_history")
            assert (got, launches) == (want, firings), (B, ell, scheme)
    # 104^3: 242.1 GB per 128 steps (31 firings) with the doubling plan, 124.1 GB per
    # 64 steps (16 firings) with the fitted one
    ctx.P, ctx.ell = (210, 210, 210), 182
    for scheme, gb, n in (("blocked_doubling", 242.098, 31), ("blocked", 124.107, 16)):
        plan = mot.level_plan(8, 182, scheme)
        ctx.levels, ctx.level_lags = [S for S, _ in plan], [a for _, a in plan]
        got, launches = bench.far_bytes_per_period(ctx, "fp32_history")
        assert launches == n and abs(got / 1e9 - gb) < 1e-3, (scheme, got)


def test_binding_refuses_buffers_the_library_would_overrun():
    """The binding's check of a caller's output buffer (the library writes
    n_rhs x n_steps x M x 3 doubles there): dtype, size, contiguity and, for the
    host-only entry point, host memory; no context or device is needed for it."""
    import torch
    from paper_2407_03323_gb300.mot import Context
    c = Context.__new__(Context)
    c.M = 10
    ok = np.zeros((4, 10, 3))
    c._check_out(ok, 4)
    c._check_out(torch.zeros((4, 10, 3), dtype=torch.float64), 4, host_only=True)
    c._check_out(np.zeros((2, 4, 10, 3)), 4, n_rhs=2)
    with pytest.raises(TypeError):
        c._check_out(np.zeros((4, 10, 3), dtype=np.float32), 4)
    with pytest.raises(TypeError):
        c._check_out(torch.zeros((4, 10, 3), dtype=torch.float32), 4)
    with pytest.raises(TypeError):
        c._check_out([0.0] * 120, 4)
    with pytest.raises(ValueError):
        c._check_out(np.zeros((3, 10, 3)), 4)                  # one step short
    with pytest.raises(ValueError):
        c._check_out(np.zeros((4, 10, 3)), 4, n_rhs=2)          # one right-hand side short
    with pytest.raises(ValueError):
        c._check_out(np.zeros((4, 10, 6))[:, :, ::2], 4)        # strided view
    with pytest.raises(ValueError):
        c._check_out(torch.zeros((4, 3, 10), dtype=torch.float64).transpose(1, 2), 4)

    class Device:
        dtype = "torch.float64"
        device = "cuda:0"

        def data_ptr(self):
            return 0

    with pytest.raises(TypeError):
        c._check_out(Device(), 4, host_only=True)               # device memory, host-only call
