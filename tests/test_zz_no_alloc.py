"""mot_plane_wave_static (the allocation-free host-output plane wave) against
mot_plane_wave through the C ABI: two calls in a row, each equal to the allocating
entry point; requests beyond its fixed scratch are rejected with a clear error; the
calls take no device memory (free memory unchanged across calls, and the entry point
still works when the caller has taken all but a few MiB of the device's memory, where
the allocating entry point reports MOT_ERR_OOM)."""
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


def _fill_device(torch, leave):
    """Take device memory in tensors until less than `leave` bytes are free (pieces of
    at most `cap` bytes, halved whenever one does not fit); returns the tensors."""
    hold = []
    step = 2 << 20
    cap = None
    for _ in range(10000):
        free = torch.cuda.mem_get_info()[0]
        if free < leave:
            break
        want = max(step, ((free - leave // 2) // step) * step)
        if cap is not None:
            want = min(want, cap)
        try:
            hold.append(torch.empty(want, dtype=torch.uint8, device="cuda"))
        except RuntimeError:
            if want <= step:
                break
            cap = max(step, (want // 2 // step) * step)
    return hold


def test_static_plane_wave_takes_no_device_memory(mot):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = 24
    eps = wl.sphere(N, 12.0)
    p = wl.pulse(N, 12.0, k_hat=(1.0, 2.0, 2.0), p_hat=(0.0, 1.0, -1.0))
    steps = SCRATCH_DOUBLES // (3 * N ** 3)
    need = 8 * 3 * N ** 3 * steps                # bytes the allocating entry point stages
    wave = (p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"])
    with mot.Context(eps) as ctx:
        ref = ctx.plane_wave(*wave, 1, steps)
        ctx.plane_wave_static(*wave, 1, steps)   # first call: scratch address, kernels loaded
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for n_first in (1 + steps, 1, 1 + steps):
            ctx.plane_wave_static(*wave, n_first, steps)
            assert torch.cuda.mem_get_info()[0] == free0
        hold = _fill_device(torch, need)
        try:
            assert torch.cuda.mem_get_info()[0] < need
            got = ctx.plane_wave_static(*wave, 1, steps)
            assert np.array_equal(got, ref)
            with pytest.raises(mot.MotError) as e:
                ctx.plane_wave(*wave, 1, steps)
            assert e.value.status == mot.MOT_ERR_OOM
        finally:
            del hold
            torch.cuda.empty_cache()
        # both entry points work again once the memory is back
        assert np.array_equal(ctx.plane_wave(*wave, 1, steps), ref)
        assert np.array_equal(ctx.plane_wave_static(*wave, 1, steps), ref)
