"""Failure detection of the march, made on the host side: an iteration cap the solver
cannot meet, a growth limit the pulse must exceed, invalid arguments.  Nothing here
faults, traps or hangs a GPU; every case returns a status the caller reads."""
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


def _pulse_ctx(mot, N=6, **kw):
    eps = wl.cube(N, 5.0)
    p = wl.pulse(N, 5.0)
    ctx = mot.Context(eps, **kw)
    E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 60, 1, 48)
    ctx.set_excitation(E)
    return ctx


def test_not_converged_status_and_recovery(mot):
    """An iteration cap below what the solve needs gives MOT_ERR_NOT_CONVERGED with the
    step recorded; the context stays usable and converges again with the cap lifted."""
    ctx = _pulse_ctx(mot)
    ctx.set_solver(tol=1e-13, max_iter=1)
    with pytest.raises(mot.MotError) as ei:
        ctx.march(8)
    assert ei.value.status == mot.MOT_ERR_NOT_CONVERGED
    info = ctx.info()
    assert 1 <= info["fail_step"] <= 8
    ctx.set_solver(tol=1e-13, max_iter=200)
    ctx.march(8)
    assert ctx.info()["n_done"] == 16
    ctx.close()


def test_unstable_status_on_growth(mot):
    """A growth limit just above 1 trips on the rising edge of the pulse: the monitor
    reports MOT_ERR_UNSTABLE and the step where it happened."""
    ctx = _pulse_ctx(mot)
    ctx.set_solver(tol=1e-13, max_iter=200, growth_limit=1.0001)
    with pytest.raises(mot.MotError) as ei:
        ctx.march(48)
    assert ei.value.status == mot.MOT_ERR_UNSTABLE
    assert ctx.info()["fail_step"] > 0
    ctx.close()


def test_bad_arguments(mot):
    with pytest.raises(mot.MotError) as ei:
        mot.Context(wl.cube(4, 0.5))
    assert ei.value.status == mot.MOT_ERR_ARG
    with pytest.raises(mot.MotError) as ei:
        mot.Context(wl.cube(4, 3.0), scheme="blocked", block=3)
    assert ei.value.status == mot.MOT_ERR_ARG
    with mot.Context(wl.cube(4, 3.0)) as ctx:
        with pytest.raises(mot.MotError) as ei:
            ctx.march(0)
        assert ei.value.status == mot.MOT_ERR_ARG
        # buffers the library would read or write past their end are refused in Python
        with pytest.raises(ValueError):
            ctx.march(4, out=np.zeros((3, 64, 3)))
        with pytest.raises(TypeError):
            ctx.set_excitation(np.zeros((4, 64, 3), dtype=np.float32))
        with pytest.raises(ValueError):
            ctx.set_excitation(np.zeros((4, 64, 3))[:, ::2])
        with pytest.raises(ValueError):
            ctx.set_excitation_rhs(np.zeros((2, 4, 60, 3)))
        with pytest.raises(mot.MotError) as ei:
            ctx.eval_history(np.zeros((ctx.ell + 1, 64, 3)))
        assert ei.value.status == mot.MOT_ERR_ARG


def test_vacuum_voxels_stay_zero(mot):
    """Voxels with eps_r = 1 (chi = 0) carry no current (reading R5)."""
    N = 8
    eps = wl.sphere(N, 12.0)
    p = wl.pulse(N, 12.0)
    with mot.Context(eps) as ctx:
        E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 80, 1, 64)
        ctx.set_excitation(E)
        J = ctx.march(64)
    out = eps.reshape(-1) == 1.0
    assert np.abs(J[:, ~out]).max() > 0
    assert np.abs(J[:, out]).max() == 0.0


@pytest.mark.parametrize("precision,factors,tol", [("fp64", (1e-60, 1e60), 1e-12),
                                                    ("fp32_history", (1e-20, 1e20), 1e-6)])
def test_tiny_and_huge_excitations_scale_linearly(mot, precision, factors, tol):
    """The march is linear: an excitation scaled by f gives the current scaled by f.
    The solver normalises residuals in FP64 before its FP32 inner iterations, so tiny
    or huge right-hand sides neither underflow nor overflow there.  The FP32-history
    variant stores the spectra of J in FP32, so its range is that of FP32 (|J| within
    about 1e-30 .. 1e30); FP64 is exercised at 1e+-60."""
    N = 6
    eps = wl.cube(N, 4.0)
    p = wl.pulse(N, 4.0)
    res = {}
    for f in (1.0,) + tuple(factors):
        with mot.Context(eps, precision=precision, scheme="blocked", block=4) as ctx:
            E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 40, 1, 40)
            ctx.set_excitation(E * f)
            res[f] = ctx.march(40)
    for f in factors:
        assert np.isfinite(res[f]).all()
        assert np.linalg.norm(res[f] / f - res[1.0]) < tol * np.linalg.norm(res[1.0])


@pytest.mark.parametrize("precision", ["fp64", "fp32_history"])
def test_nan_in_excitation_is_unstable_at_its_step(mot, precision):
    """A NaN placed by the host in E_k (one component of one voxel): the solve of step k
    stops on the non-finite residual instead of iterating, returns J_k as NaN, and the
    monitor reports MOT_ERR_UNSTABLE with fail_step = k; the steps before k are finite."""
    k = 17
    eps = wl.cube(6, 5.0)
    p = wl.pulse(6, 5.0)
    with mot.Context(eps, precision=precision) as ctx:
        E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 60, 1, 32)
        E[k - 1, 100, 1] = np.nan
        ctx.set_excitation(E)
        J = np.zeros((32, ctx.M, 3))
        with pytest.raises(mot.MotError) as ei:
            ctx.march(32, out=J)
        assert ei.value.status == mot.MOT_ERR_UNSTABLE
        info = ctx.info()
        assert info["fail_step"] == k
        assert info["n_done"] == 32
        assert np.isfinite(J[:k - 1]).all()
        assert not np.isfinite(J[k - 1]).all()


def test_grid_too_large_for_the_device_is_oom(mot):
    """A 1024 x 1024 x 1 grid (ell = 1450, padded 2048 x 2048 x 2) needs a 292 GB FP64
    spectral ring, more than the device holds: mot_create returns MOT_ERR_OOM, frees
    what it had allocated, and the next context works."""
    eps = np.full((1, 1024, 1024), 2.0)
    with pytest.raises(mot.MotError) as ei:
        mot.Context(eps)
    assert ei.value.status == mot.MOT_ERR_OOM
    with mot.Context(wl.cube(4, 3.0)) as ctx:
        ctx.march(4)
        assert ctx.info()["n_done"] == 4


def test_grid_barrier_passes_every_round(mot):
    """The bounded grid barrier of the solve kernel, every block present: 2000 rounds
    pass with no timeout."""
    st, passed, rnd = mot.barrier_check(96, 2000)
    assert st == mot.MOT_OK and passed == 96 and rnd == 0


def test_grid_barrier_wait_runs_out(mot):
    """A block that never arrives (a barrier that nothing completes): the others' wait
    runs out after its 0.2 s budget, the launch ends with MOT_ERR_TIMEOUT at round 1,
    and the device stays usable (a march right after is correct)."""
    import time
    t0 = time.perf_counter()
    st, passed, rnd = mot.barrier_check(96, 50, absent=7, budget_s=0.2)
    dt = time.perf_counter() - t0
    assert st == mot.MOT_ERR_TIMEOUT and passed == 0 and rnd == 1
    assert dt < 10.0
    ctx = _pulse_ctx(mot)
    ctx.march(16)
    assert ctx.info()["n_done"] == 16 and np.isfinite(ctx.info()["last_norm"])
    ctx.close()
