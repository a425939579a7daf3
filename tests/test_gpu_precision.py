"""FP32-history against the FP64 march on the sphere workloads (relative L2 over all
J_n, the march's own variables), and late-time stability of a 10x-extended
FP32-history march: ||J_n|| must not grow after the pulse has passed (Secs. 5-6: the
FIR-regularised scheme is stable; the FP32 history must not undo that).

Bounds: the target, 1e-5, on both spheres.  What sets the deviation is not the
random rounding of FP32 arithmetic and storage (rounding the J spectra and the history
spectrum to FP32 in an otherwise FP64 march moves it by 2e-7 over 2048 steps at 32^3)
but systematic changes of the operator, which shift the resonances of these high-Q
eps_r = 12 spheres so that the error grows with time: FP32-rounded FFT twiddles alone
(in an FP64 march) gave 2.9e-5, the FP32 kernel spectra 3e-6.  The FP32 transforms
therefore apply their DFT constants and the spatial twiddles as float pairs hi + lo
(the far levels' four-step twiddles hardly matter and stay plain), and the deviation
is 6.3e-6 on the 32^3 sphere over 2048 steps and 7.1e-6 at 104^3 over 640 steps."""
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


def _context(mot, cfg, precision, block=8):
    return mot.Context(cfg["eps_r"], cfg["taps"], precision=precision, scheme="blocked",
                       block=block)


def _march_pulse(ctx, cfg, n_first, n_steps, shift=0.0):
    """Stage the tested plane wave for steps n_first .. n_first + n_steps - 1, march."""
    p = cfg["pulse"]
    E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - shift, n_first,
                       n_steps)
    ctx.set_excitation(E)
    return ctx.march(n_steps)


def test_sphere32_fp32_vs_fp64_and_10x_stability(mot):
    """32^3 sphere, FIR3 (delta = 1e-7 M): 2048 steps in both precisions, then the FP32-history march
    continued to 20,480 steps (10x) with E = 0 after the pulse."""
    cfg = wl.config("sphere32")
    steps, chunk, total = 2048, 256, 20480
    with _context(mot, cfg, "fp64") as c64, _context(mot, cfg, "fp32_history") as c32:
        num = den = 0.0
        norms = []
        for k in range(steps // chunk):
            a = _march_pulse(c64, cfg, 1 + k * chunk, chunk)
            b = _march_pulse(c32, cfg, 1 + k * chunk, chunk)
            num += float(np.sum((b - a) ** 2))
            den += float(np.sum(a ** 2))
            norms.extend(np.sqrt(np.sum(b.reshape(chunk, -1) ** 2, axis=1)))
        rel = np.sqrt(num / den)
        for _ in range((total - steps) // chunk):
            b = c32.march(chunk)
            norms.extend(np.sqrt(np.sum(b.reshape(chunk, -1) ** 2, axis=1)))
    norms = np.array(norms)
    peak = norms[:steps].max()
    last = norms[-2048:].max()
    prev = norms[-4096:-2048].max()
    print("\nsphere32: FP32-history vs FP64 rel L2 over %d steps = %.3e; ||J|| peak %.3e, "
          "max over steps %d..%d = %.3e (previous 2048: %.3e)"
          % (steps, rel, peak, total - 2047, total, last, prev))
    assert np.all(np.isfinite(norms))
    assert rel < 1e-5                  # the FP32-history target
    windows = [norms[i:i + 2048].max() for i in range(2048, total, 2048)]
    assert all(b <= 1.05 * a for a, b in zip(windows, windows[1:]))   # never growing
    assert last < 0.2 * peak                                          # ringing down


def test_sphere104_fp32_vs_fp64(mot):
    """104^3 sphere (1.12M voxels), FIR3 (delta = 0.1125), 640 steps through the pulse: FP32-history
    against FP64, both blocked (B = 8), marched in lockstep chunks."""
    cfg = wl.config("sphere104")
    steps, chunk = 640, 64
    with _context(mot, cfg, "fp64") as c64, _context(mot, cfg, "fp32_history") as c32:
        num = den = 0.0
        for k in range(steps // chunk):
            a = _march_pulse(c64, cfg, 1 + k * chunk, chunk, shift=150.0)
            b = _march_pulse(c32, cfg, 1 + k * chunk, chunk, shift=150.0)
            num += float(np.sum((b - a) ** 2))
            den += float(np.sum(a ** 2))
    rel = np.sqrt(num / den)
    print("\nsphere104: FP32-history vs FP64 rel L2 over %d steps = %.3e" % (steps, rel))
    assert den > 0
    assert rel < 1e-5                  # the FP32-history target
