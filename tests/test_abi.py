"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/mot.h declares (no GPU call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_03323_gb300 import build, mot
    if not os.path.exists(mot.LIB_PATH):
        build.build()
    return mot.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mot_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("mot_create", "mot_set_excitation", "mot_march", "mot_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_2407_03323_gb300 import mot
    assert sorted(mot.EXPORTS) == declared_symbols()


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    """Argument validation happens on the host: a non-cubic voxel, c dt != h and
    eps_r < 1 are MOT_ERR_ARG with a message."""
    out = ctypes.c_void_p()
    eps = (ctypes.c_double * 8)(*([2.0] * 8))
    grid = (ctypes.c_int * 3)(2, 2, 2)
    h_bad = (ctypes.c_double * 3)(1.0, 1.0, 2.0)
    st = lib.mot_create(ctypes.cast(grid, ctypes.c_void_p), ctypes.cast(h_bad, ctypes.c_void_p),
                        1.0, ctypes.cast(eps, ctypes.c_void_p), None, 0, 0, 0, 0,
                        ctypes.byref(out))
    assert st == 1 and not out.value
    assert b"cubes" in lib.mot_last_error(None)
    h = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    st = lib.mot_create(ctypes.cast(grid, ctypes.c_void_p), ctypes.cast(h, ctypes.c_void_p),
                        0.5, ctypes.cast(eps, ctypes.c_void_p), None, 0, 0, 0, 0,
                        ctypes.byref(out))
    assert st == 1 and b"dt" in lib.mot_last_error(None)
    eps[3] = 0.5
    st = lib.mot_create(ctypes.cast(grid, ctypes.c_void_p), ctypes.cast(h, ctypes.c_void_p),
                        1.0, ctypes.cast(eps, ctypes.c_void_p), None, 0, 0, 0, 0,
                        ctypes.byref(out))
    assert st == 1 and b"eps_r" in lib.mot_last_error(None)


def test_fir_magnitude_host_call(lib):
    """mot_fir_magnitude is host-only: the FIR2/3/4 taps of Sec. 6.2 (FIR4 per reading
    R7) have the magnitudes delta sin^k(theta / 2), k = 1, 2, 3 (Eq. FIRmagnitude)."""
    import numpy as np
    import workloads as wl
    from paper_2407_03323_gb300 import mot
    th = np.linspace(0.0, np.pi, 41)
    for k, name in ((1, "fir2"), (2, "fir3"), (3, "fir4")):
        mag = mot.fir_magnitude(wl.fir_taps(name, 0.1), th)
        assert np.abs(mag - 0.1 * np.sin(th / 2) ** k).max() < 1e-15


def test_diagnostic_entry_points_reject_bad_arguments_on_the_host(lib):
    """The PDSA, truncation and frequency-response entry points validate their
    arguments before any device work (NULL context, bad sizes) and return MOT_ERR_ARG."""
    import numpy as np
    out = np.zeros(8)
    info = (ctypes.c_int * 2)()
    assert lib.mot_pdsa_apply(None, 0, 0, out.ctypes.data, out.ctypes.data) == 1
    assert lib.mot_pdsa_bounds(None, 0, 0, out.ctypes.data) == 1
    assert lib.mot_pdsa_lanczos(None, 0, 0, 4, 1, 1, out.ctypes.data,
                                ctypes.cast(info, ctypes.c_void_p), out.ctypes.data) == 1
    assert lib.mot_truncate_table(None, 1e-6) == 1
    J = np.zeros((4, 1, 3))
    f = np.array([0.1])
    e_bad = np.array([1.0])                      # eps_r must exceed 1 at a probe
    assert lib.mot_frequency_response(4, 1, J.ctypes.data, 1.0, 0.2, e_bad.ctypes.data, 0.1,
                                      5.0, 1, f.ctypes.data, out.ctypes.data, None) == 1
    e_ok = np.array([4.0])
    assert lib.mot_frequency_response(4, 1, J.ctypes.data, 1.0, 1.5, e_ok.ctypes.data, 0.1,
                                      5.0, 1, f.ctypes.data, out.ctypes.data, None) == 1
    assert lib.mot_fir_magnitude(None, 3, 1, f.ctypes.data, out.ctypes.data) == 1


def test_barrier_check_rejects_bad_arguments_on_the_host(lib):
    """mot_barrier_check validates its counts and budget before any CUDA call."""
    a, b = ctypes.c_int(), ctypes.c_int()
    for args in ((4, 0, -1, 0.2), (4, 10, 4, 0.2), (4, 10, -2, 0.2), (4, 10, -1, 0.0),
                 (4, 10, -1, 11.0)):
        assert lib.mot_barrier_check(*args, ctypes.byref(a), ctypes.byref(b)) == 1, args


def test_create_padded_rejects_bad_lengths_on_the_host(lib):
    """mot_create_padded checks every FFT length (even, 7-smooth, >= 2N - 1, <= 4096)
    before any CUDA call."""
    out = ctypes.c_void_p()
    eps = (ctypes.c_double * 64)(*([2.0] * 64))
    grid = (ctypes.c_int * 3)(4, 4, 4)
    h = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    for bad in ((6, 8, 8), (8, 8, 9), (22, 8, 8), (8, 8, 4098)):
        fl = (ctypes.c_int * 3)(*bad)
        st = lib.mot_create_padded(ctypes.cast(grid, ctypes.c_void_p),
                                   ctypes.cast(h, ctypes.c_void_p), 1.0,
                                   ctypes.cast(eps, ctypes.c_void_p), None, 0, 0, 0, 0,
                                   ctypes.cast(fl, ctypes.c_void_p), ctypes.byref(out))
        assert st == 1 and not out.value, bad
        assert b"fft_len" in lib.mot_last_error(None)


def test_padding_rules():
    """The host mirror of the library's padding (smallest even 7-smooth length >= 2N - 1)
    and the codelet alternative the tuner may choose."""
    from paper_2407_03323_gb300 import mot
    from paper_2407_03323_gb300.batch import fft_lengths
    for N in range(1, 130):
        P = mot.pad_size(N)
        assert P >= 2 * N - 1 and P % 2 == 0 and mot.smooth7(P)
        assert all(q % 2 or not mot.smooth7(q) for q in range(max(2 * N - 1, 2), P))
        C = mot.codelet_size(N)
        assert C >= 2 * N - 1 and (C == P or (C in mot.CODELET_LENGTHS and C <= 1.5 * P))
    assert fft_lengths(24, "pad") == (48, 48, 48) and fft_lengths(24, "codelet") == (64,) * 3
    assert fft_lengths(40, "codelet") == (96,) * 3 and fft_lengths(104, "pad") == (210,) * 3


def test_level_plan_covers_the_far_lags_causally():
    """mot_level_plan (host only): for every block B and ell, the far levels cover the
    lags B..ell once each in contiguous blocks [a, a + S) that start where the previous
    one ended; every block uses computed currents only (S <= a, Sec. 4.1); the doubling
    plan has S = a = B 2^k; the fitted plan differs at most in its last level, which is
    then the shortest B 2^j reaching ell and at most half its doubling length; and no
    level lies wholly beyond ell."""
    from paper_2407_03323_gb300 import mot
    for B in (2, 4, 8, 16):
        for ell in range(1, 700):
            try:
                dbl = mot.level_plan(B, ell, "blocked_doubling")
            except mot.MotError as e:               # more than 8 levels: raise B
                assert e.status == 1 and B * 2 ** 8 <= ell, (B, ell)
                with pytest.raises(mot.MotError):
                    mot.level_plan(B, ell, "blocked")
                continue
            fit = mot.level_plan(B, ell, "blocked")
            assert dbl == [(B << k, B << k) for k in range(len(dbl))]
            for plan in (dbl, fit):
                if ell < B:
                    assert plan == []
                    continue
                nxt = B
                for S, a in plan:
                    assert a == nxt and S <= a and S % B == 0 and S & (S - 1) == 0
                    assert a <= ell                  # some lag of the level is live
                    nxt = a + S
                assert nxt - 1 >= ell                # lags up to ell are covered
            assert fit[:-1] == dbl[:-1] if dbl else fit == []
            if dbl and fit[-1] != dbl[-1]:
                S, a = fit[-1]
                rest = ell - a + 1
                assert len(dbl) >= 2 and rest <= a // 2
                assert S >= rest and (S == B or S // 2 < rest) and S < dbl[-1][0]
            elif len(dbl) >= 2:
                assert ell - dbl[-1][1] + 1 > dbl[-1][0] // 2
    assert mot.level_plan(8, 182) == [(8, 8), (16, 16), (32, 32), (64, 64), (64, 128)]
    assert mot.level_plan(8, 182, "blocked_doubling")[-1] == (128, 128)
    assert mot.level_plan(8, 182, "direct") == []


def test_level_plan_rejects_bad_arguments(lib):
    n = ctypes.c_int()
    for args in ((3, 100, 1), (1, 100, 1), (8, 0, 1), (8, 100, 7)):
        assert lib.mot_level_plan(*args, 8, ctypes.byref(n), None, None) == 1, args
    assert lib.mot_level_plan(8, 100, 1, 8, None, None, None) == 1
