"""Direct-sum march for grids whose dense Z_l do not fit in memory.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The history P_{n-1} = sum_{l>=1} Z_l J_{n-l} (Eq. PnMOT) is summed term by term over
target voxels, source voxels and lags by the plain C loops of ``direct_sum.c`` (built
here with gcc; OpenMP over target voxels when the compiler offers it), and
Z_0 J_n = E_n - P_{n-1} (Eq. MOTInversion) is solved by a dense LU factorisation of
Z_0 restricted to the voxels with chi > 0.  Voxels with eps_r = 1 carry no current
(reading R5: their row reads (T(0) + delta_0) J_n = -(T(1) + ...) J_{n-1} - ... with
every term zero), so they are left out of both the sources and the solve.

``march.march`` (dense Z_l) and this march solve the same system; a ``-m "not gpu"``
test checks that they agree on the 8^3 cube.
"""
import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg

from .march import g_block, offsets_and_index
from .spline import T_at_lag

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "direct_sum.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_direct.so")

_lib = None


def build():
    """Compile direct_sum.c into oracle/_build/liboracle_direct.so (gcc; OpenMP if the
    compiler accepts -fopenmp, else single-threaded)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".tmp"
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", SRC, "-o", tmp]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("gcc failed for %s:\n%s" % (SRC, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.oracle_history.argtypes = [I, I, I, I, P, P, P, I, I, P, I, P, I, P, P]
        lib.oracle_history.restype = I
        _lib = lib
    return _lib


def history(Goct, eps_r, taps, J, n, src, tgt):
    """P_{n-1} (Eq. PnMOT, FIR taps included) at the voxels `tgt` from the currents of
    the voxels `src`, J[k] = J_{k+1} ([>= n-1][M][3]); Goct [ell+1][6][W][V][U] is the
    octant table of a grid of shape eps_r [W][V][U].  Returns [len(tgt)][3]."""
    lib = _load()
    W, V, U = eps_r.shape
    G = np.ascontiguousarray(Goct, dtype=np.float64)
    if G.shape[1:] != (6, W, V, U):
        raise ValueError("table shape %r does not match the grid %r" % (G.shape, eps_r.shape))
    e = np.ascontiguousarray(eps_r, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(np.zeros(0) if taps is None else taps, dtype=np.float64)
    s = np.ascontiguousarray(src, dtype=np.int32)
    g = np.ascontiguousarray(tgt, dtype=np.int32)
    Jc = np.ascontiguousarray(J, dtype=np.float64)
    if n > 1 and Jc.shape[0] < n - 1:
        raise ValueError("J must hold J_1 .. J_{n-1}")
    out = np.zeros((g.size, 3))
    st = lib.oracle_history(U, V, W, G.shape[0], G.ctypes.data, e.ctypes.data,
                            t.ctypes.data if t.size else None, int(t.size), int(s.size),
                            s.ctypes.data, int(g.size), g.ctypes.data, int(n), Jc.ctypes.data,
                            out.ctypes.data)
    if st != 0:
        raise MemoryError("oracle_history: scratch allocation failed")
    return out


def z0_active(Goct, eps_r, taps, active):
    """Dense Z_0 (Eq. Z at lag 0, FIR tap delta_0) on the voxels `active`, unknowns
    ordered [voxel][component]."""
    W, V, U = eps_r.shape
    e = eps_r.reshape(-1)
    chi = (e - 1.0) / e
    idx = offsets_and_index(U, V, W)[active]
    d = idx[:, None, :] - idx[None, :, :]
    B = g_block(Goct, 0, d)                                    # (na, na, 3, 3)
    na = len(active)
    Z = -np.repeat(chi[active], 3)[:, None] * B.transpose(0, 2, 1, 3).reshape(3 * na, 3 * na)
    diag = T_at_lag(0) / np.repeat(e[active], 3) + (taps[0] if len(taps) else 0.0)
    Z[np.arange(3 * na), np.arange(3 * na)] += diag
    return Z


def march(Goct, eps_r, taps, E):
    """J[n, m, b], n = 1..N_t, for the excitation E[n, m, b] by forward substitution
    (Eqs. MOTInversion, PnMOT) with the C direct history sum; J = 0 on voxels with
    eps_r = 1."""
    taps = np.zeros(0) if taps is None else np.asarray(taps, dtype=np.float64)
    Nt, M, _ = E.shape
    e = eps_r.reshape(-1)
    active = np.nonzero(e > 1.0)[0].astype(np.int32)
    J = np.zeros((Nt, M, 3))
    if active.size == 0:
        return J
    lu = scipy.linalg.lu_factor(z0_active(Goct, eps_r, taps, active))
    for n in range(1, Nt + 1):
        P = history(Goct, eps_r, taps, J, n, active, active) if n > 1 else 0.0
        rhs = (E[n - 1, active] - P).reshape(-1)
        J[n - 1, active] = scipy.linalg.lu_solve(lu, rhs).reshape(-1, 3)
    return J
