"""The oracle's C direct-sum history and march (oracle/direct.py, direct_sum.c) and its
sparse-source history (march.history_sparse) against the dense-matrix definitions of
oracle/march.py, which are pinned by the other oracle tests (Eq. PnMOT, Eq.
MOTInversion).  CPU only."""
import numpy as np
import pytest

import workloads as wl


@pytest.fixture(scope="module")
def hetero8(cube8_oracle):
    eps = cube8_oracle["cfg"]["eps_r"].copy()
    eps[2:5, 1:7, 3] = 9.0
    eps[0, 0, :] = 1.0                       # a row of vacuum voxels (chi = 0)
    return eps


def test_c_history_equals_dense_definition(cube8_oracle, hetero8):
    """Random currents on every voxel (vacuum voxels included) and the 9-tap FIR: the C
    loops give the dense sum of Z_l J_{n-l} at every voxel."""
    from oracle import direct, march
    G, ell = cube8_oracle["G"], cube8_oracle["ell"]
    taps = wl.fir_taps("hp9", 0.05)
    rng = np.random.default_rng(3)
    M = hetero8.size
    n = ell + 1
    J = rng.normal(size=(ell, M, 3))                  # J_1 .. J_ell
    Jhist = J[::-1]                                   # Jhist[l-1] = J_{n-l}
    ref = march.history_at(G, hetero8, taps, Jhist, list(range(M)))
    got = direct.history(G, hetero8, taps, J, n, np.arange(M), np.arange(M))
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    # a step early in the march reads only the currents that exist (J_n = 0 for n <= 0)
    n = 4
    ref = march.history_at(G, hetero8, taps, J[:n - 1][::-1], list(range(M)))
    got = direct.history(G, hetero8, taps, J, n, np.arange(M), np.arange(M))
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_c_march_equals_dense_march():
    """The 8^3 eps_r = 12 sphere (vacuum corners) with the 9-tap FIR, 120 steps: the
    march with the C history and the LU of Z_0 on the active voxels equals the dense
    march (LU of the full Z_0)."""
    from oracle import direct, excitation, kernel_table, march
    from oracle.spline import num_lags
    N = 8
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("hp9", 0.05)
    p = wl.pulse(N, 12.0, k_hat=(1.0, 2.0, 2.0), p_hat=(0.0, 1.0, -1.0))
    G, _, _ = kernel_table.octant_table(N, num_lags(N, N, N) + 1)
    E = excitation.tested_excitation(eps, p, 120, n_first=int(p["t0"]) - 60)
    ref = march.march(G, eps, taps, E)
    got = direct.march(G, eps, taps, E)
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)
    out = eps.reshape(-1) == 1.0
    assert np.abs(got[:, out]).max() == 0.0


def test_sparse_history_equals_dense_definition(cube8_oracle, hetero8):
    """history_sparse (elements per offset, parity signs by hand) equals the dense sum
    for currents supported on a few voxels, at the sources and 40 other voxels."""
    from oracle import march
    G, ell = cube8_oracle["G"], cube8_oracle["ell"]
    taps = wl.fir_taps("fir3", 0.1)
    rng = np.random.default_rng(8)
    M = hetero8.size
    src = [0, 77, 300, 511, 8 * 64 + 3]                 # includes a vacuum voxel (0)
    src = [s for s in src if s < M]
    Jh = np.zeros((ell, M, 3))
    Jh[:, src] = rng.normal(size=(ell, len(src), 3))
    tgt = sorted(set(src) | set(int(v) for v in rng.choice(M, 40, replace=False)))
    ref = march.history_at(G, hetero8, taps, Jh, tgt)
    got = march.history_sparse(hetero8, taps, src, Jh[:, src], tgt, ell + 1)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
