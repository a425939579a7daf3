"""Positive definite stability analysis matrices (Eq. Dn) and frequency-domain
quantities of the MOT system (Eq. MatrixEquation).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reading of Eq. Dn (R8): D_n = sum_{i=0}^{n} (-1)^i binom(ell - i, n - i) Z_i, so that
D_0 = Z_0 and D_ell = sum_i (-1)^i Z_i = Z(z = -1), the operator at the normalised
frequency theta = pi where the paper's late-time instability lives (Sec. 5.2).
"""
from math import comb

import numpy as np

from .march import dense_Z, g_block


def pdsa_matrices(Goct, eps_r, taps, ell):
    """[D_0, ..., D_ell] as dense matrices (Eq. Dn, reading R8)."""
    Zs = [dense_Z(Goct, l, eps_r, taps) for l in range(ell + 1)]
    out = []
    for n in range(ell + 1):
        D = np.zeros_like(Zs[0])
        for i in range(n + 1):
            D += (-1) ** i * comb(ell - i, n - i) * Zs[i]
        out.append(D)
    return out


def min_eigs_symmetrised(Ds, eps_r):
    """Smallest eigenvalue of diag(1/chi) D_n for each n (chi > 0 everywhere); the
    scaling by 1/chi makes D_n symmetric for heterogeneous chi (reading R4)."""
    e = np.repeat(eps_r.reshape(-1), 3)
    chi = (e - 1.0) / e
    out = []
    for D in Ds:
        A = D / chi[:, None]
        out.append(float(np.linalg.eigvalsh(0.5 * (A + A.T)).min()))
    return out


def z_operator(Goct, eps_r, taps, z):
    """Z(z) = sum_l Z_l z^{-l} (dense, complex)."""
    nlag = Goct.shape[0]
    out = None
    for l in range(nlag):
        Zl = dense_Z(Goct, l, eps_r, taps) * z ** (-l)
        out = Zl if out is None else out + Zl
    return out


def frequency_identity_solve(Goct, eps_r, taps, E, J, z):
    """Solve Z(z) x = E_N(z) + tail(z) and return (x, J_N(z)) where
    J_N(z) = sum_{n=1}^{N} J_n z^{-n}, E_N(z) likewise, and
    tail(z) = sum_{l} sum_{m=N-l+1}^{N} Z_l J_m z^{-(m+l)} (the terms of the truncated
    product that fall beyond step N).  For the exact march x == J_N(z)."""
    nlag = Goct.shape[0]
    Nt = E.shape[0]
    Jf = J.reshape(Nt, -1)
    Ef = E.reshape(Nt, -1)
    n = np.arange(1, Nt + 1)
    JN = (Jf * (z ** (-n))[:, None]).sum(axis=0)
    EN = (Ef * (z ** (-n))[:, None]).sum(axis=0)
    tail = np.zeros_like(JN)
    for l in range(1, nlag):
        Zl = dense_Z(Goct, l, eps_r, taps)
        for m in range(Nt - l + 1, Nt + 1):
            if m >= 1:
                tail = tail + (Zl @ Jf[m - 1]) * z ** (-(m + l))
    x = np.linalg.solve(z_operator(Goct, eps_r, taps, z), EN + tail)
    return x, JN


def scaled_pdsa_matrix(Goct, eps_r, taps, ell, n):
    """A_n = diag(1/chi) D_n / C(ell, n) restricted to the active voxels (chi > 0).

    D_n follows Eq. Dn (reading R8).  Rows of voxels with chi = 0 only hold their own
    diagonal (their currents stay zero), so the definiteness of D_n is that of its
    active block; the positive factor 1 / C(ell, n) (the weight of Z_0 in D_n) keeps
    the entries of order one for every n and changes no sign.  Symmetric (reading R4).
    """
    Zs = [dense_Z(Goct, l, eps_r, taps) for l in range(n + 1)]
    D = np.zeros_like(Zs[0])
    for i in range(n + 1):
        D += (-1) ** i * comb(ell - i, n - i) * Zs[i]
    e = np.repeat(eps_r.reshape(-1), 3)
    chi = (e - 1.0) / e
    act = chi > 0.0
    A = D[act][:, act] / chi[act][:, None] / comb(ell, n)
    return 0.5 * (A + A.T)


def pdsa_coefficients(ell, n):
    """Weights of Z_i in A_n: (-1)^i C(ell - i, n - i) / C(ell, n), i = 0..n (Eq. Dn)."""
    return np.array([(-1) ** i * comb(ell - i, n - i) / comb(ell, n) for i in range(n + 1)])


def circulant_embedding(Goct, coef, shape, P):
    """Kernel of sum_i coef[i] G_i on the torus of sizes P = (Pu, Pv, Pw) (App. A):
    K[a, b, w, v, u] = G^{ab}(d) at the torus point d mod P for every grid offset
    |d_i| <= N_i - 1, zero elsewhere.  shape = (W, V, U) of the grid."""
    W, V, U = shape
    Pu, Pv, Pw = P
    Gc = np.tensordot(np.asarray(coef), Goct[:len(coef)], axes=(0, 0))[None]
    dz, dy, dx = np.meshgrid(np.arange(-(W - 1), W), np.arange(-(V - 1), V),
                             np.arange(-(U - 1), U), indexing="ij")
    d = np.stack([dx, dy, dz], axis=-1)
    B = g_block(Gc, 0, d)                                  # [..., 3, 3]
    K = np.zeros((3, 3, Pw, Pv, Pu))
    K[:, :, dz % Pw, dy % Pv, dx % Pu] = B.transpose(3, 4, 0, 1, 2)
    return K


def circulant_symbol_eigs(K):
    """Eigenvalues of the circulant operator of K: the 3x3 blocks of its DFT over the
    torus, Khat(k) = sum_d K(d) exp(-2 pi i k . d / P), are real symmetric (parity of
    G), and the circulant is block-diagonalised by the DFT.  Returns [Pw, Pv, Pu, 3]."""
    Kh = np.fft.fftn(K, axes=(2, 3, 4))
    assert np.abs(Kh.imag).max() <= 1e-9 * max(np.abs(Kh.real).max(), 1e-300)
    blocks = np.ascontiguousarray(Kh.real.transpose(2, 3, 4, 0, 1))
    return np.linalg.eigvalsh(0.5 * (blocks + blocks.transpose(0, 1, 2, 4, 3)))


def diagonal_of_scaled(eps_r, taps, ell, n):
    """Diagonal part a_m of A_n = diag(a) - sum_i c_i G_i on the active voxels:
    a_m = sum_i c_i (T(i) / (eps_m - 1) + delta_i / chi_m) (Eq. Z with the FIR taps)."""
    from .spline import T_at_lag
    c = pdsa_coefficients(ell, n)
    e = eps_r.reshape(-1)
    e = e[e > 1.0]
    chi = (e - 1.0) / e
    a = np.zeros_like(e)
    for i in range(n + 1):
        t = taps[i] if i < len(taps) else 0.0
        a += c[i] * (T_at_lag(i) / (e - 1.0) + t / chi)
    return a


def circulant_bounds(Goct, eps_r, taps, ell, n, P):
    """Bracket of the spectrum of A_n (scaled_pdsa_matrix) from the circulant
    embedding of its Toeplitz part: A_n = diag(a) - E^T C E with E selecting the
    active voxels of the torus, so by Weyl's inequality and Cauchy interlacing
        min a - max eig(C) <= lambda(A_n) <= max a - min eig(C).
    Returns (lo, hi, min eig(C), max eig(C))."""
    K = circulant_embedding(Goct, pdsa_coefficients(ell, n), eps_r.shape, P)
    ev = circulant_symbol_eigs(K)
    a = diagonal_of_scaled(eps_r, taps, ell, n)
    return a.min() - ev.max(), a.max() - ev.min(), ev.min(), ev.max()


def circulant_apply(Goct, eps_r, taps, ell, n, P, x, round32=False):
    """A_n x (x, result [M][3], zero rows on voxels with chi = 0) through the circulant
    embedding of the Toeplitz part (App. A): y = a x - E^T IFFT(Khat FFT(E x)).
    With round32 every lag's kernel spectrum Khat_i (i >= 1) is rounded to float32
    before it is weighted: an FP32 store of the spectra, the perturbation N of
    Eq. DellFinitePrecision."""
    W, V, U = eps_r.shape
    Pu, Pv, Pw = P
    c = pdsa_coefficients(ell, n)
    if round32:
        Kh = np.zeros((3, 3, Pw, Pv, Pu))
        for i in range(n + 1):
            one = np.zeros(i + 1)
            one[i] = 1.0
            Ki = np.fft.fftn(circulant_embedding(Goct, one, eps_r.shape, P), axes=(2, 3, 4)).real
            if i >= 1:
                Ki = Ki.astype(np.float32).astype(np.float64)
            Kh += c[i] * Ki
    else:
        Kh = np.fft.fftn(circulant_embedding(Goct, c, eps_r.shape, P), axes=(2, 3, 4)).real
    e = eps_r.reshape(-1)
    act = e > 1.0
    xs = np.where(act[:, None], x, 0.0)
    X = np.zeros((3, Pw, Pv, Pu))
    X[:, :W, :V, :U] = xs.T.reshape(3, W, V, U)
    Xh = np.fft.fftn(X, axes=(1, 2, 3))
    Yh = np.einsum("abwvu,bwvu->awvu", Kh, Xh)
    conv = np.fft.ifftn(Yh, axes=(1, 2, 3)).real[:, :W, :V, :U].reshape(3, -1).T
    a = np.zeros(e.size)
    a[act] = diagonal_of_scaled(eps_r, taps, ell, n)
    return np.where(act[:, None], a[:, None] * xs - conv, 0.0)
