"""Positive definite stability analysis matrices (Eq. Dn) and frequency-domain
quantities of the MOT system (Eq. MatrixEquation).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reading of Eq. Dn (R8): D_n = sum_{i=0}^{n} (-1)^i binom(ell - i, n - i) Z_i, so that
D_0 = Z_0 and D_ell = sum_i (-1)^i Z_i = Z(z = -1), the operator at the normalised
frequency theta = pi where the paper's late-time instability lives (Sec. 5.2).
"""
from math import comb

import numpy as np

from .march import dense_Z


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
