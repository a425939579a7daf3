"""Adjoint of the march and the gradient with respect to the permittivity.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The march solves the block lower-triangular system sum_{l=0}^{ell} Z_l J_{n-l} = E_n,
n = 1..N (Eq. MatrixEquation), with Z_l = T(l)(1 - chi) I + delta_l I - diag(chi) G_l
(Eq. Z, reading R2) and E_n = chi e_n (Eq. E, e_n the voxel-averaged incident field).
For an objective O(J_1..J_N) with g_n = dO/dJ_n, the adjoint variables solve the
transposed (block upper-triangular) system, i.e. a march backwards in time:

    Z_0^T lambda_n = g_n - sum_{l=1}^{ell} Z_l^T lambda_{n+l},    n = N .. 1,

and the gradient is dO/dchi_m = sum_n lambda_n . (dE_n/dchi_m - sum_l dZ_l/dchi_m J_{n-l}),
written out here term by term from the definitions (no identity of the discrete
system is used), then dO/deps_m = dO/dchi_m / eps_m^2.
"""
import numpy as np
import scipy.linalg

from .march import dense_G, dense_Z
from .spline import T_at_lag


def adjoint(Goct, eps_r, taps, g):
    """lambda[n, m, b] for n = 1..N by backward substitution with dense Z_l^T."""
    nlag = Goct.shape[0]
    Nt, M, _ = g.shape
    Zs = [dense_Z(Goct, l, eps_r, taps) for l in range(nlag)]
    lu = scipy.linalg.lu_factor(Zs[0].T)
    lam = np.zeros((Nt, 3 * M))
    gf = g.reshape(Nt, -1)
    for n in range(Nt - 1, -1, -1):
        rhs = gf[n].copy()
        for l in range(1, nlag):
            if n + l < Nt:
                rhs -= Zs[l].T @ lam[n + l]
        lam[n] = scipy.linalg.lu_solve(lu, rhs)
    return lam.reshape(Nt, M, 3)


def gradient_chi(Goct, eps_r, taps, e_inc, J, lam):
    """dO/dchi_m = sum_n lambda_n . (e_n - sum_l dZ_l/dchi J_{n-l}) per voxel, with
    dZ_l/dchi_m = -T(l) P_m - P_m G_l (P_m the projector on voxel m's 3 rows) and
    dE_n/dchi_m = P_m e_n."""
    W, V, U = eps_r.shape
    nlag = Goct.shape[0]
    Nt, M, _ = J.shape
    Gs = [dense_G(Goct, l, U, V, W) for l in range(nlag)]
    Jf = J.reshape(Nt, -1)
    out = np.zeros(M)
    for n in range(Nt):
        s = e_inc[n].reshape(-1).copy()
        for l in range(nlag):
            if n - l < 0:
                break
            s += T_at_lag(l) * Jf[n - l] + Gs[l] @ Jf[n - l]
        out += (lam[n].reshape(-1) * s).reshape(M, 3).sum(axis=1)
    return out


def gradient_eps(Goct, eps_r, taps, e_inc, J, lam):
    """dO/deps_m = dO/dchi_m * dchi/deps = dO/dchi_m / eps_m^2."""
    return gradient_chi(Goct, eps_r, taps, e_inc, J, lam) / eps_r.reshape(-1) ** 2
