"""Tested incident field (Eq. E).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

E^b_{m,n} = chi_m (1/V) int_{V_m} eps0 E^i_b(r, n dt) dV with chi_m = (eps_m - 1)/eps_m
(Eq. E; its m', n' subscripts are a typo for m, n).  The incident field is the
modulated Gaussian plane wave p_hat sin(2 pi f_c tau) exp(-tau^2/(2 sigma_t^2)),
tau = t - t0 - r . k_hat (units c0 = 1, eps0 = 1, h = 1).  The voxel average is a
tensor Gauss-Legendre rule with 8 points per axis; the pulse spans many voxels so
the rule is exact to rounding.
"""
import numpy as np


def incident(tau, f_c, sigma_t):
    return np.sin(2.0 * np.pi * f_c * tau) * np.exp(-tau * tau / (2.0 * sigma_t * sigma_t))


def tested_excitation(eps_r, pulse, n_steps, n_first=1, npts=8, with_chi=True):
    """E[n, m, b] for n = n_first .. n_first + n_steps - 1 (1-based times, t = n dt),
    m = u + U (v + V w) (Sec. 2.2, 0-based), b = x, y, z.  Returns an array of shape
    (n_steps, M, 3).  with_chi=False returns the voxel-averaged incident field e_n
    itself (E_n = chi e_n)."""
    W, V, U = eps_r.shape
    chi = (eps_r - 1.0) / eps_r if with_chi else np.ones_like(eps_r)
    xg, wg = np.polynomial.legendre.leggauss(npts)
    off = 0.5 * xg            # offsets inside a unit voxel about its centre
    wo = 0.5 * wg
    k = np.asarray(pulse["k_hat"], float)
    p = np.asarray(pulse["p_hat"], float)
    cu = np.arange(U) + 0.5
    cv = np.arange(V) + 0.5
    cw = np.arange(W) + 0.5
    # projection of the voxel centre and of the quadrature offsets on k_hat
    proj_c = (cw[:, None, None] * k[2] + cv[None, :, None] * k[1] + cu[None, None, :] * k[0])
    proj_o = (off[:, None, None] * k[2] + off[None, :, None] * k[1] + off[None, None, :] * k[0])
    wq = wo[:, None, None] * wo[None, :, None] * wo[None, None, :]
    out = np.zeros((n_steps, U * V * W, 3))
    for i in range(n_steps):
        t = float(n_first + i)
        tau = t - pulse["t0"] - (proj_c[..., None, None, None] + proj_o[None, None, None])
        avg = np.sum(incident(tau, pulse["f_c"], pulse["sigma_t"]) * wq, axis=(-3, -2, -1))
        out[i] = (chi * avg).reshape(-1)[:, None] * p[None, :]
    return out
