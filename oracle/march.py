"""Direct MOT-JVIE march: Eq. PnMOT summed term by term and Eq. MOTInversion solved
with a dense LU factorisation of Z_0.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Layout (Eqs. CurrentVector, ExcitationVector): unknown index 3 m + b, voxel index
m = u + U (v + V w) (0-based), b = x, y, z.  Times are 1-based in the paper
(J_1 is the first unknown) and J_n = 0 for n <= 0 (the field arrives after t = 0).

    Z_l = D_l + fir_l I - diag(chi) G_l,   D_l = T(l) diag(1/eps)   (T(l) = 1/2 at l=0,1)
    Z_0 J_n = E_n - P_{n-1},   P_{n-1} = sum_{l=1}^{ell} Z_l J_{n-l}

The FIR regularisation replaces Z_n by Z_n + delta_n I (Sec. 6.1).
"""
import numpy as np
import scipy.linalg

from .kernel_table import COMPONENTS
from .spline import T_at_lag


def offsets_and_index(U, V, W):
    """Voxel integer coordinates (u, v, w) in m order."""
    w, v, u = np.meshgrid(np.arange(W), np.arange(V), np.arange(U), indexing="ij")
    return np.stack([u.ravel(), v.ravel(), w.ravel()], axis=1)


def g_block(Goct, l, d):
    """3x3 block G_l(d) for integer offset arrays d[..., 3] from the octant table
    (parity: diagonal even in each d_i, (a, b) component odd in d_a and d_b)."""
    ad = np.abs(d)
    out = np.zeros(d.shape[:-1] + (3, 3))
    for c, (a, b) in enumerate(COMPONENTS):
        val = Goct[l, c, ad[..., 2], ad[..., 1], ad[..., 0]]
        if a != b:
            val = val * np.sign(d[..., a]) * np.sign(d[..., b])
        out[..., a, b] = val
        out[..., b, a] = val
    return out


def dense_G(Goct, l, U, V, W):
    """Dense 3M x 3M matrix of G_l over the grid: block (m, m') = G_l(r_m - r_m')."""
    idx = offsets_and_index(U, V, W)
    d = idx[:, None, :] - idx[None, :, :]
    B = g_block(Goct, l, d)                       # (M, M, 3, 3)
    M = idx.shape[0]
    return B.transpose(0, 2, 1, 3).reshape(3 * M, 3 * M)


def dense_Z(Goct, l, eps_r, taps):
    """Z_l (with FIR tap) as a dense 3M x 3M matrix (Eq. Z, reading R2)."""
    W, V, U = eps_r.shape
    e = eps_r.reshape(-1)
    chi = (e - 1.0) / e
    M = e.size
    Z = -np.repeat(chi, 3)[:, None] * dense_G(Goct, l, U, V, W)
    diag = T_at_lag(l) / np.repeat(e, 3)
    if l < len(taps):
        diag = diag + taps[l]
    Z[np.arange(3 * M), np.arange(3 * M)] += diag
    return Z


def march(Goct, eps_r, taps, E, ell=None):
    """J[n, m, b] for n = 1..N_t given E[n, m, b] (same layout), by forward
    substitution with the direct history sum (Eqs. MOTInversion, PnMOT)."""
    nlag = Goct.shape[0]
    if ell is None:
        ell = nlag - 1
    Nt, M, _ = E.shape
    Zs = [dense_Z(Goct, l, eps_r, taps) for l in range(ell + 1)]
    lu = scipy.linalg.lu_factor(Zs[0])
    Zh = np.concatenate(Zs[1:], axis=1)          # [Z_1 | Z_2 | ... | Z_ell]
    J = np.zeros((Nt, 3 * M))
    hist = np.zeros((ell, 3 * M))                # hist[l-1] = J_{n-l}
    for n in range(Nt):
        P = Zh @ hist.reshape(-1)
        J[n] = scipy.linalg.lu_solve(lu, E[n].reshape(-1) - P)
        hist = np.roll(hist, 1, axis=0)
        hist[0] = J[n]
    return J.reshape(Nt, M, 3)


def history_at(Goct, eps_r, taps, Jhist, m_list):
    """P_{n-1} at the voxels m_list by the direct sum over all sources and lags,
    with Jhist[l-1] = J_{n-l} (shape (ell, M, 3)).  Returns (len(m_list), 3)."""
    W, V, U = eps_r.shape
    e = eps_r.reshape(-1)
    chi = (e - 1.0) / e
    idx = offsets_and_index(U, V, W)
    out = np.zeros((len(m_list), 3))
    for i, m in enumerate(m_list):
        d = idx[m][None, :] - idx
        acc = np.zeros(3)
        for l in range(1, Jhist.shape[0] + 1):
            if l >= Goct.shape[0]:
                break
            B = g_block(Goct, l, d)                # (M, 3, 3)
            acc -= chi[m] * np.einsum("mab,mb->a", B, Jhist[l - 1])
            diag = T_at_lag(l) / e[m] + (taps[l] if l < len(taps) else 0.0)
            acc += diag * Jhist[l - 1][m]
        out[i] = acc
    return out


def residual(Goct, eps_r, taps, E, J):
    """max_n |sum_{l=0}^{ell} Z_l J_{n-l} - E_n| / max|E| (the march's defining system)."""
    nlag = Goct.shape[0]
    Zs = [dense_Z(Goct, l, eps_r, taps) for l in range(nlag)]
    Nt = E.shape[0]
    Jf = J.reshape(Nt, -1)
    worst = 0.0
    for n in range(Nt):
        acc = -E[n].reshape(-1)
        for l in range(nlag):
            if n - l < 0:
                break
            acc = acc + Zs[l] @ Jf[n - l]
        worst = max(worst, float(np.abs(acc).max()))
    return worst / max(float(np.abs(E).max()), 1e-300)


def history_sparse(eps_r, taps, src, Jsrc, tgt, nlag, elements=None):
    """P_{n-1} = sum_{l=1}^{nlag-1} Z_l J_{n-l} (Eq. PnMOT, FIR taps included) at the
    voxels `tgt` for a history supported on the voxels `src` only:
    Jsrc[l-1][k] = J_{n-l} at voxel src[k] (shape (nlag-1, len(src), 3)).  Each element
    block G_l(d) comes from ``kernel_table.offset_elements`` at |d| with the parity signs,
    so no octant table of the whole grid is needed.  `elements` may hold a dict
    |d| -> (vol, face) to reuse between calls.  Returns (len(tgt), 3)."""
    from .kernel_table import offset_elements
    W, V, U = eps_r.shape
    e = eps_r.reshape(-1)
    chi = (e - 1.0) / e
    idx = offsets_and_index(U, V, W)
    cache = {} if elements is None else elements
    nh = Jsrc.shape[0]
    out = np.zeros((len(tgt), 3))
    for i, m in enumerate(tgt):
        acc = np.zeros(3)
        for k, s in enumerate(src):
            d = idx[m] - idx[s]
            key = tuple(int(v) for v in np.abs(d))
            if key not in cache:
                cache[key] = offset_elements(key, nlag)
            vol, face = cache[key]
            sg = np.sign(d)
            G = face.copy()                          # [a][b][l]
            for a in range(3):
                for b in range(3):
                    if a != b:
                        G[a, b] *= sg[a] * sg[b]
                G[a, a] -= vol
            for l in range(1, min(nh, nlag - 1) + 1):
                acc -= chi[m] * (G[:, :, l] @ Jsrc[l - 1, k])
        where = np.nonzero(np.asarray(src) == m)[0]
        for k in where:                              # identity part at a source voxel
            for l in range(1, min(nh, nlag - 1) + 1):
                coef = T_at_lag(l) / e[m] + (taps[l] if l < len(taps) else 0.0)
                acc += coef * Jsrc[l - 1, k]
        out[i] = acc
    return out
