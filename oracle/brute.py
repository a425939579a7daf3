"""Per-lag element integrals by Cartesian iterated quadrature that resolves the shells.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Used only by the pins of
``kernel_table``: an independent route to every lag and every component of Eq. Z.

Reading R2 of Eq. Z (see ``kernel_table``): with C_d the autocorrelation of two unit
voxels at offset d, C_d(x) = Lam(x - dx) Lam(y - dy) Lam(z - dz) (Lam the unit hat),

    K^vol_l(d)       = int C_d(x) T''(l - r) / (4 pi r) dx,
    K^face_l^{ab}(d) = int (d_a d_b C_d)(x) T(l - r) / (4 pi r) dx,      r = |x|.

For a != b the weight d_a d_b C_d = Lam'(x_a - d_a) Lam'(x_b - d_b) Lam(x_c - d_c) is
a polynomial on every unit cell of the support [d - 1, d + 1]^3.  For a = b,
d_a^2 Lam(x_a - d_a) = delta(x_a - d_a + 1) - 2 delta(x_a - d_a) + delta(x_a - d_a - 1),
so K^face_aa is a combination of three plane integrals.

T(l - r) and T''(l - r) (``spline``) change form only on the spheres r = k, k integer.
This route never uses cylindrical coordinates, arcs or tanh-sinh (the construction of
``kernel_table``).  Every unit cell (square) is integrated by iterated one-dimensional
Gauss-Legendre rules, x outermost, each interval split wherever the integrand of the
inner integrals changes form:
  z at  +-sqrt(k^2 - x^2 - y^2)               (the sphere itself),
  y at  +-sqrt(k^2 - x^2 - Zb), Zb in {0, z0^2, z1^2}   (a z split point enters or
        leaves the cell, or two of them merge),
  x at  +-sqrt(k^2 - Yb - Zb),  Yb in {0, y0^2, y1^2}.
The inner z pieces carry analytic integrands; the outer pieces can behave like a
square root at their ends, which the substitution t -> 3 t^2 - 2 t^3 of each piece
removes.  Cells (squares) with a corner at the origin, where 1/r is singular, are
mapped by Duffy's pyramids (x_lead = u, the others u v, u w), which cancel 1/r; there
r = u sqrt(1 + v^2 + w^2) < 2, so only the sphere r = 1 splits the u-interval.
"""
import functools

import numpy as np

from .spline import T, T2

FOUR_PI = 4.0 * np.pi


@functools.lru_cache(maxsize=None)
def _gl01(n):
    """Gauss-Legendre nodes and weights on (0, 1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _pieces(lo, hi, cand):
    """Boundaries of the pieces of [lo, hi] split at those candidate points `cand`
    (shape (..., k), NaN = none) that lie inside it: returns (a, b), each (..., p) with
    p - 1 the largest number of inside points of any row; rows with fewer get pieces of
    zero length at the end."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    shape = cand.shape[:-1]
    lo_b = np.broadcast_to(lo, shape)[..., None]
    hi_b = np.broadcast_to(hi, shape)[..., None]
    inside = (cand > lo_b) & (cand < hi_b)            # False for NaN
    c = np.sort(np.where(inside, cand, np.inf), axis=-1)
    k = int(inside.sum(axis=-1).max()) if inside.size else 0
    c = np.minimum(c[..., :k], hi_b)
    B = np.concatenate([lo_b, c, hi_b], axis=-1)
    return B[..., :-1], B[..., 1:]


def _nodes(a, b, n, smooth):
    """Nodes and weights of an n-point rule on every piece [a, b] (arrays (..., p)),
    returned flattened over pieces: (..., p * n).  smooth: t -> 3 t^2 - 2 t^3 first."""
    t, w = _gl01(n)
    if smooth:
        s = t * t * (3.0 - 2.0 * t)
        ds = 6.0 * t * (1.0 - t)
    else:
        s, ds = t, np.ones_like(t)
    L = (b - a)[..., None]
    x = a[..., None] + L * s
    wt = L * (ds * w)
    return x.reshape(x.shape[:-2] + (-1,)), wt.reshape(wt.shape[:-2] + (-1,))


def _sqrt_pm(v):
    """+-sqrt(v) where v > 0, NaN elsewhere; last axis doubled."""
    s = np.where(v > 0.0, np.sqrt(np.maximum(v, 0.0)), np.nan)
    return np.concatenate([s, -s], axis=-1)


def _shells(lo_corner, dim):
    """Integers k strictly between the least and the largest |x| over the unit cell
    (square) with lower corner lo_corner."""
    lo = np.asarray(lo_corner, dtype=np.float64)
    near = np.where(lo > 0, lo, np.where(lo + 1 < 0, -(lo + 1), 0.0))
    far = np.maximum(np.abs(lo), np.abs(lo + 1))
    rmin = float(np.sqrt(np.sum(near ** 2)))
    rmax = float(np.sqrt(np.sum(far ** 2)))
    k0 = int(np.floor(rmin)) + 1
    return [k for k in range(k0, int(np.ceil(rmax))) if rmin < k < rmax]


def _cell3_nodes(c0, n):
    """Nodes (x, y, z) and weights of the iterated rule on the unit cell with lower
    corner c0 (integers), not touching the origin."""
    x0, y0, z0 = (float(v) for v in c0)
    x1, y1, z1 = x0 + 1.0, y0 + 1.0, z0 + 1.0
    K = np.array(_shells(c0, 3), dtype=np.float64)
    Zb = np.array([0.0, z0 * z0, z1 * z1])
    Yb = np.array([0.0, y0 * y0, y1 * y1])
    if K.size:
        cx = _sqrt_pm((K[:, None, None] ** 2 - Yb[None, :, None] - Zb[None, None, :]).ravel())
    else:
        cx = np.zeros(0)
    ax, bx = _pieces(x0, x1, cx[None, :])
    X, WX = _nodes(ax[0], bx[0], n, True)                     # (nx,)
    if K.size:
        cy = _sqrt_pm((K[None, :, None] ** 2 - X[:, None, None] ** 2
                       - Zb[None, None, :]).reshape(X.size, -1))
    else:
        cy = np.zeros((X.size, 0))
    ay, by = _pieces(y0, y1, cy)
    Y, WY = _nodes(ay, by, n, True)                           # (nx, ny)
    if K.size:
        cz = _sqrt_pm(K[None, None, :] ** 2 - X[:, None, None] ** 2 - Y[:, :, None] ** 2)
    else:
        cz = np.zeros(Y.shape + (0,))
    az, bz = _pieces(z0, z1, cz)
    Z, WZ = _nodes(az, bz, n, False)                          # (nx, ny, nz)
    X3 = np.broadcast_to(X[:, None, None], Z.shape)
    Y3 = np.broadcast_to(Y[:, :, None], Z.shape)
    W3 = WX[:, None, None] * WY[:, :, None] * WZ
    return X3.ravel(), Y3.ravel(), Z.ravel(), W3.ravel()


def _duffy3_nodes(c0, n):
    """Nodes and weights on a unit cell with a corner at the origin: three pyramids
    x_lead = u, x_other = u v, u w (v, w in [0, 1]), Jacobian u^2; u split at the
    sphere r = 1 (u = 1 / sqrt(1 + v^2 + w^2))."""
    sg = np.array([1.0 if v == 0 else -1.0 for v in c0])
    t, wt = _gl01(n)
    V, Wv = np.meshgrid(t, t, indexing="ij")
    WVW = np.outer(wt, wt)
    q = np.sqrt(1.0 + V * V + Wv * Wv)
    us = 1.0 / q
    a = np.stack([np.zeros_like(us), us], axis=-1)
    b = np.stack([us, np.ones_like(us)], axis=-1)
    U, WU = _nodes(a, b, n, False)                            # (n, n, 2n)
    xs, ys, zs, ws = [], [], [], []
    for lead in range(3):
        o1, o2 = [i for i in range(3) if i != lead]
        coords = [None, None, None]
        coords[lead] = U
        coords[o1] = U * V[..., None]
        coords[o2] = U * Wv[..., None]
        w = WU * WVW[..., None] * U * U
        xs.append((sg[0] * coords[0]).ravel())
        ys.append((sg[1] * coords[1]).ravel())
        zs.append((sg[2] * coords[2]).ravel())
        ws.append(w.ravel())
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(zs), np.concatenate(ws)


def _square_nodes(c0, h, n):
    """Nodes (p, q) and weights on the unit square with lower corner c0 in the plane at
    height h (r = sqrt(h^2 + p^2 + q^2))."""
    p0, q0 = (float(v) for v in c0)
    p1, q1 = p0 + 1.0, q0 + 1.0
    at_origin = h == 0.0 and p0 in (-1.0, 0.0) and q0 in (-1.0, 0.0)
    if at_origin:     # two triangles p = u, q = u v (and swapped), Jacobian u
        sg = np.array([1.0 if p0 == 0 else -1.0, 1.0 if q0 == 0 else -1.0])
        t, wt = _gl01(n)
        s = np.sqrt(1.0 + t * t)
        us = 1.0 / s
        a = np.stack([np.zeros_like(us), us], axis=-1)
        b = np.stack([us, np.ones_like(us)], axis=-1)
        U, WU = _nodes(a, b, n, False)                        # (n, 2n)
        ps, qs, ws = [], [], []
        for lead in range(2):
            c = [None, None]
            c[lead] = U
            c[1 - lead] = U * t[:, None]
            ps.append((sg[0] * c[0]).ravel())
            qs.append((sg[1] * c[1]).ravel())
            ws.append((WU * wt[:, None] * U).ravel())
        return np.concatenate(ps), np.concatenate(qs), np.concatenate(ws)
    hh = h * h
    near = np.array([p0 if p0 > 0 else (-p1 if p1 < 0 else 0.0),
                     q0 if q0 > 0 else (-q1 if q1 < 0 else 0.0)])
    far = np.array([max(abs(p0), abs(p1)), max(abs(q0), abs(q1))])
    rmin = np.sqrt(hh + np.sum(near ** 2))
    rmax = np.sqrt(hh + np.sum(far ** 2))
    K = np.array([k for k in range(int(np.floor(rmin)) + 1, int(np.ceil(rmax)))
                  if rmin < k < rmax], dtype=np.float64)
    Qb = np.array([0.0, q0 * q0, q1 * q1])
    cp = _sqrt_pm((K[:, None] ** 2 - hh - Qb[None, :]).ravel()) if K.size else np.zeros(0)
    ap, bp = _pieces(p0, p1, cp[None, :])
    Pn, WP = _nodes(ap[0], bp[0], n, True)
    cq = _sqrt_pm(K[None, :] ** 2 - hh - Pn[:, None] ** 2) if K.size else np.zeros((Pn.size, 0))
    aq, bq = _pieces(q0, q1, cq)
    Qn, WQ = _nodes(aq, bq, n, False)                         # (np, nq)
    P2 = np.broadcast_to(Pn[:, None], Qn.shape)
    return P2.ravel(), Qn.ravel(), (WP[:, None] * WQ).ravel()


def _hat(x, d):
    return np.maximum(0.0, 1.0 - np.abs(x - d))


def _dhat(x, d):
    """Lam'(x - d): +1 on (d - 1, d), -1 on (d, d + 1) (the nodes never sit on a knot)."""
    return np.where(x < d, 1.0, -1.0) * (np.abs(x - d) < 1.0)


def _accumulate(r, w, nlag, second):
    """sum over nodes of w T(l - r) / (4 pi r) (or T'') for l = 0..nlag-1."""
    out = np.zeros(nlag)
    f = w / (FOUR_PI * r)
    j = np.floor(r).astype(np.int64)
    for i in range(3):                # T(l - r) != 0 only for l - r in (-1, 2)
        l = j + i
        v = f * (T2(l - r) if second else T(l - r))
        ok = l < nlag
        out += np.bincount(l[ok], weights=v[ok], minlength=nlag)[:nlag]
    return out


def element_lags(d, nlag, n=12):
    """K^vol_l(d) and K^face_l^{ab}(d), l = 0..nlag-1, by the iterated Cartesian rule
    with n nodes per piece.  Returns (vol[nlag], face[3, 3, nlag])."""
    d = np.array([float(v) for v in d])
    vol = np.zeros(nlag)
    face = np.zeros((3, 3, nlag))
    # volume weights on the 8 cells of the support
    for cx in (-1.0, 0.0):
        for cy in (-1.0, 0.0):
            for cz in (-1.0, 0.0):
                c0 = (d[0] + cx, d[1] + cy, d[2] + cz)
                if all(v in (-1.0, 0.0) for v in c0):
                    X, Y, Z, Wn = _duffy3_nodes(c0, n)
                else:
                    X, Y, Z, Wn = _cell3_nodes(c0, n)
                r = np.sqrt(X * X + Y * Y + Z * Z)
                P = (X, Y, Z)
                h = [_hat(P[i], d[i]) for i in range(3)]
                g = [_dhat(P[i], d[i]) for i in range(3)]
                vol += _accumulate(r, Wn * h[0] * h[1] * h[2], nlag, True)
                for a, b in ((0, 1), (0, 2), (1, 2)):
                    c = 3 - a - b
                    face[a, b] += _accumulate(r, Wn * g[a] * g[b] * h[c], nlag, False)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        face[b, a] = face[a, b]
    # diagonal components: planes x_a = d_a + e with weights 1, -2, 1
    for a in range(3):
        p, q = [i for i in range(3) if i != a]
        for e, we in ((-1.0, 1.0), (0.0, -2.0), (1.0, 1.0)):
            hgt = d[a] + e
            for sp in (-1.0, 0.0):
                for sq in (-1.0, 0.0):
                    Pn, Qn, Wn = _square_nodes((d[p] + sp, d[q] + sq), hgt, n)
                    r = np.sqrt(hgt * hgt + Pn * Pn + Qn * Qn)
                    w = Wn * _hat(Pn, d[p]) * _hat(Qn, d[q])
                    face[a, a] += we * _accumulate(r, w, nlag, False)
    return vol, face
