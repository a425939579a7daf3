"""Independent Cartesian route to the lag-summed element integrals, used only to pin
``kernel_table``.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

It shares nothing with the cylindrical construction of ``kernel_table``.

Static (lag-summed) integrals.  Because T is a partition of unity that reproduces
polynomials up to degree 2 (sum_l T(l - r) = 1, sum_l l T(l - r) = r + 1/2,
sum_l l^2 T(l - r) = r^2 + r + 1/2), the lag moments of the table reduce to static
integrals over the voxel autocorrelation C_d (Eq. Z summed over n - n'):

    sum_l l^2 K^vol_l(d)      = 2 int C_d / (4 pi r)                 = 2 S(d)
    sum_l K^face_l^{ab}(d)    = int d_a d_b C_d / (4 pi r)           = F^{ab}(d)
    sum_l l K^face_l^{ab}(d)  = F^{ab}(d) / 2
    sum_l l^2 K^face_l^{ab}(d)= int d_a d_b C_d r / (4 pi) + F^{ab}(d) / 2

computed here by tensor Gauss-Legendre on the unit cells of C_d, with a Duffy
(pyramid) map on cells that have the 1/r singularity at a corner.

Each lag and component on its own is pinned by ``brute`` (a Cartesian iterated rule
that resolves the shells r = integer).
"""
import functools
import itertools
import numpy as np

FOUR_PI = 4.0 * np.pi


@functools.lru_cache(maxsize=None)
def _gl(n):
    return np.polynomial.legendre.leggauss(n)


def _hat(x, d):
    return np.maximum(0.0, 1.0 - np.abs(x - d))


def _dhat(x, d):
    """Derivative of Lam(x - d): +1 on (d-1, d), -1 on (d, d+1)."""
    return np.where((x > d - 1.0) & (x < d), 1.0, np.where((x > d) & (x < d + 1.0), -1.0, 0.0))


def _weight3(d, kind, a=None, b=None):
    """Weight on R^3 for the static integrals: C_d ('C') or d_a d_b C_d, a != b ('AB')."""
    dx, dy, dz = d

    def w(x, y, z):
        X = (x, y, z)
        if kind == "C":
            return _hat(x, dx) * _hat(y, dy) * _hat(z, dz)
        out = np.ones_like(x)
        for i in range(3):
            if i in (a, b):
                out = out * _dhat(X[i], d[i])
            else:
                out = out * _hat(X[i], d[i])
        return out
    return w


def _cell_integral3(w, f, lo, n=20):
    """int over the unit cell [lo, lo+1]^3 of w(x) f(|x|) dx."""
    xg, wg = _gl(n)
    t = 0.5 * (xg + 1.0)
    wt = 0.5 * wg
    corner_at_origin = all(v in (-1.0, 0.0) for v in lo)
    if not corner_at_origin:
        X = lo[0] + t[:, None, None]
        Y = lo[1] + t[None, :, None]
        Z = lo[2] + t[None, None, :]
        X, Y, Z = np.broadcast_arrays(X, Y, Z)
        W = wt[:, None, None] * wt[None, :, None] * wt[None, None, :]
        r = np.sqrt(X * X + Y * Y + Z * Z)
        return float(np.sum(W * w(X, Y, Z) * f(r)))
    # Duffy: the origin is a corner; direction of the cell along each axis
    sgn = [1.0 if v == 0.0 else -1.0 for v in lo]
    U = t[:, None, None]
    V = t[None, :, None]
    Wv = t[None, None, :]
    U, V, Wv = np.broadcast_arrays(U, V, Wv)
    Wt = wt[:, None, None] * wt[None, :, None] * wt[None, None, :]
    total = 0.0
    for lead in range(3):
        coords = [None, None, None]
        others = [i for i in range(3) if i != lead]
        coords[lead] = U
        coords[others[0]] = U * V
        coords[others[1]] = U * Wv
        X = sgn[0] * coords[0]
        Y = sgn[1] * coords[1]
        Z = sgn[2] * coords[2]
        r = np.sqrt(X * X + Y * Y + Z * Z)
        total += float(np.sum(Wt * U * U * w(X, Y, Z) * f(r)))
    return total


def _cell_integral2(w2, f, h, lo, n=20):
    """int over the unit square [lo, lo+1]^2 (in the plane at height h) of
    w2(p, q) f(sqrt(h^2 + p^2 + q^2))."""
    xg, wg = _gl(n)
    t = 0.5 * (xg + 1.0)
    wt = 0.5 * wg
    if h != 0.0 or not all(v in (-1.0, 0.0) for v in lo):
        P = lo[0] + t[:, None]
        Q = lo[1] + t[None, :]
        P, Q = np.broadcast_arrays(P, Q)
        W = wt[:, None] * wt[None, :]
        return float(np.sum(W * w2(P, Q) * f(np.sqrt(h * h + P * P + Q * Q))))
    sgn = [1.0 if v == 0.0 else -1.0 for v in lo]
    U = t[:, None]
    V = t[None, :]
    U, V = np.broadcast_arrays(U, V)
    W = wt[:, None] * wt[None, :]
    total = 0.0
    for lead in range(2):
        c = [None, None]
        c[lead] = U
        c[1 - lead] = U * V
        P = sgn[0] * c[0]
        Q = sgn[1] * c[1]
        total += float(np.sum(W * U * w2(P, Q) * f(np.sqrt(P * P + Q * Q))))
    return total


def _support_cells(d):
    return [(d[0] + i, d[1] + j, d[2] + k) for i in (-1.0, 0.0) for j in (-1.0, 0.0)
            for k in (-1.0, 0.0)]


def static_S(d, n=20):
    """S(d) = int C_d(x) / (4 pi |x|) dx  (static potential of two unit voxels)."""
    w = _weight3(tuple(float(v) for v in d), "C")
    f = lambda r: 1.0 / (FOUR_PI * r)
    return sum(_cell_integral3(w, f, lo, n) for lo in _support_cells(d))


def static_face(d, a, b, moment=-1, n=20):
    """int (d_a d_b C_d)(x) r^(moment+1) / (4 pi r) dx, i.e. F^{ab}(d) for moment=-1
    and int d_a d_b C_d r / (4 pi) for moment=+1 (rewritten with f(r) = r^m / 4pi)."""
    d = tuple(float(v) for v in d)
    f = (lambda r: 1.0 / (FOUR_PI * r)) if moment == -1 else (lambda r: r / FOUR_PI)
    if a != b:
        w = _weight3(d, "AB", a, b)
        return sum(_cell_integral3(w, f, lo, n) for lo in _support_cells(d))
    # diagonal: d_a^2 Lam = delta(x_a - d_a + 1) - 2 delta(x_a - d_a) + delta(...)
    p, q = [i for i in range(3) if i != a]
    w2 = lambda P, Q: _hat(P, d[p]) * _hat(Q, d[q])
    total = 0.0
    for e, we in ((-1.0, 1.0), (0.0, -2.0), (1.0, 1.0)):
        h = d[a] + e
        for lo in [(d[p] + i, d[q] + j) for i in (-1.0, 0.0) for j in (-1.0, 0.0)]:
            total += we * _cell_integral2(w2, f, h, lo, n)
    return total
