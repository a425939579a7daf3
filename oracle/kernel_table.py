"""Interaction-element quadrature for the MOT-JVIE (Eq. Z, operator S of Eq. TDJVIE).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Units: voxel edge h = 1, c dt = 1, eps0 = 1 (the paper's runs all have c dt = h).

Reading of Eq. Z (R2).  With A(r,t) the retarded potential of F and
(lap - c^-2 d_t^2) A = -F, the operator is S(F) = grad div A - c^-2 d_t^2 A + F.
Testing with the voxel average at t = n dt (Eq. TestOperator) and expanding with
piecewise-constant voxels (Eq. SpatialBasis) and the spline T (``spline``) gives

    Z_l^{ba}(m, m') = delta_ab delta_mm' T(l)(1 - chi_m) - chi_m G_l^{ba}(d),
    G_l^{ba}(d)     = K^face_l^{ba}(d) - delta_ab K^vol_l(d),     d = r_m - r_m',

where, with C_d(x) = Lam(x-dx) Lam(y-dy) Lam(z-dz) the autocorrelation of two unit
voxels (Lam the unit hat) and r = |x|,

    K^vol_l(d)       = int C_d(x) T''(l - r) / (4 pi r) dx ,
    K^face_l^{ba}(d) = int (d_b d_a C_d)(x) T(l - r) / (4 pi r) dx .

The second form is the double surface integral -(1/V) oint oint n_b n'_a T/(4 pi R)
of the grad-div term after moving both derivatives onto the voxel indicators.

Route (the oracle's): cylindrical coordinates about one axis.  Every weight used is
separable, w(x, y, z) = w_xy(x, y) w_z(z), so

    int w f(r) dx = int_0^inf  s A(s) H(s) ds,
    A(s) = int_0^{2 pi} w_xy(s cos phi, s sin phi) dphi      (closed form, arcs),
    H(s) = int w_z(z) f(sqrt(s^2 + z^2)) dz                  (Gauss-Legendre per piece,
                                                              closed form for r < 1).

The s-integral is split at every radius where A or H changes form and each piece is
integrated with the tanh-sinh rule, which absorbs the square-root and logarithmic
end-point behaviour at those radii.
"""
import functools
import numpy as np

FOUR_PI = 4.0 * np.pi

# ---------------------------------------------------------------- quadrature rules


@functools.lru_cache(maxsize=None)
def _tanh_sinh(h=1.0 / 10.0, tmax=3.2):
    """Tanh-sinh nodes/weights on [0, 1]: x = (1 + tanh(pi/2 sinh t)) / 2."""
    k = np.arange(-int(np.ceil(tmax / h)), int(np.ceil(tmax / h)) + 1)
    t = k * h
    u = 0.5 * np.pi * np.sinh(t)
    x = 1.0 / (1.0 + np.exp(-2.0 * u))
    w = h * 0.25 * np.pi * np.cosh(t) / np.cosh(u) ** 2
    keep = (x > 0.0) & (x < 1.0) & (w > 1e-300)
    return x[keep], w[keep]


@functools.lru_cache(maxsize=None)
def _gauss_legendre(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


# ---------------------------------------------------------------- 2D weights (arcs)

def _hat_pieces(d, deriv):
    """Pieces (lo, hi, a0, a1) of Lam(x - d) (deriv=0) or Lam'(x - d) (deriv=1)."""
    if deriv == 0:
        return [(d - 1.0, d, 1.0 - d, 1.0), (d, d + 1.0, 1.0 + d, -1.0)]
    return [(d - 1.0, d, 1.0, 0.0), (d, d + 1.0, -1.0, 0.0)]


def _reflect(piece):
    lo, hi, a0, a1 = piece
    if hi <= 0.0:                       # piece lies in x <= 0: x -> -x
        return (-hi, -lo, a0, -a1)
    return piece


def _cells(dp, dq, deriv):
    """First-quadrant cells of w_xy = L(p - dp) L(q - dq), L = Lam or Lam' (deriv).

    Each cell is (x0, x1, y0, y1, wx0, sx, wy0, sy): on the cell the weight is
    (wx0 + sx (x - x0)) (wy0 + sy (y - y0)), i.e. stored in coordinates local to the
    cell corner so that far cells lose no digits to large polynomial coefficients."""
    cells = []
    for px in _hat_pieces(dp, deriv):
        x0, x1, a0, a1 = _reflect(px)
        for py in _hat_pieces(dq, deriv):
            y0, y1, b0, b1 = _reflect(py)
            cells.append((x0, x1, y0, y1, a0 + a1 * x0, a1, b0 + b1 * y0, b1))
    return cells


_ARC_GL = 12


def _arc_integral(s, cells):
    """A(s) = int_0^{2pi} w_xy(s cos phi, s sin phi) dphi for first-quadrant cells.

    On a first-quadrant cell the circle is a single arc [phi_a, phi_b]: phi_a is the
    larger of the angles where it leaves x <= x1 and enters y >= y0, phi_b the
    smaller of the angles where it leaves x >= x0 and y <= y1.  The (entire)
    integrand is integrated over the arc with a 12-point Gauss rule."""
    out = np.zeros_like(s)
    xg, wg = _gauss_legendre(_ARC_GL)
    for (x0, x1, y0, y1, wx0, sx, wy0, sy) in cells:
        s2 = s * s
        xa1 = np.where(x1 < s, x1, s)
        ya1 = np.where(x1 < s, np.sqrt(np.maximum(s2 - x1 * x1, 0.0)), 0.0)
        xa2 = np.sqrt(np.maximum(s2 - y0 * y0, 0.0))
        ya2 = np.full_like(s, y0)
        pick = ya2 > ya1
        Xa = np.where(pick, xa2, xa1)
        Ya = np.where(pick, ya2, ya1)
        xb1 = np.full_like(s, x0)
        yb1 = np.sqrt(np.maximum(s2 - x0 * x0, 0.0))
        xb2 = np.where(y1 < s, np.sqrt(np.maximum(s2 - y1 * y1, 0.0)), 0.0)
        yb2 = np.where(y1 < s, y1, s)
        pick = yb2 < yb1
        Xb = np.where(pick, xb2, xb1)
        Yb = np.where(pick, yb2, yb1)
        valid = (x0 < s) & (y0 < s) & (Yb > Ya)
        pa = np.arctan2(Ya, Xa)
        pb = np.arctan2(Yb, Xb)
        half = np.where(valid, 0.5 * (pb - pa), 0.0)
        phi = (0.5 * (pa + pb))[:, None] + half[:, None] * xg[None, :]
        x = s[:, None] * np.cos(phi)
        y = s[:, None] * np.sin(phi)
        w = (wx0 + sx * (x - x0)) * (wy0 + sy * (y - y0))
        out += half * (w @ wg)
    return out


# ---------------------------------------------------------------- lag scatter

def _scatter(r, w, j, kind, nlag):
    """Add w * f_l(r) into lag bins for the three lags j, j+1, j+2 reached from the
    shell j = floor(r): f = T(l - r)/(4 pi r) (kind 'T') or T''(l - r)/(4 pi r)."""
    out = np.zeros(nlag + 3)
    sig = r - j
    base = w / (FOUR_PI * r)
    if kind == "T":
        v0 = base * 0.5 * (1.0 - sig) ** 2
        v1 = base * 0.5 * (1.0 + 2.0 * sig - 2.0 * sig * sig)
        v2 = base * 0.5 * sig * sig
    else:
        v0, v1, v2 = base, -2.0 * base, base
    out += np.bincount(j, weights=v0, minlength=nlag + 3)[: nlag + 3]
    out += np.bincount(j + 1, weights=v1, minlength=nlag + 3)[: nlag + 3]
    out += np.bincount(j + 2, weights=v2, minlength=nlag + 3)[: nlag + 3]
    return out[:nlag]


def _shell0_moments(s, z0, z1, a, b):
    """Closed-form int_{z0}^{z1} (a + b z) r^k dz, k = -1, 0, 1, r = sqrt(s^2 + z^2)."""
    r0 = np.sqrt(s * s + z0 * z0)
    r1 = np.sqrt(s * s + z1 * z1)
    as0 = np.arcsinh(z0 / s)
    as1 = np.arcsinh(z1 / s)
    Im1 = a * (as1 - as0) + b * (r1 - r0)
    I0 = a * (z1 - z0) + b * 0.5 * (z1 * z1 - z0 * z0)
    I1 = (a * 0.5 * ((z1 * r1 + s * s * as1) - (z0 * r0 + s * s * as0))
          + b * (r1 ** 3 - r0 ** 3) / 3.0)
    return Im1, I0, I1


# ---------------------------------------------------------------- one axis pass

def _axis_pass(dp, dq, dz, nlag_out, n_z=20, ts=None):
    """Integrals for one cylinder axis (z) at in-plane offset (dp, dq) and axial dz.

    Returns (vol, diag, off): arrays over lags of
      vol  = int Lam Lam Lam  T''/(4 pi r)               (K^vol)
      diag = int Lam Lam (d_z^2 Lam) T/(4 pi r)          (K^face along the axis)
      off  = int Lam' Lam' Lam T/(4 pi r)                (K^face in the (p, q) plane)
    """
    nlag = nlag_out + 3
    cellsL = _cells(dp, dq, 0)
    cellsD = _cells(dp, dq, 1)
    zk = np.array([dz - 1.0, dz, dz + 1.0])
    smax = max(np.hypot(c[1], c[3]) for c in cellsL)
    zmax = max(abs(dz - 1.0), abs(dz + 1.0))
    rmax = np.hypot(smax, zmax)
    J = int(np.floor(rmax)) + 1
    # shells that can meet the support box: j from floor(r_min) to floor(r_max) + 1
    rmin = np.sqrt(max(abs(dp) - 1.0, 0.0) ** 2 + max(abs(dq) - 1.0, 0.0) ** 2
                   + max(abs(dz) - 1.0, 0.0) ** 2)
    J0 = max(int(np.floor(rmin)), 1)
    # breakpoints in s
    bp = [0.0, smax]
    for c in cellsL:
        x0, x1, y0, y1 = c[:4]
        bp += [x0, x1, y0, y1, np.hypot(x0, y0), np.hypot(x0, y1), np.hypot(x1, y0),
               np.hypot(x1, y1)]
    for j in range(J0, J + 1):
        bp.append(float(j))
        for ze in zk:
            if j > abs(ze):
                bp.append(np.sqrt(j * j - ze * ze))
    bp = np.unique(np.clip(np.array(bp), 0.0, smax))
    keep = np.concatenate([[True], np.diff(bp) > 1e-14])
    bp = bp[keep]
    a, b = bp[:-1], bp[1:]
    xt, wt = ts if ts is not None else _tanh_sinh()
    s = (a[:, None] + (b - a)[:, None] * xt[None, :]).ravel()
    ws = ((b - a)[:, None] * wt[None, :]).ravel()
    AL = _arc_integral(s, cellsL)
    AD = _arc_integral(s, cellsD)
    outer_L = ws * s * AL
    outer_D = ws * s * AD

    # ---- diag face: z-weight is delta(z-dz+1) - 2 delta(z-dz) + delta(z-dz-1)
    diag = np.zeros(nlag)
    for ze, we in zip(zk, (1.0, -2.0, 1.0)):
        r = np.sqrt(s * s + ze * ze)
        j = np.floor(r).astype(np.int64)
        diag += _scatter(r, we * outer_L, j, "T", nlag)

    # ---- H(s) with the hat weight in z: pieces between knots and shell crossings
    cand = [np.broadcast_to(zk[None, :], (s.size, 3))]
    for j in range(J0, J + 1):
        zc = np.sqrt(np.maximum(j * j - s * s, 0.0))
        ok = j > s
        cand.append(np.where(ok, zc, zk[0])[:, None])
        cand.append(np.where(ok, -zc, zk[0])[:, None])
    Z = np.clip(np.concatenate(cand, axis=1), zk[0], zk[2])
    Z.sort(axis=1)
    z0, z1 = Z[:, :-1], Z[:, 1:]
    zm = 0.5 * (z0 + z1)
    # hat weight a + b z of the z-cell holding the piece
    in_lo = zm < dz
    ha = np.where(in_lo, 1.0 - dz, 1.0 + dz)
    hb = np.where(in_lo, 1.0, -1.0)
    S = np.broadcast_to(s[:, None], z0.shape)
    rm = np.sqrt(S * S + zm * zm)
    jpiece = np.floor(rm).astype(np.int64)
    length = z1 - z0
    live = length > 0.0
    vol = np.zeros(nlag)
    off = np.zeros(nlag)
    # shell 0 (r < 1): closed form
    m0 = live & (jpiece == 0)
    if np.any(m0):
        Im1, I0, I1 = _shell0_moments(S[m0], z0[m0], z1[m0], ha[m0], hb[m0])
        oL = np.broadcast_to(outer_L[:, None], z0.shape)[m0]
        oD = np.broadcast_to(outer_D[:, None], z0.shape)[m0]
        vol[0] += np.sum(oL * Im1) / FOUR_PI
        vol[1] += -2.0 * np.sum(oL * Im1) / FOUR_PI
        vol[2] += np.sum(oL * Im1) / FOUR_PI
        c = 1.0 / (2.0 * FOUR_PI)
        off[0] += c * np.sum(oD * (Im1 - 2.0 * I0 + I1))
        off[1] += c * np.sum(oD * (Im1 + 2.0 * I0 - 2.0 * I1))
        off[2] += c * np.sum(oD * I1)
    # shells j >= 1: Gauss-Legendre on each piece
    m1 = live & (jpiece >= 1)
    if np.any(m1):
        xg, wg = _gauss_legendre(n_z)
        Sm, z0m, z1m = S[m1], z0[m1], z1[m1]
        ham, hbm, jm = ha[m1], hb[m1], jpiece[m1]
        oL = np.broadcast_to(outer_L[:, None], z0.shape)[m1]
        oD = np.broadcast_to(outer_D[:, None], z0.shape)[m1]
        half = 0.5 * (z1m - z0m)
        zz = 0.5 * (z0m + z1m)[:, None] + half[:, None] * xg[None, :]
        rr = np.sqrt(Sm[:, None] ** 2 + zz * zz)
        wz = half[:, None] * wg[None, :] * (ham[:, None] + hbm[:, None] * zz)
        jj = np.broadcast_to(jm[:, None], zz.shape).ravel()
        rr = rr.ravel()
        vol += _scatter(rr, (wz * oL[:, None]).ravel(), jj, "T2", nlag)
        off += _scatter(rr, (wz * oD[:, None]).ravel(), jj, "T", nlag)
    return vol[:nlag_out], diag[:nlag_out], off[:nlag_out]


# ---------------------------------------------------------------- per offset

def offset_elements(d, nlag, n_z=20, ts=None):
    """K^vol_l(d) and K^face_l^{ba}(d), l = 0..nlag-1, for one offset d = (dx, dy, dz).

    Three cylinder-axis passes: axis z gives K^face_zz and K^face_xy, axis x gives
    K^face_xx and K^face_yz, axis y gives K^face_yy and K^face_zx.  K^vol is taken
    from the z pass (the other two passes recompute it by another cut; tests compare).
    Returns (vol[nlag], face[3, 3, nlag]).
    """
    dx, dy, dz = (float(v) for v in d)
    face = np.zeros((3, 3, nlag))
    vol_z, face[2, 2], face[0, 1] = _axis_pass(dx, dy, dz, nlag, n_z, ts)
    _, face[0, 0], face[1, 2] = _axis_pass(dy, dz, dx, nlag, n_z, ts)
    _, face[1, 1], face[2, 0] = _axis_pass(dz, dx, dy, nlag, n_z, ts)
    face[1, 0] = face[0, 1]
    face[2, 1] = face[1, 2]
    face[0, 2] = face[2, 0]
    return vol_z, face


# component order used for tables: xx, yy, zz, xy, xz, yz
COMPONENTS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def octant_table(N, nlag=None, n_z=20, ts=None):
    """G_l^{ba}(d) on the octant d in [0, N-1]^3 for an N^3 grid.

    Returns (G, Kvol, Kface): G[l, c, dz, dy, dx] with c over ``COMPONENTS``,
    Kvol[l, dz, dy, dx], Kface[l, c, dz, dy, dx].  Uses the axis-permutation symmetry
    of the cube: elements are computed once per sorted offset and permuted.
    Other octants follow from parity: diagonal components and K^vol are even in each
    d_i, the (a, b) off-diagonal component is odd in d_a and d_b.
    """
    from .spline import num_lags
    if nlag is None:
        nlag = num_lags(N, N, N) + 1
    G = np.zeros((nlag, 6, N, N, N))
    Kv = np.zeros((nlag, N, N, N))
    Kf = np.zeros((nlag, 6, N, N, N))
    import itertools
    done = {}
    for dz in range(N):
        for dy in range(N):
            for dx in range(N):
                d = (dx, dy, dz)
                key = tuple(sorted(d, reverse=True))
                if key not in done:
                    done[key] = offset_elements(key, nlag, n_z, ts)
                vol_k, face_k = done[key]
                # find permutation p with d[i] = key[p[i]]
                for p in itertools.permutations(range(3)):
                    if all(d[i] == key[p[i]] for i in range(3)):
                        break
                Kv[:, dz, dy, dx] = vol_k
                for c, (a, b) in enumerate(COMPONENTS):
                    Kf[:, c, dz, dy, dx] = face_k[p[a], p[b]]
                    G[:, c, dz, dy, dx] = face_k[p[a], p[b]] - (vol_k if a == b else 0.0)
    return G, Kv, Kf


def full_offset_value(Goct, l, a, b, d):
    """G_l^{ab}(d) for any integer d from the octant table using the parity rules."""
    comp = COMPONENTS.index((min(a, b), max(a, b)))
    ad = [abs(int(v)) for v in d]
    val = Goct[l, comp, ad[2], ad[1], ad[0]]
    if a != b:
        val = val * np.sign(d[a]) * np.sign(d[b])
    return val
