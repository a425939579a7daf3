"""Pins of the oracle's element quadrature (Eq. Z) against mathematics that does not
go through its cylindrical construction."""
import itertools
import os

import numpy as np
import pytest

from oracle import kernel_table as kt
from oracle import spline, static

OFFSETS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 1, 0), (3, 2, 1), (6, 0, 2),
           (5, 5, 4)]


def test_spline_partition_of_unity_and_moments():
    """T reproduces polynomials of degree <= 2 (the B-spline reading R1)."""
    for r in np.linspace(0.0, 7.3, 41):
        l = np.arange(-3, 12)
        Tv = spline.T(l - r)
        assert abs(Tv.sum() - 1.0) < 1e-14
        assert abs((l * Tv).sum() - (r + 0.5)) < 1e-13
        assert abs((l * l * Tv).sum() - (r * r + r + 0.5)) < 1e-12
        assert abs(spline.T2(l - r).sum()) < 1e-14
    # C^1 continuity at the knots and support (-1, 2)
    for k in (-1.0, 0.0, 1.0, 2.0):
        e = 1e-7
        assert abs(spline.T(k - e) - spline.T(k + e)) < 1e-6
    assert spline.T(-1.0) == 0.0 and spline.T(2.0) == 0.0
    assert spline.T_at_lag(0) == 0.5 and spline.T_at_lag(1) == 0.5 and spline.T_at_lag(2) == 0


def test_num_lags_eq_ell():
    """Eq. Ell for the grids used by the runs."""
    assert spline.num_lags(8, 8, 8) == 15
    assert spline.num_lags(32, 32, 32) == 57
    assert spline.num_lags(48, 48, 48) == 85
    assert spline.num_lags(104, 104, 104) == 182


@pytest.mark.parametrize("d", OFFSETS)
def test_trace_identity(d):
    """sum_a K^face_aa,l(d) = K^vol_l(d) - delta_{d,0} T(l): follows from
    lap[T(t - r)/(4 pi r)] = T''(t - r)/(4 pi r) - T(t) delta(x) and ties the plane
    (delta-weight) integrals to the volume integral."""
    nl = 24
    vol, face = kt.offset_elements(d, nl)
    tr = face[0, 0] + face[1, 1] + face[2, 2]
    dlt = np.array([spline.T_at_lag(l) if d == (0, 0, 0) else 0.0 for l in range(nl)])
    assert np.abs(tr - (vol - dlt)).max() < 1e-13 * max(1.0, np.abs(vol).max())


@pytest.mark.parametrize("d", OFFSETS)
def test_lag_moments_match_static_route(d):
    """Lag moments of the table equal static integrals computed by an independent
    Cartesian tensor-Gauss / Duffy route."""
    nl = 24
    l = np.arange(nl)
    vol, face = kt.offset_elements(d, nl)
    S = static.static_S(d)
    assert abs(vol.sum()) < 1e-14
    assert abs((l * vol).sum()) < 1e-13
    assert abs((l * l * vol).sum() - 2.0 * S) < 1e-13
    for a, b in itertools.product(range(3), range(3)):
        F = static.static_face(d, a, b)
        Q = static.static_face(d, a, b, moment=1)
        assert abs(face[a, b].sum() - F) < 1e-13
        assert abs((l * face[a, b]).sum() - 0.5 * F) < 1e-13
        assert abs((l * l * face[a, b]).sum() - (Q + 0.5 * F)) < 2e-13


def test_self_term_demagnetisation():
    """Static self term of a cube: sum_l K^face_aa(0) = -1/3 for every a, zero
    off-diagonal; S(0) is the unit-cube self potential."""
    vol, face = kt.offset_elements((0, 0, 0), 8)
    for a in range(3):
        assert abs(face[a, a].sum() + 1.0 / 3.0) < 1e-14
        for b in range(3):
            if a != b:
                assert abs(face[a, b]).max() < 1e-15
    assert abs(static.static_S((0, 0, 0)) - 0.149789680899496) < 1e-13


def test_parity_zero_components():
    """The (a, b) off-diagonal element is odd in d_a and d_b, so it vanishes when
    d_a = 0 or d_b = 0."""
    vol, face = kt.offset_elements((2, 0, 3), 12)
    assert np.abs(face[0, 1]).max() < 1e-15
    assert np.abs(face[1, 2]).max() < 1e-15
    assert np.abs(face[0, 2]).max() > 1e-4


def test_vol_is_axis_independent():
    """K^vol computed with the cylinder axis along x, y or z agrees."""
    d = (4, 2, 1)
    v = [kt._axis_pass(d[0], d[1], d[2], 12)[0], kt._axis_pass(d[1], d[2], d[0], 12)[0],
         kt._axis_pass(d[2], d[0], d[1], 12)[0]]
    assert np.abs(v[0] - v[1]).max() < 1e-15 and np.abs(v[0] - v[2]).max() < 1e-15


@pytest.mark.parametrize("d", [(0, 0, 0), (3, 1, 2), (20, 11, 7)])
def test_lag_support_window(d):
    """Nonzero lags only where (l+1) > R_min and (l-2) < R_max (support of T)."""
    nl = 40
    vol, face = kt.offset_elements(d, nl)
    ad = np.abs(np.array(d, float))
    rmin = np.sqrt(np.sum(np.maximum(ad - 1, 0) ** 2))
    rmax = np.sqrt(np.sum((ad + 1) ** 2))
    for l in range(nl):
        inside = (l + 1 > rmin) and (l - 2 < rmax)
        if not inside:
            assert vol[l] == 0.0 and np.all(face[:, :, l] == 0.0)


def test_largest_lag_is_ell():
    """For the corner-to-corner offset of an N^3 box the last nonzero lag is
    floor(N sqrt 3) + 2 = ell (Eq. Ell)."""
    N = 8
    ell = spline.num_lags(N, N, N)
    vol, face = kt.offset_elements((N - 1, N - 1, N - 1), ell + 3)
    nz = np.nonzero(np.abs(face).sum(axis=(0, 1)) > 0)[0]
    assert nz[-1] == ell


BRUTE_OFFSETS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 1, 1), (3, 2, 1), (5, 5, 4)]


@pytest.mark.parametrize("d", BRUTE_OFFSETS)
def test_every_lag_and_component_against_cartesian_rule(d):
    """Each lag of K^vol and of all nine K^face components (off-diagonal ones included)
    against the independent Cartesian iterated rule of ``brute`` that resolves every
    shell r = k (no cylinder, arcs or tanh-sinh): equal to 1e-9 of the largest element
    at that offset (the Cartesian rule itself is converged to ~1e-12 at 16 nodes per
    piece; see the next test)."""
    from oracle import brute
    nl = 12
    vol, face = kt.offset_elements(d, nl)
    bv, bf = brute.element_lags(d, nl, n=16)
    scale = max(np.abs(vol).max(), np.abs(face).max())
    assert np.abs(vol - bv).max() < 1e-9 * scale
    for a, b in itertools.product(range(3), range(3)):
        assert np.abs(face[a, b] - bf[a, b]).max() < 1e-9 * scale, (a, b)


def test_cartesian_rule_converged():
    """The Cartesian rule at 12 and at 20 nodes per piece agrees to 1e-8 of the largest
    element (its error decays geometrically once the shells are resolved)."""
    from oracle import brute
    for d in ((1, 0, 0), (2, 1, 1)):
        v0, f0 = brute.element_lags(d, 10, n=12)
        v1, f1 = brute.element_lags(d, 10, n=20)
        scale = max(np.abs(v1).max(), np.abs(f1).max())
        assert np.abs(v0 - v1).max() < 1e-8 * scale
        assert np.abs(f0 - f1).max() < 1e-8 * scale


def test_moment_preserving_lag_error_is_caught(monkeypatch):
    """A mistake planted in the oracle that moves weight of the Lam'Lam' (xy) component
    between four neighbouring lags as eps (1, -3, 3, -1), which keeps the lag moments of
    order 0, 1, 2 and the trace (the other pins), is caught by the per-lag comparison."""
    from oracle import brute
    d, nl = (2, 1, 1), 12
    good = kt.offset_elements

    def planted(dd, nlag, *a, **k):
        vol, face = good(dd, nlag, *a, **k)
        eps = 1e-6 * np.abs(face).max()
        pat = eps * np.array([1.0, -3.0, 3.0, -1.0])
        face = face.copy()
        face[0, 1, 2:6] += pat
        face[1, 0, 2:6] += pat
        return vol, face

    monkeypatch.setattr(kt, "offset_elements", planted)
    vol, face = kt.offset_elements(d, nl)
    vol0, face0 = good(d, nl)
    l = np.arange(nl)
    for k in range(3):                 # the moment pins cannot see it
        assert abs(((l ** k) * (face[0, 1] - face0[0, 1])).sum()) < 1e-15
    bv, bf = brute.element_lags(d, nl, n=16)
    scale = max(np.abs(vol).max(), np.abs(face).max())
    assert np.abs(face[0, 1] - bf[0, 1]).max() > 1e-7 * scale


def test_rule_refinement_converged():
    """Halving the tanh-sinh step and raising the z-rule order leaves the elements
    unchanged to ~1e-13 relative."""
    for d in [(0, 0, 0), (2, 1, 0), (30, 29, 0), (103, 103, 103)]:
        nl = 186
        v0, f0 = kt.offset_elements(d, nl)
        v1, f1 = kt.offset_elements(d, nl, n_z=32, ts=kt._tanh_sinh(1.0 / 20.0, 3.6))
        assert np.abs(v0 - v1).max() < 2e-13 * np.abs(v0).max()
        assert np.abs(f0 - f1).max() < 2e-13 * np.abs(f0).max()
