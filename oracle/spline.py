"""Quadratic temporal B-spline basis T (Sec. 2.3).

The paper expands time with a "quadratic spline" T_n'(t) = T(t - n' dt) whose
definition it defers to its companion paper.  Reading used here (R1): T is the
uniform quadratic B-spline with support (-dt, 2 dt):

    tau/dt in [-1, 0]:  (1 + tau)^2 / 2
    tau/dt in [ 0, 1]:  (1 + 2 tau - 2 tau^2) / 2
    tau/dt in [ 1, 2]:  (2 - tau)^2 / 2

With this support and Dirac testing at t = n dt, the largest lag with a nonzero
interaction is floor(D / (c dt)) + 2 for a box of diagonal D, which is exactly
Eq. Ell; the operator is causal, and Z_0 is a 27-point stencil when c dt = h
(Sec. 5.2).  Units: dt = 1 throughout the oracle.
"""
import numpy as np


def T(tau):
    """T(tau) for tau in units of dt (reading R1 of Sec. 2.3)."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.zeros_like(tau)
    m = (tau > -1.0) & (tau <= 0.0)
    out[m] = (1.0 + tau[m]) ** 2 / 2.0
    m = (tau > 0.0) & (tau <= 1.0)
    out[m] = (1.0 + 2.0 * tau[m] - 2.0 * tau[m] ** 2) / 2.0
    m = (tau > 1.0) & (tau < 2.0)
    out[m] = (2.0 - tau[m]) ** 2 / 2.0
    return out


def T2(tau):
    """Second time derivative T''(tau) (per dt^2): +1, -2, +1 on the three pieces."""
    tau = np.asarray(tau, dtype=np.float64)
    out = np.zeros_like(tau)
    out[(tau > -1.0) & (tau < 0.0)] = 1.0
    out[(tau > 0.0) & (tau < 1.0)] = -2.0
    out[(tau > 1.0) & (tau < 2.0)] = 1.0
    return out


def T_at_lag(l):
    """T(l dt) at integer lag l: 1/2 for l = 0, 1 and 0 otherwise."""
    return 0.5 if l in (0, 1) else 0.0


def num_lags(U, V, W, hx=1.0, hy=1.0, hz=1.0, c_dt=1.0):
    """Eq. Ell: ell = floor(sqrt((U hx)^2 + (V hy)^2 + (W hz)^2) / (c dt)) + 2."""
    D = np.sqrt((U * hx) ** 2 + (V * hy) ** 2 + (W * hz) ** 2)
    return int(np.floor(D / c_dt)) + 2
