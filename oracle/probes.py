"""Scattered field at probes outside the grid: the objective of the adjoint workload.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reading R18.  The objective sums the squared scattered field at probe points around
the scatterer.  Here each probe is a virtual voxel on the grid's lattice (the point
rounded to the nearest voxel centre) and its field is the voxel-averaged one, the
tested field of Eq. E:

    E^s_p(t_n) = sum_{l>=0} sum_{m'} G_l(r_p - r_m') J_{n-l, m'}            (Eq. Z),

with the same elements G_l(d) = K^face_l(d) - delta_ab K^vol_l(d) as the march, for
offsets beyond the grid.  The probe voxel lies in vacuum, so no local term enters.
"""
import itertools

import numpy as np

from .kernel_table import offset_elements


def fibonacci_probes(N, n_probes=64, radius_factor=2.0, seed=240703324):
    """The probe voxels of the adjoint workload (seeded input; see
    ``workloads.fibonacci_probes``)."""
    import workloads
    return workloads.fibonacci_probes(N, n_probes, radius_factor, seed)


def _elements_at(d, nlag, cache):
    """G_l^{ab}(d), l < nlag, for one integer offset d = (dx, dy, dz), from the
    element quadrature of the sorted |d| with the axis permutation and parity signs
    (diagonal even in every d_i, (a, b) odd in d_a and d_b)."""
    ad = tuple(abs(int(v)) for v in d)
    key = tuple(sorted(ad, reverse=True))
    if key not in cache:
        cache[key] = offset_elements(key, nlag)
    vol, face = cache[key]
    for perm in itertools.permutations(range(3)):
        if all(ad[i] == key[perm[i]] for i in range(3)):
            break
    G = np.zeros((nlag, 3, 3))
    for a in range(3):
        for b in range(3):
            g = face[perm[a], perm[b]] - (vol if a == b else 0.0)
            if a != b:
                g = g * np.sign(d[a]) * np.sign(d[b])
            G[:, a, b] = g
    return G


def probe_elements(probes, shape, nlag):
    """Gp[p, m, l, a, b] = G_l^{ab}(r_p - r_m) for probes (lattice indices u, v, w) and
    the voxels m = u + U (v + V w) of a [W][V][U] grid."""
    W, V, U = shape
    cache = {}
    out = np.zeros((len(probes), U * V * W, nlag, 3, 3))
    for pi, p in enumerate(probes):
        for w in range(W):
            for v in range(V):
                for u in range(U):
                    m = u + U * (v + V * w)
                    out[pi, m] = _elements_at((p[0] - u, p[1] - v, p[2] - w), nlag, cache)
    return out


def probe_field(Gp, J):
    """E[n, p, a] = sum_{l} sum_{m} Gp[p, m, l, a, b] J[n - l, m, b] for J[n, m, b]
    (n = 0 is time step 1; earlier currents are zero)."""
    Nt = J.shape[0]
    nlag = Gp.shape[2]
    E = np.zeros((Nt, Gp.shape[0], 3))
    for n in range(Nt):
        for l in range(min(nlag, n + 1)):
            E[n] += np.einsum("pmab,mb->pa", Gp[:, :, l], J[n - l])
    return E


def probe_objective(E, first):
    """O = sum_{n >= first} sum_p |E^s_p(t_n)|^2 (first: 0-based step index)."""
    return float((E[first:] ** 2).sum())


def probe_objective_gradient(Gp, E, first):
    """dO/dJ[k, m, b] = 2 sum_{n >= first} sum_p sum_a Gp[p, m, n - k, a, b] E[n, p, a]:
    the transposed probe operator applied to the gated field, the source term of the
    adjoint march for this objective."""
    Nt = E.shape[0]
    nlag = Gp.shape[2]
    M = Gp.shape[1]
    g = np.zeros((Nt, M, 3))
    for n in range(first, Nt):
        for l in range(min(nlag, n + 1)):
            g[n - l] += 2.0 * np.einsum("pmab,pa->mb", Gp[:, :, l], E[n])
    return g
