"""Pins of the oracle's march (Eqs. MOTInversion, PnMOT), PDSA (Eq. Dn), excitation
(Eq. E) and the FIR taps (Eqs. FIR2-4, RegReq1)."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import excitation, kernel_table, march, pdsa
from oracle.spline import num_lags

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(N, eps, taps=None, steps=64, k_hat=(0, 0, 1), p_hat=(1, 0, 0)):
    eps_r = wl.cube(N, eps)
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    pulse = wl.pulse(N, eps, k_hat, p_hat)
    E = excitation.tested_excitation(eps_r, pulse, steps)
    taps = np.zeros(0) if taps is None else taps
    return eps_r, G, E, taps, ell


def test_march_solves_its_system(cube8_oracle):
    """sum_{l=0}^{ell} Z_l J_{n-l} = E_n for every step (the definition)."""
    o = cube8_oracle
    r = march.residual(o["G"], o["cfg"]["eps_r"], o["cfg"]["taps"], o["E"][:80], o["J"][:80])
    assert r < 1e-13


def test_march_bounded_and_decaying(cube8_oracle):
    """The pulse passes and the response rings down (no late-time growth)."""
    nrm = np.sqrt((cube8_oracle["J"] ** 2).sum(axis=(1, 2)))
    assert nrm.max() > 1.0
    assert nrm[-32:].max() < 0.05 * nrm.max()


def test_clausius_mossotti_single_voxel():
    """One voxel driven by a step: the late-time current is the static response
    3 (eps - 1)/(eps + 2) e, which follows from sum_l T = 1, sum_l K^vol = 0 and the
    self demagnetisation -1/3 (static limit of Eq. MatrixEquation)."""
    eps = 4.0
    eps_r = np.full((1, 1, 1), eps)
    ell = num_lags(1, 1, 1)
    G, _, _ = kernel_table.octant_table(1, ell + 1)
    chi = (eps - 1) / eps
    e = np.array([1.0, -0.3, 0.2])
    Nt = 400
    E = np.broadcast_to(chi * e, (Nt, 1, 3)).copy()
    J = march.march(G, eps_r, np.zeros(0), E)
    assert np.abs(J[-1, 0] - 3 * (eps - 1) / (eps + 2) * e).max() < 1e-10


def test_frequency_domain_solve_matches_transient():
    """DFT-of-transient equals a frequency-domain solve of the same discretisation:
    Z(z) J_N(z) = E_N(z) + tail(z), solved densely, on a damped and an undamped z."""
    eps_r, G, E, taps, ell = _small(3, 6.0, steps=48)
    J = march.march(G, eps_r, taps, E)
    for z in (np.exp(0.37j), 1.05 * np.exp(2.1j), -1.0 + 0j):
        x, JN = pdsa.frequency_identity_solve(G, eps_r, taps, E, J, z)
        assert np.abs(x - JN).max() < 1e-10 * np.abs(JN).max()


def test_rotation_permutes_components():
    """A cube lit along z with x polarisation is the axis-swapped (x <-> z) image of
    the same cube lit along x with z polarisation."""
    N = 3
    eps_r, G, E1, taps, _ = _small(N, 5.0, steps=40, k_hat=(0, 0, 1), p_hat=(1, 0, 0))
    _, _, E2, _, _ = _small(N, 5.0, steps=40, k_hat=(1, 0, 0), p_hat=(0, 0, 1))
    J1 = march.march(G, eps_r, taps, E1).reshape(40, N, N, N, 3)   # [n, w, v, u, b]
    J2 = march.march(G, eps_r, taps, E2).reshape(40, N, N, N, 3)
    J2s = J2.transpose(0, 3, 2, 1, 4)[..., ::-1]                      # swap x <-> z
    assert np.abs(J1 - J2s).max() < 1e-12 * np.abs(J1).max()


def test_linearity():
    eps_r, G, E, taps, _ = _small(2, 3.0, steps=30)
    rng = np.random.default_rng(3)
    E2 = rng.normal(size=E.shape)
    Ja = march.march(G, eps_r, taps, E)
    Jb = march.march(G, eps_r, taps, E2)
    Jc = march.march(G, eps_r, taps, 2.0 * E - 0.5 * E2)
    assert np.abs(Jc - (2.0 * Ja - 0.5 * Jb)).max() < 1e-12 * np.abs(Jc).max()


def test_z0_symmetrised_is_spd():
    """diag(1/chi) Z_0 is symmetric positive definite (reading R4; D_0 = Z_0 of the
    PDSA), which is what allows conjugate gradients for the per-step solve."""
    N = 4
    eps_r = wl.sphere(N, 12.0) * 0 + 12.0
    eps_r[0, 0, 0] = 3.0                       # heterogeneous chi
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, 1)
    Z0 = march.dense_Z(G, 0, eps_r, np.zeros(0))
    e = np.repeat(eps_r.reshape(-1), 3)
    A = Z0 / ((e - 1) / e)[:, None]
    assert np.abs(A - A.T).max() < 1e-15
    assert np.linalg.eigvalsh(A).min() > 0.0


def test_reciprocity_of_every_lag():
    """Reciprocity (Sec. 6: the matrices are symmetric): diag(1/chi) Z_l is symmetric
    for every lag l on a heterogeneous grid with a vacuum voxel excluded, and the
    unscaled Z_l is not (the chi factor multiplies rows), so a column-scaled assembly
    fails this test."""
    N = 3
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    rng = np.random.default_rng(9)
    eps_r = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    e = np.repeat(eps_r.reshape(-1), 3)
    chi = (e - 1) / e
    taps = wl.fir_taps("fir3", 0.05)
    for l in range(ell + 1):
        Z = march.dense_Z(G, l, eps_r, taps)
        A = Z / chi[:, None]
        scale = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-15 * scale, l
        if np.abs(Z - np.diag(np.diag(Z))).max() > 1e-6 * scale:
            assert np.abs(Z - Z.T).max() > 1e-8 * scale, l


def test_pdsa_binomials_and_fir_identity():
    """D_0 = Z_0, D_ell = sum (-1)^i Z_i, and FIR taps with sum (-1)^n delta_n = delta
    shift D_ell by exactly delta I (Eqs. Dn, Regularization, RegReq1)."""
    N = 2
    eps_r = wl.cube(N, 12.0)
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    taps = wl.fir_taps("fir3", 0.1)
    D = pdsa.pdsa_matrices(G, eps_r, np.zeros(0), ell)
    Dd = pdsa.pdsa_matrices(G, eps_r, taps, ell)
    Z = [march.dense_Z(G, l, eps_r, np.zeros(0)) for l in range(ell + 1)]
    assert np.abs(D[0] - Z[0]).max() == 0.0
    alt = sum((-1) ** i * Z[i] for i in range(ell + 1))
    assert np.abs(D[ell] - alt).max() < 1e-15
    assert np.abs(Dd[ell] - D[ell] - 0.1 * np.eye(D[0].shape[0])).max() < 1e-15
    mins = pdsa.min_eigs_symmetrised(D, eps_r)
    assert all(m > 0 for m in mins)          # a 2^3 cube is well inside the PD regime


def _pdsa_case(N, seed, n_inactive=2):
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    rng = np.random.default_rng(seed)
    eps = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    eps[0, 0, :n_inactive] = 1.0
    return ell, G, eps


def test_pdsa_circulant_embedding_pins():
    """Circulant embedding of sum_i c_i G_i on a torus P >= 2N - 1 (App. A): restricted
    to the grid it is the dense Toeplitz matrix sum_i c_i G_i built by dense_G; its
    eigenvalues (3x3 blocks of the FFT) are those of the dense circulant matrix built
    entry by entry; and min a - max eig <= lambda(A_n) <= max a - min eig for a
    heterogeneous grid with inactive voxels (Weyl + Cauchy interlacing)."""
    N = 3
    ell, G, eps = _pdsa_case(N, 11)
    taps = wl.fir_taps("fir3", 0.05)
    P = (6, 8, 6)
    Pu, Pv, Pw = P
    pw, pv, pu = np.meshgrid(np.arange(Pw), np.arange(Pv), np.arange(Pu), indexing="ij")
    tor = np.stack([pu.ravel(), pv.ravel(), pw.ravel()], axis=1)        # torus points
    on_grid = np.nonzero((tor < N).all(axis=1))[0]
    for n in (0, 3, ell):
        c = pdsa.pdsa_coefficients(ell, n)
        K = pdsa.circulant_embedding(G, c, eps.shape, P)
        d = (tor[:, None, :] - tor[None, :, :]) % np.array([Pu, Pv, Pw])
        Cd = K[:, :, d[..., 2], d[..., 1], d[..., 0]].transpose(2, 0, 3, 1).reshape(
            3 * len(tor), 3 * len(tor))
        rows = (3 * on_grid[:, None] + np.arange(3)).reshape(-1)
        T = sum(c[i] * march.dense_G(G, i, N, N, N) for i in range(n + 1))
        assert np.abs(Cd[np.ix_(rows, rows)] - T).max() <= 1e-15 * np.abs(T).max()
        ev_fft = np.sort(pdsa.circulant_symbol_eigs(K).reshape(-1))
        ev_dense = np.linalg.eigvalsh(Cd)
        assert np.abs(ev_fft - ev_dense).max() <= 1e-12 * np.abs(ev_dense).max()
        lam = np.linalg.eigvalsh(pdsa.scaled_pdsa_matrix(G, eps, taps, ell, n))
        lo, hi, smin, smax = pdsa.circulant_bounds(G, eps, taps, ell, n, P)
        assert lo <= lam.min() + 1e-12 and lam.max() <= hi + 1e-12
        assert smin == ev_fft[0] and smax == ev_fft[-1]


def test_pdsa_scaled_operator_pins():
    """A_n = diag(1/chi) D_n / C(ell, n) on the active voxels: its off-diagonal part is
    -sum_i c_i G_i and its diagonal a_m = sum_i c_i (T(i)/(eps_m - 1) + delta_i/chi_m)
    (Eq. Z); D_ell = Z(z = -1) gives a = delta / chi for the FIR taps (T(0) = T(1));
    the circulant product equals the dense product, and rounding each lag spectrum to
    float32 moves it by no more than sum_i |c_i| 2^-24 max_k ||Khat_i(k)||_F ||x||."""
    N = 4
    ell, G, eps = _pdsa_case(N, 12)
    taps = wl.fir_taps("fir3", 0.05)
    act = eps.reshape(-1) > 1.0
    e = eps.reshape(-1)[act]
    chi = (e - 1.0) / e
    P = (8, 8, 8)
    x = np.random.default_rng(3).normal(size=(N ** 3, 3))
    for n in (0, 1, 5, ell):
        A = pdsa.scaled_pdsa_matrix(G, eps, taps, ell, n)
        c = pdsa.pdsa_coefficients(ell, n)
        T = sum(c[i] * march.dense_G(G, i, N, N, N) for i in range(n + 1))
        rows = (3 * np.nonzero(act)[0][:, None] + np.arange(3)).reshape(-1)
        off = A + T[np.ix_(rows, rows)]
        a = pdsa.diagonal_of_scaled(eps, taps, ell, n)
        assert np.abs(off - np.diag(np.repeat(a, 3))).max() <= 1e-14 * np.abs(A).max()
        if n == ell:
            assert np.abs(a - 0.05 / chi).max() <= 1e-14 * np.abs(a).max()
        y = pdsa.circulant_apply(G, eps, taps, ell, n, P, x)
        yd = np.zeros_like(x)
        yd[act] = (A @ x[act].reshape(-1)).reshape(-1, 3)
        assert np.abs(y - yd).max() <= 1e-13 * np.abs(yd).max()
        y32 = pdsa.circulant_apply(G, eps, taps, ell, n, P, x, round32=True)
        bound = 0.0
        for i in range(1, n + 1):
            one = np.zeros(i + 1)
            one[i] = 1.0
            Ki = np.fft.fftn(pdsa.circulant_embedding(G, one, eps.shape, P), axes=(2, 3, 4)).real
            bound += abs(c[i]) * 2.0 ** -24 * np.sqrt((Ki ** 2).sum(axis=(0, 1))).max()
        dy = np.linalg.norm(y32 - y)
        assert dy <= bound * np.linalg.norm(x[act]) and (n == 0 or dy > 0)


def test_fir_taps_against_paper():
    """Eqs. FIR2-FIR4 as printed (FIR4 last tap per reading R7), Eq. RegReq1, and the
    magnitude (Eq. FIRmagnitude) of the 9-tap binomial member of the family in closed
    form, delta sin^8(theta / 2)."""
    rows = {}
    for line in open(os.path.join(GOLDEN, "fir_taps_paper.txt")):
        if line.strip() and not line.startswith("#"):
            parts = line.split()
            rows[parts[0]] = np.array([float(v) for v in parts[1:]])
    for k in ("fir2", "fir3", "fir4"):
        taps = wl.fir_taps(k, 1.0)
        assert np.array_equal(taps, rows[k])
        assert abs(np.sum(taps * (-1.0) ** np.arange(len(taps))) - 1.0) < 1e-15
    b = wl.fir_taps("binom9", 0.1125)                # the FIR2/FIR3 family at 9 taps
    assert abs(np.sum(b * (-1.0) ** np.arange(9)) - 0.1125) < 1e-15
    th = np.linspace(0.0, np.pi, 7)
    mag = np.abs(np.exp(-1j * np.outer(th, np.arange(9))) @ b)   # Eq. FIRmagnitude
    assert np.abs(mag - 0.1125 * np.sin(th / 2) ** 8).max() < 1e-15
    assert np.abs(b - b[::-1]).max() == 0.0
    h = wl.fir_taps("hp9", 0.1125)
    assert abs(np.sum(h * (-1.0) ** np.arange(9)) - 0.1125) < 1e-15
    assert np.abs(h - h[::-1]).max() < 1e-15          # type-I linear phase
    assert abs(h.sum()) < 1e-15                       # high-pass: no DC gain


def test_sphere_voxelisation_tie_free():
    for N in (8, 32, 104):
        c = np.arange(N) + 0.5 - N / 2.0
        r2 = c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2
        assert np.abs(r2 - (N / 2.0) ** 2).min() > 0.2
    assert int((wl.sphere(32, 12.0) > 1).sum()) == 17256


def test_excitation_quadrature_converged():
    """Eq. E voxel average with 8 and 12 point rules agree (the pulse is smooth on the
    voxel scale)."""
    cfg = wl.config("cube8")
    a = excitation.tested_excitation(cfg["eps_r"], cfg["pulse"], 4, n_first=95, npts=8)
    b = excitation.tested_excitation(cfg["eps_r"], cfg["pulse"], 4, n_first=95, npts=12)
    assert np.abs(a - b).max() < 1e-14 * np.abs(a).max()


def test_adjoint_duality():
    """For any g and E: sum_n <g_n, J_n> = sum_n <lambda_n, E_n> when Z J = E and
    Z^T lambda = g (the adjoint march solves the transposed system)."""
    from oracle import adjoint
    eps_r, G, E, taps, _ = _small(3, 7.0, steps=30)
    taps = wl.fir_taps("fir3", 0.05)
    J = march.march(G, eps_r, taps, E)
    g = np.random.default_rng(2).normal(size=J.shape)
    lam = adjoint.adjoint(G, eps_r, taps, g)
    lhs = np.sum(g * J)
    rhs = np.sum(lam * E)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_adjoint_gradient_matches_finite_differences():
    """dO/deps_m of O = sum_n <g_n, J_n(eps)> by the adjoint against central differences
    of two forward marches (E depends on eps through chi as well)."""
    from oracle import adjoint
    N = 3
    rng = np.random.default_rng(4)
    eps_r = 3.0 + 4.0 * rng.uniform(size=(N, N, N))
    taps = wl.fir_taps("fir3", 0.05)
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    pulse = wl.pulse(N, 5.0)
    steps = 30
    g = rng.normal(size=(steps, N ** 3, 3))

    def objective(eps):
        E = excitation.tested_excitation(eps, pulse, steps)
        return np.sum(g * march.march(G, eps, taps, E))

    E = excitation.tested_excitation(eps_r, pulse, steps)
    e_inc = excitation.tested_excitation(eps_r, pulse, steps, with_chi=False)
    J = march.march(G, eps_r, taps, E)
    lam = adjoint.adjoint(G, eps_r, taps, g)
    grad = adjoint.gradient_eps(G, eps_r, taps, e_inc, J, lam)
    h = 1e-5
    for m in (0, 13, 26):
        ep = eps_r.copy().reshape(-1)
        em = eps_r.copy().reshape(-1)
        ep[m] += h
        em[m] -= h
        fd = (objective(ep.reshape(eps_r.shape)) - objective(em.reshape(eps_r.shape))) / (2 * h)
        assert abs(fd - grad[m]) < 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max())


def test_response_pins():
    """Tapered DFT and the incident spectrum (Eq. Halpha): a cosine on a DFT bin gives
    N dt / 2 there and 0 on the other bins without taper; a constant series gives
    dt (n_flat + (T - 1) / 2) at f = 0 with a T-sample half-cosine taper; |e^i(f)|
    equals the FFT of the densely sampled pulse."""
    from oracle import response
    N, dt = 240, 0.5
    t = dt * np.arange(1, N + 1)
    k0 = 17
    J = np.cos(2 * np.pi * k0 / (N * dt) * t)[:, None]
    f = np.arange(0, N // 2) / (N * dt)
    jf = np.abs(response.tapered_dft(J, dt, 0.0, f))[:, 0]
    assert abs(jf[k0] - N * dt / 2) < 1e-10
    assert np.delete(jf, k0).max() < 1e-10
    w = response.taper_weights(N, 0.2)
    T = int(np.floor(0.2 * N))
    assert abs(w.sum() - ((N - T) + (T - 1) / 2)) < 1e-12
    assert w[N - T - 1] == 1.0 and abs(w[-1]) < 1e-15
    one = np.ones((N, 1))
    assert abs(response.tapered_dft(one, dt, 0.2, [0.0])[0, 0] - dt * w.sum()) < 1e-12
    fc, st = 0.03, 20.0
    h = 0.25
    ts = h * np.arange(-4000, 4000)
    x = np.sin(2 * np.pi * fc * ts) * np.exp(-ts ** 2 / (2 * st ** 2))
    X = h * np.abs(np.fft.fft(x))
    fr = np.fft.fftfreq(ts.size, h)
    sel = (fr >= 0) & (fr < 0.1)
    ref = response.incident_amplitude(fr[sel], fc, st)
    assert np.abs(X[sel] - ref).max() < 1e-10 * ref.max()


def test_pdsa_smallest_eigenvalue_is_at_n_ell_and_falls_with_N():
    """PDSA on eps_r = 12 cubes (Sec. 5.1): over n = 0..ell the smallest eigenvalue of
    A_n = diag(1/chi) D_n / C(ell, n) is the one of D_ell, and lambda_min(A_ell) is
    positive and falls as the cube grows (N = 3, 4, 6), the trend behind the paper's
    loss of definiteness at larger N."""
    mins = []
    for N in (3, 4, 6):
        ell = num_lags(N, N, N)
        G, _, _ = kernel_table.octant_table(N, ell + 1)
        eps = wl.cube(N, 12.0)
        lam = [np.linalg.eigvalsh(pdsa.scaled_pdsa_matrix(G, eps, np.zeros(0), ell, n)).min()
               for n in (range(ell + 1) if N < 6 else (0, ell // 2, ell - 1, ell))]
        assert int(np.argmin(lam)) == len(lam) - 1
        assert lam[-1] > 0.0
        mins.append(lam[-1])
    assert mins[0] > mins[1] > mins[2]


def test_probe_field_pins():
    """Probe field of the adjoint workload's objective (reading R18): probes placed on
    voxels of the grid itself reproduce the dense history rows sum_l dense_G(l) J_{n-l}
    (an independent assembly from the octant table); Fibonacci probes sit at the
    requested distance, outside the grid."""
    from oracle import probes as pr
    N = 3
    ell = num_lags(N, N, N)
    G, _, _ = kernel_table.octant_table(N, ell + 1)
    rng = np.random.default_rng(17)
    J = rng.normal(size=(6, N ** 3, 3))
    inside = np.array([(0, 0, 0), (2, 1, 0), (1, 2, 2)])
    Gp = pr.probe_elements(inside, (N, N, N), ell + 1)
    E = pr.probe_field(Gp, J)
    dense = [march.dense_G(G, l, N, N, N) for l in range(ell + 1)]
    for n in range(J.shape[0]):
        ref = sum(dense[l] @ J[n - l].reshape(-1) for l in range(min(ell + 1, n + 1)))
        for k, (u, v, w) in enumerate(inside):
            m = u + N * (v + N * w)
            assert np.abs(E[n, k] - ref[3 * m:3 * m + 3]).max() <= 1e-14 * np.abs(ref).max()
    P = pr.fibonacci_probes(8, 64)
    c = P + 0.5 - 4.0
    r = np.linalg.norm(c, axis=1)
    assert len(P) >= 60 and np.all(np.abs(r - 16.0) <= 0.87)
    assert np.all(((P < 0) | (P > 7)).any(axis=1))    # every probe outside the 8^3 grid


def test_probe_objective_gradient_against_differences():
    """The transposed probe operator gives dO/dJ of the gated probe energy: central
    differences in a few entries of J (O is quadratic in J, so they are exact up to
    rounding)."""
    from oracle import probes as pr
    N = 2
    nlag = 12
    P = np.array([(5, 1, 0), (-3, 0, 2), (1, 6, -2)])
    Gp = pr.probe_elements(P, (N, N, N), nlag)
    rng = np.random.default_rng(23)
    J = rng.normal(size=(10, N ** 3, 3))
    first = 4
    E = pr.probe_field(Gp, J)
    g = pr.probe_objective_gradient(Gp, E, first)
    h = 1e-3
    for (k, m, b) in [(0, 0, 0), (3, 5, 2), (7, 2, 1), (9, 7, 0)]:
        Jp = J.copy(); Jp[k, m, b] += h
        Jm = J.copy(); Jm[k, m, b] -= h
        fd = (pr.probe_objective(pr.probe_field(Gp, Jp), first)
              - pr.probe_objective(pr.probe_field(Gp, Jm), first)) / (2 * h)
        assert abs(fd - g[k, m, b]) <= 1e-8 * max(1.0, abs(g).max()), (k, m, b, fd, g[k, m, b])
