"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the element tables of both sides are independent FP64 quadratures
(~1e-14 of the largest element each), so tables agree to 1e-12 of the largest
element; the FP64 march must match the oracle to a relative L2 of 1e-10 over all
J_n; the FP32-history march must stay within 1e-5 relative L2 of the FP64 march.
"""
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mot():
    from paper_2407_03323_gb300 import build, mot as m
    if not os.path.exists(m.LIB_PATH):
        build.build()
    m.load_library()
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_table_matches_oracle_cube8(mot, cube8_oracle):
    o = cube8_oracle
    with mot.Context(o["cfg"]["eps_r"]) as ctx:
        assert ctx.ell == o["ell"]
        g = ctx.table(0, ctx.ell + 1)
    G = o["G"]                                   # [l][c][dz][dy][dx]
    assert g.shape == G.shape
    assert np.abs(g - G).max() < 1e-12 * np.abs(G).max()


def test_table_matches_oracle_sampled_offsets(mot):
    """A 40^3 grid: the table at offsets up to 39 against the oracle's elements."""
    from oracle import kernel_table as kt
    N = 40
    with mot.Context(wl.cube(N, 2.0), precision="fp32_history") as ctx:
        ell = ctx.ell
        g = ctx.table(0, ell + 1)
    rng = np.random.default_rng(7)
    offs = [(0, 0, 0), (1, 0, 0), (39, 39, 39), (39, 0, 0), (17, 3, 29)]
    offs += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(12)]
    for d in offs:
        vol, face = kt.offset_elements(d, ell + 1)
        comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        for c, (a, b) in enumerate(comps):
            ref = face[a, b] - (vol if a == b else 0.0)
            got = g[:, c, d[2], d[1], d[0]]
            assert np.abs(got - ref).max() < 1e-12 * max(np.abs(ref).max(), 1e-6), (d, c)


def test_spectrum_matches_direct_dft(mot, cube8_oracle):
    """Ghat_l(k) = sum_d G_l(d) exp(-2 pi i k.d/P) (App. A) at every octant bin, with
    the oracle's table and the plain definition of the DFT."""
    from oracle.march import g_block
    o = cube8_oracle
    N = 8
    with mot.Context(o["cfg"]["eps_r"]) as ctx:
        P = ctx.P[0]
        for l in (1, 5, ctx.ell):
            S = ctx.spectrum(l)                  # [6][Hw][Hv][Hu]
            r = np.arange(-(N - 1), N)
            dz, dy, dx = np.meshgrid(r, r, r, indexing="ij")
            d = np.stack([dx, dy, dz], axis=-1)
            B = g_block(o["G"], l, d)            # [.., 3, 3]
            H = P // 2 + 1
            k = np.arange(H)
            ex = np.exp(-2j * np.pi * np.outer(k, r) / P)   # [k, d]
            comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
            for c, (a, b) in enumerate(comps):
                ref = np.einsum("zyx,az,by,cx->abc", B[..., a, b], ex, ex, ex)
                assert np.abs(ref.imag).max() < 1e-12
                assert np.abs(S[c] - ref.real).max() < 1e-11 * np.abs(ref).max()


def test_excitation_matches_oracle(mot):
    from oracle import excitation
    cfg = wl.config("sphere12")
    p = cfg["pulse"]
    with mot.Context(cfg["eps_r"]) as ctx:
        E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"], 70, 12)
    ref = excitation.tested_excitation(cfg["eps_r"], p, 12, n_first=70)
    assert np.abs(E - ref).max() < 1e-13 * np.abs(ref).max()


def test_excitation_long_call_oblique(mot):
    """One call of 12,000 steps (several tables of the interpolated voxel average) with an
    oblique wave and a short pulse, sampled at its start, middle and end against the
    oracle's tensor rule."""
    from oracle import excitation
    eps = wl.cube(10, 6.0)
    p = {"k_hat": np.array([0.48, -0.6, 0.64]), "p_hat": np.array([0.8, 0.6, 0.0]),
         "f_c": 0.11, "sigma_t": 5.0}
    n = 12000
    with mot.Context(eps) as ctx:
        for t0 in (40.0, 6050.0, 11990.0):
            q = dict(p, t0=t0)
            E = ctx.plane_wave(q["k_hat"], q["p_hat"], q["f_c"], q["sigma_t"], t0, 1, n)
            for a in (0, 6000, n - 30):
                ref = excitation.tested_excitation(eps, q, 30, n_first=a + 1)
                scale = max(np.abs(ref).max(), 1e-300)
                if scale > 1e-12:
                    assert np.abs(E[a:a + 30] - ref).max() < 1e-13 * scale, (t0, a)


@pytest.mark.parametrize("precision", ["fp64", "fp32_history"])
def test_history_matches_direct_sum(mot, cube8_oracle, precision):
    """P_{n-1} = sum_l Z_l J_{n-l} through the FFT / ring / MAC path equals the
    oracle's direct space-time sum (Eq. PnMOT) on random histories."""
    from oracle import march
    o = cube8_oracle
    eps = o["cfg"]["eps_r"].copy()
    eps[2:5, 1:7, 3] = 9.0                      # heterogeneous chi
    taps = wl.fir_taps("hp9", 0.05)
    rng = np.random.default_rng(11)
    ell = o["ell"]
    M = eps.size
    Jh = rng.normal(size=(ell, M, 3))
    with mot.Context(eps, taps, precision=precision) as ctx:
        P = ctx.eval_history(Jh)
    ref = march.history_at(o["G"], eps, taps, Jh, list(range(M)))
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert rel_l2(P, ref) < tol


def test_history_sparse_sources_32(mot):
    """32^3 grid (P = 64): a history supported on a few source voxels, compared at
    sampled test voxels with the oracle's direct sum over those sources."""
    from oracle import kernel_table as kt
    from oracle.march import offsets_and_index
    from oracle.spline import T_at_lag
    N = 32
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("hp9", 1e-7 * N ** 3)
    rng = np.random.default_rng(5)
    with mot.Context(eps, taps) as ctx:
        ell = ctx.ell
        M = eps.size
        active = np.nonzero(eps.reshape(-1) > 1)[0]
        src = rng.choice(active, 6, replace=False)
        Jh = np.zeros((ell, M, 3))
        Jh[:, src, :] = rng.normal(size=(ell, len(src), 3))
        P = ctx.eval_history(Jh)
    idx = offsets_and_index(N, N, N)
    e = eps.reshape(-1)
    chi = (e - 1) / e
    tests = list(rng.choice(active, 10, replace=False)) + list(src[:2])
    cache = {}
    for m in tests:
        acc = np.zeros(3)
        for s in src:
            d = idx[m] - idx[s]
            key = tuple(int(v) for v in np.abs(d))
            if key not in cache:
                cache[key] = kt.offset_elements(key, ell + 1)
            vol, face = cache[key]
            sg = np.sign(d)
            G = face.copy()
            for a in range(3):
                for b in range(3):
                    if a != b:
                        G[a, b] = G[a, b] * sg[a] * sg[b]
                G[a, a] = G[a, a] - vol
            for l in range(1, ell + 1):
                acc -= chi[m] * G[:, :, l] @ Jh[l - 1, s]
        for l in range(1, ell + 1):
            acc += (T_at_lag(l) / e[m] + (taps[l] if l < len(taps) else 0.0)) * Jh[l - 1, m]
        assert np.abs(P[m] - acc).max() < 1e-11 * max(np.abs(acc).max(), 1e-3)


def test_march_cube8_fp64_matches_oracle(mot, cube8_oracle):
    o = cube8_oracle
    with mot.Context(o["cfg"]["eps_r"], o["cfg"]["taps"]) as ctx:
        ctx.set_excitation(o["E"])
        J = ctx.march(o["E"].shape[0])
        info = ctx.info()
    assert info["n_done"] == o["E"].shape[0]
    assert rel_l2(J, o["J"]) < 1e-10


def test_march_cube8_fp32_history_close_to_fp64(mot, cube8_oracle):
    o = cube8_oracle
    with mot.Context(o["cfg"]["eps_r"], o["cfg"]["taps"], precision="fp32_history") as ctx:
        ctx.set_excitation(o["E"])
        J = ctx.march(o["E"].shape[0])
    assert rel_l2(J, o["J"]) < 1e-5


def test_march_fir_sphere_matches_oracle(mot):
    """Sphere eps_r = 12 in 8^3 with the 9-tap linear-phase high-pass FIR (delta = 0.05),
    excitation computed on each side independently."""
    from oracle import excitation, kernel_table, march
    from oracle.spline import num_lags
    N = 8
    eps = wl.sphere(N, 12.0)
    taps = wl.fir_taps("hp9", 0.05)
    p = wl.pulse(N, 12.0, k_hat=(1.0, 2.0, 2.0), p_hat=(0.0, 1.0, -1.0))
    steps = 160
    G, _, _ = kernel_table.octant_table(N, num_lags(N, N, N) + 1)
    E = excitation.tested_excitation(eps, p, steps)
    Jref = march.march(G, eps, taps, E)
    with mot.Context(eps, taps) as ctx:
        Eg = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"], 1, steps)
        ctx.set_excitation(Eg)
        J = ctx.march(steps)
    assert rel_l2(J, Jref) < 1e-10


def test_march_in_chunks_equals_one_call(mot, cube8_oracle):
    o = cube8_oracle
    E = o["E"][:96]
    with mot.Context(o["cfg"]["eps_r"]) as ctx:
        ctx.set_excitation(E)
        J1 = ctx.march(96)
    with mot.Context(o["cfg"]["eps_r"]) as ctx:
        parts = []
        for a in range(0, 96, 32):
            ctx.set_excitation(E[a:a + 32])
            parts.append(ctx.march(32))
        J2 = np.concatenate(parts)
    assert np.array_equal(J1, J2)


# ---------------------------------------------------------------- blocked temporal scheme

@pytest.mark.parametrize("block", [2, 4, 8])
def test_march_cube8_blocked_matches_oracle(mot, cube8_oracle, block):
    """Lags >= B through block Toeplitz products with temporal FFTs (Secs. 4-5) give
    the oracle's march (8^3: ell = 15, levels up to S = 8)."""
    o = cube8_oracle
    with mot.Context(o["cfg"]["eps_r"], o["cfg"]["taps"], scheme="blocked", block=block) as ctx:
        ctx.set_excitation(o["E"])
        J = ctx.march(o["E"].shape[0])
    assert rel_l2(J, o["J"]) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32_history"])
def test_history_blocked_matches_direct_sum(mot, cube8_oracle, precision):
    from oracle import march
    o = cube8_oracle
    eps = o["cfg"]["eps_r"].copy()
    eps[1:6, 2:4, 0:5] = 7.0
    taps = wl.fir_taps("fir3", 0.1)
    rng = np.random.default_rng(13)
    ell = o["ell"]
    M = eps.size
    Jh = rng.normal(size=(ell, M, 3))
    with mot.Context(eps, taps, precision=precision, scheme="blocked", block=2) as ctx:
        P = ctx.eval_history(Jh)
    ref = march.history_at(o["G"], eps, taps, Jh, list(range(M)))
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert rel_l2(P, ref) < tol


def test_blocked_equals_direct_sphere32(mot):
    """32^3 sphere with the 9-tap FIR, 200 steps: blocked (B = 8, levels 8..32) and
    direct march agree to rounding in FP64 and to 1e-6 in FP32-history."""
    cfg = wl.config("sphere32")
    eps, taps, p = cfg["eps_r"], cfg["taps"], cfg["pulse"]
    steps = 200
    out = {}
    for scheme, prec in (("direct", "fp64"), ("blocked", "fp64"), ("blocked", "fp32_history")):
        with mot.Context(eps, taps, precision=prec, scheme=scheme, block=8) as ctx:
            E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 150, 1,
                               steps)
            ctx.set_excitation(E)
            out[(scheme, prec)] = ctx.march(steps)
    ref = out[("direct", "fp64")]
    assert np.linalg.norm(ref) > 0
    assert rel_l2(out[("blocked", "fp64")], ref) < 1e-12
    assert rel_l2(out[("blocked", "fp32_history")], ref) < 1e-5


def test_long_grid_levels_to_128(mot):
    """A 150 x 6 x 5 voxel grid (ell = 152) reaches every far level up to S = 128, whose
    length-256 temporal lines are split over 8 threads: the GPU table at sampled
    offsets against the oracle's elements; the blocked history (B = 4, doubling levels
    4..128, or the last level fitted to ell: 32 lags from lag 128) against the direct
    sum for a random history of ell steps; and a 300-step blocked march against the
    direct march (FP64 to rounding, FP32-history to 1e-5)."""
    from oracle import kernel_table as kt
    rng = np.random.default_rng(31)
    eps = 2.0 + 10.0 * rng.uniform(size=(5, 6, 150))
    eps[2, 3, 40:44] = 1.0
    taps = wl.fir_taps("hp9", 1e-3)
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    with mot.Context(eps, taps) as ctx:
        ell = ctx.ell
        assert ell >= 129
        g = ctx.table(0, ell + 1)
    for d in [(149, 5, 4), (0, 5, 0), (77, 2, 3), (149, 0, 0), (128, 1, 4)]:
        vol, face = kt.offset_elements(d, ell + 1)
        refs = [face[a, b] - (vol if a == b else 0.0) for a, b in comps]
        scale = max(np.abs(r).max() for r in refs)   # quadrature error ~ largest element
        for c, ref in enumerate(refs):
            got = g[:, c, d[2], d[1], d[0]]
            assert np.abs(got - ref).max() < 1e-12 * scale, (d, c)

    Jh = rng.normal(size=(ell, eps.size, 3))
    P = {}
    blocked = ("blocked", "blocked_doubling")
    runs = [("direct", "fp64")] + [(b, pr) for b in blocked for pr in ("fp64", "fp32_history")]
    for scheme, prec in runs:
        with mot.Context(eps, taps, precision=prec, scheme=scheme, block=4) as ctx:
            if scheme == "blocked_doubling":
                assert ctx.levels == [4, 8, 16, 32, 64, 128]
            elif scheme == "blocked":
                assert ctx.levels == [4, 8, 16, 32, 64, 32]
                assert ctx.level_lags == [4, 8, 16, 32, 64, 128]
            P[(scheme, prec)] = ctx.eval_history(Jh)
    ref = P[("direct", "fp64")]
    for b in blocked:
        assert rel_l2(P[(b, "fp64")], ref) < 1e-12, b
        assert rel_l2(P[(b, "fp32_history")], ref) < 5e-6, b

    p = wl.pulse(0, 6.0, k_hat=(1.0, 0.0, 0.0), p_hat=(0.0, 1.0, 0.0))
    steps = 300
    out = {}
    for scheme, prec in runs:
        with mot.Context(eps, taps, precision=prec, scheme=scheme, block=4) as ctx:
            E = ctx.plane_wave(p["k_hat"], p["p_hat"], p["f_c"], p["sigma_t"], p["t0"] - 60, 1,
                               steps)
            ctx.set_excitation(E)
            out[(scheme, prec)] = ctx.march(steps)
    ref = out[("direct", "fp64")]
    assert np.linalg.norm(ref[-1]) > 1e-3 * np.abs(ref).max()
    for b in blocked:
        assert rel_l2(out[(b, "fp64")], ref) < 1e-12, b
        assert rel_l2(out[(b, "fp32_history")], ref) < 1e-5, b


def test_long_axis_through_every_pass_kernel(mot):
    """One heterogeneous problem with a 104-voxel axis (padded length 210) marched with
    that axis along z, y and x: the strided passes (z, y) and the real-to-complex pass
    (x) are different kernels, so the three marches agree only if each is right
    (components and axes permuted back; FP64, direct scheme)."""
    rng = np.random.default_rng(12)
    base = 2.0 + 8.0 * rng.uniform(size=(104, 4, 5))        # [w][v][u], long axis w
    taps = wl.fir_taps("fir3", 1e-3)
    p = wl.pulse(0, 6.0, k_hat=(0.3, 0.5, 0.81), p_hat=(0.2, -0.9, 0.3))
    k = np.asarray(p["k_hat"]); pp = np.asarray(p["p_hat"])
    steps = 60
    # axis permutations of (x, y, z) = (u, v, w): the grid axes [w][v][u] move with them
    cases = {"z": ((0, 1, 2), base),                          # identity
             "y": ((0, 2, 1), base.transpose(1, 0, 2)),       # swap y <-> z: [v][w][u] -> long v
             "x": ((2, 1, 0), base.transpose(2, 1, 0))}       # swap x <-> z: long u
    out = {}
    for name, (perm, eps) in cases.items():
        kk, pq = k[list(perm)], pp[list(perm)]
        with mot.Context(eps, taps) as ctx:
            assert 210 in ctx.P
            E = ctx.plane_wave(kk, pq, p["f_c"], p["sigma_t"], p["t0"] - 60, 1, steps)
            ctx.set_excitation(E)
            J = ctx.march(steps).reshape(steps, *eps.shape, 3)
        out[name] = J
    ref = out["z"]
    y = out["y"].transpose(0, 2, 1, 3, 4)[..., [0, 2, 1]]     # back to [w][v][u], comps x z y
    x = out["x"].transpose(0, 3, 2, 1, 4)[..., [2, 1, 0]]
    nrm = np.linalg.norm(ref)
    assert nrm > 0
    assert np.linalg.norm(y - ref) < 1e-12 * nrm
    assert np.linalg.norm(x - ref) < 1e-12 * nrm
