"""Seeded synthetic inputs for MOT-JVIE runs.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds no
step of the method's arithmetic (no element integrals, no excitation testing, no
marching): only the geometry (relative permittivity per voxel, sampled at voxel
centres as the voxelisation of Sec. 2.2 prescribes), the parameters of the
incident pulse, and the FIR regularisation tap values, all as plain numbers.

Units: voxel edge h = 1, c0 = 1, dt = h / c0 = 1 (every run of the paper has
c0 dt = dx = dy = dz).
"""
import math
import numpy as np

MASTER_SEED = 240703323


# ---------------------------------------------------------------- geometry

def voxel_centres(N):
    """Voxel centres (u - 1/2, v - 1/2, w - 1/2) for u, v, w = 1..N (Sec. 2.2)."""
    c = np.arange(N, dtype=np.float64) + 0.5
    return c


def cube(N, eps):
    """Homogeneous dielectric cube filling the N^3 box; eps_r[w, v, u]."""
    return np.full((N, N, N), float(eps))


def sphere(N, eps):
    """Sphere of radius N/2 centred in the N^3 box, eps_r sampled at voxel centres
    (Sec. 2.2); eps_r = 1 outside.  No centre lies on the surface: the sum of
    (i + 1/2 - N/2)^2 over three axes is never equal to (N/2)^2."""
    c = voxel_centres(N) - N / 2.0
    r2 = c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2
    return np.where(r2 < (N / 2.0) ** 2, float(eps), 1.0)


def smoothed_noise(N, seed=MASTER_SEED + 1, sigma=2.0):
    """Seeded uniform noise blurred by a periodic Gaussian (sigma in voxels), rescaled
    to [0, 1]."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(size=(N, N, N))
    k = np.fft.fftfreq(N)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (k[None, None, :] ** 2 + k[None, :, None] ** 2
                                               + k[:, None, None] ** 2))
    y = np.real(np.fft.ifftn(np.fft.fftn(x) * g))
    return (y - y.min()) / (y.max() - y.min())


def heterogeneous_block(N, seed=MASTER_SEED + 1):
    """eps_r = 1 + 11 * smoothed seeded noise in [0, 1]."""
    return 1.0 + 11.0 * smoothed_noise(N, seed)


# ---------------------------------------------------------------- incident pulse

def pulse(N, eps_for_fc, k_hat=(0.0, 0.0, 1.0), p_hat=(1.0, 0.0, 0.0), frac_bw=0.5):
    """Parameters of the modulated Gaussian plane wave
        E^i(r, t) = p_hat sin(2 pi f_c tau) exp(-tau^2 / (2 sigma_t^2)),
        tau = t - t0 - r . k_hat / c0.
    f_c gives 10 voxels per wavelength inside eps_for_fc; the amplitude spectrum has
    a FWHM of frac_bw * f_c; t0 = 6 sigma_t + max over the box of r . k_hat."""
    k = np.asarray(k_hat, float)
    k = k / np.linalg.norm(k)
    p = np.asarray(p_hat, float)
    p = p - np.dot(p, k) * k
    p = p / np.linalg.norm(p)
    fc = 1.0 / (10.0 * math.sqrt(eps_for_fc))
    sigma_f = frac_bw * fc / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    sigma_t = 1.0 / (2.0 * math.pi * sigma_f)
    corners = np.array([[i, j, l] for i in (0, N) for j in (0, N) for l in (0, N)], float)
    t0 = 6.0 * sigma_t + float(np.max(corners @ k))
    return {"k_hat": k, "p_hat": p, "f_c": fc, "sigma_t": sigma_t, "t0": t0}


def fibonacci_probes(N, n_probes=64, radius_factor=2.0, seed=MASTER_SEED + 1):
    """Lattice indices (u, v, w) of the probes of the adjoint workload: n_probes points
    of a Fibonacci lattice on the sphere of radius radius_factor * N about the centre of
    an N^3 grid, turned by a seeded random rotation, each rounded down to the voxel that
    contains it; duplicates after rounding are removed (first occurrence kept)."""
    i = np.arange(n_probes) + 0.5
    z = 1.0 - 2.0 * i / n_probes
    phi = np.pi * (1.0 + 5.0 ** 0.5) * i
    s = np.sqrt(1.0 - z * z)
    pts = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    pts = pts @ q.T * (radius_factor * N)
    idx = np.floor(pts + N / 2.0).astype(int)
    out = []
    for p in idx:
        t = tuple(int(v) for v in p)
        if t not in out:
            out.append(t)
    return np.array(out)


def random_directions(n, seed):
    """n seeded propagation directions uniform on S^2, each with a random orthogonal
    polarisation."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        p = rng.normal(size=3)
        p -= np.dot(p, k) * k
        p /= np.linalg.norm(p)
        out.append((k, p))
    return out


def batched_instances(n_instances=24, n_rhs=8, seed=MASTER_SEED, side_range=(16, 48)):
    """Uneven batch of scatterers: sides uniform on side_range, a sphere or a cube
    with probability 1/2, eps_r uniform on [2, 30], n_rhs plane waves per scatterer
    (directions uniform on S^2, random orthogonal polarisation), FIR3 with
    delta = 1e-7 M.  All draws from numpy.random.default_rng(seed) in that order."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        N = int(rng.integers(side_range[0], side_range[1] + 1))
        is_sphere = bool(rng.integers(0, 2))
        eps = float(rng.uniform(2.0, 30.0))
        geom = sphere(N, eps) if is_sphere else cube(N, eps)
        waves = [pulse(N, eps, k_hat=k, p_hat=pp)
                 for k, pp in random_directions(n_rhs, int(rng.integers(0, 2 ** 31)))]
        out.append({"N": N, "shape": "sphere" if is_sphere else "cube", "eps": eps,
                    "eps_r": geom, "taps": fir_taps("fir3", 1e-7 * N ** 3), "waves": waves})
    return out


# ---------------------------------------------------------------- FIR taps

def fir_taps(kind, delta=0.0):
    """Regularisation taps delta_0..delta_{L-1} added as Z_n + delta_n I (Sec. 6.1).

    'none'       no regularisation
    'fir2/3/4'   the paper's two-, three- and four-step filters (Eqs. FIR2-FIR4); the
                 last FIR4 tap is taken as -delta/8 so that sum (-1)^n delta_n = delta
                 (Eq. RegReq1) holds
    'hp9'        9-tap type-I linear-phase high-pass, windowed sinc with a Hamming
                 window and cutoff 0.05 of the sampling rate, h = unit impulse at
                 n = 4 minus the low-pass, scaled so sum (-1)^n delta_n = delta.
    'binom9'     9-tap linear-phase high-pass of the family of FIR2 and FIR3,
                 delta / 2^8 (1 - z^-1)^8: meets sum (-1)^n delta_n = delta and has the
                 smallest magnitude near theta = 0 (delta sin^8(theta / 2)).
    The two 9-tap filters are kept for experiments; with delta = 1e-7 M they leave
    the eps_r = 12 sphere marches unstable (hp9 from 32^3, binom9 at 104^3), while
    FIR3 keeps them bounded, so the named workloads use FIR3.
    """
    if kind == "none":
        return np.zeros(0)
    if kind == "fir2":
        return np.array([0.5, -0.5]) * delta
    if kind == "fir3":
        return np.array([0.25, -0.5, 0.25]) * delta
    if kind == "fir4":
        return np.array([1.0, -3.0, 3.0, -1.0]) / 8.0 * delta
    if kind == "binom9":
        return np.array([math.comb(8, n) * (-1.0) ** n for n in range(9)]) / 256.0 * delta
    if kind == "hp9":
        n = np.arange(9) - 4.0
        fc = 0.05
        lp = 2.0 * fc * np.sinc(2.0 * fc * n)
        win = 0.54 - 0.46 * np.cos(2.0 * math.pi * np.arange(9) / 8.0)
        lp = lp * win
        lp = lp / lp.sum()
        hp = -lp
        hp[4] += 1.0
        alt = np.sum(hp * (-1.0) ** np.arange(9))
        return hp * (delta / alt)
    raise ValueError(kind)


# ---------------------------------------------------------------- run configs

def config(name):
    """Named workloads (sizes and parameters only)."""
    if name == "cube8":
        N = 8
        return {"name": "cube8", "N": N, "eps_r": cube(N, 4.0), "pulse": pulse(N, 4.0),
                "taps": fir_taps("none"), "steps": 256}
    if name == "sphere32":
        N = 32
        delta = 1e-7 * N ** 3
        return {"name": "sphere32", "N": N, "eps_r": sphere(N, 12.0), "pulse": pulse(N, 12.0),
                "taps": fir_taps("fir3", delta), "steps": 2048}
    if name == "block48":
        N = 48
        return {"name": "block48", "N": N, "eps_r": heterogeneous_block(N),
                "pulse": pulse(N, 12.0), "taps": fir_taps("none"), "steps": 2048}
    if name == "sphere104":
        N = 104
        delta = 1e-7 * N ** 3
        return {"name": "sphere104", "N": N, "eps_r": sphere(N, 12.0), "pulse": pulse(N, 12.0),
                "taps": fir_taps("fir3", delta), "steps": 4096}
    if name.startswith("sphere") or name.startswith("cube"):
        # small variants used by tests, e.g. "sphere10" (FIR3) or "cube6"
        kind = "sphere" if name.startswith("sphere") else "cube"
        N = int(name[len(kind):])
        eps = 12.0 if kind == "sphere" else 4.0
        geom = sphere(N, eps) if kind == "sphere" else cube(N, eps)
        taps = fir_taps("fir3", 1e-7 * N ** 3) if kind == "sphere" else fir_taps("none")
        return {"name": name, "N": N, "eps_r": geom, "pulse": pulse(N, eps), "taps": taps,
                "steps": 256}
    if name.startswith("box"):
        # "boxWxVxU": an eps_r = 12 block filling a W x V x U grid (u fastest), FIR3,
        # plane wave along +u; small anisotropic cases that still reach long lag windows
        W, V, U = (int(v) for v in name[3:].split("x"))
        M = W * V * U
        return {"name": name, "N": max(W, V, U), "eps_r": np.full((W, V, U), 12.0),
                "pulse": pulse(0, 12.0, k_hat=(1.0, 0.0, 0.0), p_hat=(0.0, 1.0, 0.0)),
                "taps": fir_taps("fir3", 1e-7 * M), "steps": 256}
    raise ValueError(name)
