"""The scattered field at probe voxels outside the grid (the objective of the adjoint
workload) on the device: the probe operator and its transpose against the oracle
(oracle/probes.py: elements per probe-voxel offset from the oracle's quadrature, the
plain sums over voxels and lags), and the gradient of the gated probe energy through
probe field + checkpointed adjoint march against central differences.

Tolerances: the two sides' element quadratures agree to ~1e-12 of the largest element
at an offset, so each field value agrees to 1e-11 of the largest |E|."""
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


@pytest.fixture(scope="module")
def case5():
    """5^3 heterogeneous grid, 8 Fibonacci probes on the sphere of radius 2N, random
    currents of 40 steps, and the oracle's probe elements (all lags up to the largest
    probe-voxel offset)."""
    from oracle import probes as pr
    N, steps = 5, 40
    rng = np.random.default_rng(21)
    eps = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    P = wl.fibonacci_probes(N, 8)
    far = np.abs(P[:, None, :] - np.array([[0, 0, 0], [N - 1, N - 1, N - 1]])[None]).max()
    nlag = int(np.ceil(np.sqrt(3.0) * (far + 1))) + 3
    Gp = pr.probe_elements(P, (N, N, N), nlag)
    J = rng.normal(size=(steps, N ** 3, 3))
    return {"N": N, "eps": eps, "P": P, "Gp": Gp, "J": J}


def test_probe_field_matches_oracle(mot, case5):
    from oracle import probes as pr
    c = case5
    ref = pr.probe_field(c["Gp"], c["J"])
    with mot.Context(c["eps"], precision="fp32_history") as ctx:
        ctx.probe_setup(c["P"])
        E = ctx.probe_field(c["J"])
    assert np.abs(ref).max() > 0
    assert np.abs(E - ref).max() < 1e-11 * np.abs(ref).max()


def test_probe_transpose_matches_oracle_gradient(mot, case5):
    """The transposed operator on W = 2 E (gated) is the oracle's dO/dJ of the gated
    probe energy; and <P J, W> = <J, P^T W> for random W."""
    from oracle import probes as pr
    c = case5
    E = pr.probe_field(c["Gp"], c["J"])
    first = 12
    W = 2.0 * E
    W[:first] = 0.0
    ref = pr.probe_objective_gradient(c["Gp"], E, first)
    rng = np.random.default_rng(4)
    Wr = rng.normal(size=E.shape)
    with mot.Context(c["eps"], precision="fp32_history") as ctx:
        ctx.probe_setup(c["P"])
        g = ctx.probe_transpose(W)
        PJ = ctx.probe_field(c["J"])
        PtW = ctx.probe_transpose(Wr)
    assert np.abs(g - ref).max() < 1e-11 * np.abs(ref).max()
    lhs, rhs = float((PJ * Wr).sum()), float((c["J"] * PtW).sum())
    assert abs(lhs - rhs) < 1e-12 * float(np.abs(PJ * Wr).sum())


def test_probe_energy_gradient_checkpointed_against_differences(mot):
    """O = sum over steps >= 40 and 16 probes (radius 2N, outside the grid) of |E^s|^2
    for a heterogeneous 8^3 block marched 96 steps in FP64; dO/deps_r through probe_field
    and the checkpointed march (every 24 steps) against central differences of two
    forward marches at 4 voxels."""
    torch = pytest.importorskip("torch")
    from paper_2407_03323_gb300.autograd import march, probe_field
    N, steps, first = 8, 96, 40
    rng = np.random.default_rng(9)
    eps0 = 2.0 + 9.0 * rng.uniform(size=(N, N, N))
    taps = wl.fir_taps("fir3", 1e-3)
    p = wl.pulse(N, 6.0)
    w = {"k_hat": p["k_hat"], "p_hat": p["p_hat"], "f_c": p["f_c"], "sigma_t": p["sigma_t"],
         "t0": p["t0"] - 50.0}
    pctx = mot.Context(eps0, precision="fp32_history")
    pctx.probe_setup(wl.fibonacci_probes(N, 16))

    def objective(J):
        return (probe_field(J, pctx)[first:] ** 2).sum()

    eps = torch.tensor(eps0, dtype=torch.float64, requires_grad=True)
    O = objective(march(eps, taps, w, steps, checkpoint_every=24))
    O.backward()
    grad = eps.grad.numpy().reshape(-1)
    gmax = np.abs(grad).max()
    assert gmax > 0

    def value(e):
        with torch.no_grad():
            return float(objective(march(torch.tensor(e), taps, w, steps)))

    h = 1e-4
    for m in rng.choice(N ** 3, 4, replace=False):
        ep = eps0.copy().reshape(-1)
        em = eps0.copy().reshape(-1)
        ep[m] += h
        em[m] -= h
        fd = (value(ep.reshape(eps0.shape)) - value(em.reshape(eps0.shape))) / (2 * h)
        assert abs(fd - grad[m]) < 1e-6 * max(abs(fd), 1e-2 * gmax), (m, fd, grad[m])
    pctx.close()
