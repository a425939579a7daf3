import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built extension")


@pytest.fixture(scope="session")
def cube8_oracle():
    """Oracle table, excitation and march for the 8^3 eps_r = 4 cube (256 steps)."""
    import workloads as wl
    from oracle import excitation, kernel_table, march
    from oracle.spline import num_lags
    cfg = wl.config("cube8")
    N = cfg["N"]
    ell = num_lags(N, N, N)
    G, Kv, Kf = kernel_table.octant_table(N, ell + 1)
    E = excitation.tested_excitation(cfg["eps_r"], cfg["pulse"], cfg["steps"])
    J = march.march(G, cfg["eps_r"], cfg["taps"], E)
    return {"cfg": cfg, "G": G, "Kv": Kv, "Kf": Kf, "E": E, "J": J, "ell": ell}
