"""Host-side bookkeeping of the diagnostics drivers (no GPU)."""
import numpy as np


def test_growth_per_step_recovers_alternating_rate():
    """A theta = pi component (-1)^n g^n above slow ringing (after the second
    difference): the estimate is g."""
    from paper_2407_03323_gb300.diagnostics import _growth_per_step, _probe_index
    n = np.arange(4000)
    for g in (1.0005, 1.003, 1.01):
        x = 0.1 * np.cos(2 * np.pi * 0.02 * n) * np.exp(-n / 3000) + 1e-3 * (-1.0) ** n * g ** n
        assert abs(_growth_per_step(x) - g) < 1e-4, g
    x = (-1.0) ** n * 0.998 ** n                     # decaying, nothing else present
    assert abs(_growth_per_step(x) - 0.998) < 1e-6
    assert _probe_index(20) == 2 + 20 * (7 + 20 * 2)
