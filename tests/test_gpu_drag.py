"""Hasimoto's square-array drag at resolutions the CPU oracle is too slow for: radius 4, 8 and
16 (cells of 32^2 to 128^2, up to ~10^5 steps to steady state) on the CUDA path in FP64 storage,
which reproduces the oracle bit for bit (test_gpu_parity). Pins as in test_oracle_drag."""
import numpy as np
import pytest

from paper_1105_2904_gb300 import lbmp
from test_oracle_drag import steady_cylinder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()


def test_hasimoto_offset_over_a_fourfold_resolution_range():
    make = lambda L, tau, F: lbmp.Simulation(0, L, L, 1, tau, body_force=(F, 0.0, 0.0), precision="fp64")
    res = [steady_cylinder(make, r) for r in (4.0, 8.0, 16.0)]
    deltas = np.array([d for d, _ in res])
    ratios = np.array([q for _, q in res])
    print("delta", deltas, "reported / total", ratios)
    assert np.all((deltas > 0.0) & (deltas < 1.0))
    assert deltas.max() - deltas.min() <= 0.3
    assert np.all((ratios > 0.70) & (ratios < 0.80))
