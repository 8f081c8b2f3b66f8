"""Host helpers of the workflow module (no GPU)."""
import math

from oracle import maps
from paper_2402_17248_gb300 import workflow


def test_plasma_lens_k_matches_oracle_and_rigidity():
    for g_T, gamma in ((3000.0, 6111.383), (500.0, 1957.951)):
        bg = math.sqrt(gamma * gamma - 1.0)
        assert abs(workflow.plasma_lens_k(g_T, gamma) / maps.lens_k_from_gradient(g_T, bg) - 1) < 1e-14
    # 1 GeV/c: B rho = 1e9 / c T m
    gamma = math.sqrt((1000.0 / 0.51099895) ** 2 + 1.0)
    assert abs(workflow.plasma_lens_k(1000.0, gamma) * (1e9 / 299792458.0) / 1000.0 - 1) < 1e-9
