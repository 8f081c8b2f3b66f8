"""Host parts of the matching and optimisation layer (no GPU): Twiss from
moments, the library's FP64 segment matrices against the oracle's, the
matched beta of a stage against the oracle's constants, and a matching solve
checked by propagating with the oracle's maps."""
import math

import numpy as np
import pytest

from oracle import constants, maps
from paper_2402_17248_gb300 import bl, optimize
from synth import lattice


def _sigma_from_twiss(bx, ax, ex, by, ay, ey, spt=1e-6):
    S = np.zeros((6, 6))
    for i, (b, a, e) in enumerate(((bx, ax, ex), (by, ay, ey))):
        g = (1 + a * a) / b
        S[2 * i, 2 * i] = b * e
        S[2 * i, 2 * i + 1] = S[2 * i + 1, 2 * i] = -a * e
        S[2 * i + 1, 2 * i + 1] = g * e
    S[4, 4] = 1e-12
    S[5, 5] = spt * spt
    return S


def test_twiss_roundtrip():
    S = _sigma_from_twiss(3.9e-3, 0.8, 3.1e-10, 5.0e-3, -0.4, 2.7e-10)
    m28 = np.zeros(28)
    for j, (a, b) in enumerate(optimize._PAIRS):
        m28[7 + j] = S[a, b]
    S2 = optimize.sigma_matrix(m28)
    assert np.array_equal(S, S2)
    for plane, want in ((0, (3.9e-3, 0.8, 3.1e-10)), (1, (5.0e-3, -0.4, 2.7e-10))):
        got = optimize.twiss(S2, plane)
        assert np.allclose(got, want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("gamma", [1957.951, 6111.383])
def test_segment_matrix_matches_oracle(gamma):
    els = lattice.matching_section() + [lattice.plasma_lens(0.03, 1500.0), lattice.drift(0.1)]
    M = bl.bl_segment_matrix(els, gamma)
    bg = math.sqrt(gamma * gamma - 1.0)
    W = np.eye(6)
    for e in els:
        W = maps.element_matrix(e, bg) @ W
    assert np.max(np.abs(M - W)) <= 1e-13 * np.max(np.abs(W))
    assert np.array_equal(bl.bl_segment_matrix([], gamma), np.eye(6))
    with pytest.raises(bl.BlError):
        bl.bl_segment_matrix([lattice.plasma(10)], gamma)


def test_matched_beta_matches_oracle_constants():
    st = lattice.plasma(400)
    for gamma in (1957.951, 35171.0):
        kb2 = 0.5 * constants.field_g(st["E0_Vpm"]) * constants.plasma_kp(st["n0_cm3"]) \
            * math.sin(st["phi0"]) / gamma
        assert abs(optimize.matched_beta(st, gamma) * math.sqrt(kb2) - 1) < 1e-9


def test_match_section_reaches_target_under_oracle_maps():
    gamma = 6111.383
    st = lattice.plasma(400)
    beta_t = optimize.matched_beta(st, gamma)
    S = _sigma_from_twiss(3.9e-3, 0.6, 3.1e-10, 4.2e-3, 0.3, 3.0e-10)
    sec = lattice.matching_section()
    k, res = optimize.match_section(S, gamma, sec, beta_t, lattice.DESIGN_K)
    assert np.max(np.abs(res)) < 1e-9
    bg = math.sqrt(gamma * gamma - 1.0)
    M = np.eye(6)
    q = 0
    for e in sec:
        e = dict(e)
        if e["kind"] == "quad":
            e["k"] = k[q]
            q += 1
        M = maps.element_matrix(e, bg) @ M
    So = M @ S @ M.T
    for plane in (0, 1):
        b, a, _ = optimize.twiss(So, plane)
        assert abs(b / beta_t - 1) < 1e-8 and abs(a) < 1e-8
