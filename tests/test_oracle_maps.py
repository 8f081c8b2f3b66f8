"""Pins of the oracle's linear element maps (not GPU).

Each map is checked against the matrix exponential of the generator of the
element's linear Hamiltonian (an independent route), symplecticity, emittance
invariance on particles and the small-angle chicane closed form.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import maps, moments
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch

BG = [math.sqrt(1957.95 ** 2 - 1), math.sqrt(6111.38 ** 2 - 1), 3.0]
ELEMS = [
    {"kind": "drift", "L": 0.5},
    {"kind": "quad", "L": 0.1, "k": 50.0},
    {"kind": "quad", "L": 0.1, "k": -35.52},
    {"kind": "quad", "L": 0.3, "k": 1e-9},
    {"kind": "sbend", "L": 0.2, "angle": 1e-3},
    {"kind": "sbend", "L": 0.2, "angle": -1e-3},
    {"kind": "sbend", "L": 1.0, "angle": 0.3},
    {"kind": "plasma_lens", "L": 0.03, "k": 2000.0},
    {"kind": "plasma_lens", "L": 0.03, "k": -500.0},
    {"kind": "plasma_lens", "L": 0.03, "k": 1e-9},
]


@pytest.mark.parametrize("bg", BG)
@pytest.mark.parametrize("e", ELEMS)
def test_map_is_exponential_of_generator(e, bg):
    M = maps.element_matrix(e, bg)
    E = expm(e["L"] * maps.generator(e, bg))
    assert np.max(np.abs(M - E)) <= 1e-13 * max(1.0, np.max(np.abs(E)))


@pytest.mark.parametrize("bg", BG)
def test_symplectic(bg):
    Ms = [maps.element_matrix(e, bg) for e in ELEMS]
    seg = np.eye(6)
    for e in lattice.matching_section():
        seg = maps.element_matrix(e, bg) @ seg
    for M in Ms + [seg]:
        assert np.max(np.abs(M.T @ maps.J6 @ M - maps.J6)) < 1e-12


def test_quad_k_to_zero_is_drift():
    bg = BG[0]
    D = maps.drift(0.1, bg)
    for k in (1e-6, -1e-6):
        lin = D + k * maps.dquad_dk(0.1, 0.0, bg)
        assert np.max(np.abs(maps.quad(0.1, k, bg) - lin)) < 1e-14
    assert np.array_equal(maps.quad(0.1, 0.0, bg), D)


def test_dquad_dk_central_difference():
    bg = BG[0]
    for k in (50.0, -35.52, 0.0):
        h = 1e-5
        fd = (maps.quad(0.1, k + h, bg) - maps.quad(0.1, k - h, bg)) / (2 * h)
        assert np.max(np.abs(maps.dquad_dk(0.1, k, bg) - fd)) < 1e-9


def test_emittance_invariant_under_uncoupled_maps():
    z, g = gaussian_bunch(BunchRecipe(n=4000, seed=3))
    zz = np.stack([z[k] for k in ("x", "px", "y", "py", "t", "pt")])
    bg = math.sqrt(g * g - 1)
    d0 = moments.derived(moments.moments28(zz), g)
    for e in ELEMS[:4]:
        zo = maps.element_matrix(e, bg) @ zz
        d1 = moments.derived(moments.moments28(zo), g)
        for key in ("eps_n_x", "eps_n_y"):
            assert abs(d1[key] / d0[key] - 1) < 1e-12
    # a bend couples x and t: the 6D volume (det Sigma) is invariant
    S0 = moments.sigma_matrix(moments.moments28(zz))
    M = maps.element_matrix(ELEMS[6], bg)
    S1 = moments.sigma_matrix(moments.moments28(M @ zz))
    assert abs(np.linalg.det(S1) / np.linalg.det(S0) - 1) < 1e-9


def test_chicane_r56_small_angle():
    bg = BG[0]
    th, Lb, gap = 1e-3, 0.2, 0.25
    M = np.eye(6)
    els = lattice.chicane(th, Lb, gap)
    for e in els:
        M = maps.element_matrix(e, bg) @ M
    Ltot = sum(e["L"] for e in els)
    r56 = M[4, 5] - Ltot / (bg * bg)
    closed = 2 * th * th * (gap + 2.0 * Lb / 3.0)
    assert abs(r56 / closed - 1) < 10 * th * th
    # dispersion closes to third order in the angle
    assert abs(M[0, 5]) < 10 * th ** 3 * Ltot and abs(M[1, 5]) < 10 * th ** 3


def _rotation(theta):
    """Rotation by theta about the beam axis, acting on (x, y) and (px, py)."""
    c, s_ = math.cos(theta), math.sin(theta)
    R = np.eye(6)
    for a, b in ((0, 2), (1, 3)):
        R[a, a], R[a, b], R[b, a], R[b, b] = c, -s_, s_, c
    return R


def test_plasma_lens_is_round():
    """A plasma lens focuses both planes alike, so it commutes with rotations
    about the axis; a quadrupole of the same strength does not."""
    bg = BG[0]
    R = _rotation(0.37)
    Ml = maps.plasma_lens(0.03, 2000.0, bg)
    Mq = maps.quad(0.03, 2000.0, bg)
    assert np.max(np.abs(R @ Ml @ R.T - Ml)) < 1e-14
    assert np.max(np.abs(R @ Mq @ R.T - Mq)) > 1e-2


def test_plasma_lens_thin_limit_and_drift_limit():
    bg = BG[0]
    f = 0.25  # focal length [m]
    for L in (1e-3, 1e-4):
        M = maps.plasma_lens(L, 1.0 / (f * L), bg)
        for a in (0, 2):
            assert abs(M[a + 1, a] + 1.0 / f) < 2.0 * L / f ** 2  # -1/f (1 - O(L/f))
            assert abs(M[a, a] - 1.0) < L / f
    D = maps.drift(0.03, bg)
    assert np.array_equal(maps.plasma_lens(0.03, 0.0, bg), D)


def test_lens_strength_from_gradient():
    """k = e g / p: at p = 1 GeV/c the magnetic rigidity is 1e9 / c T m."""
    bg = 1000.0 / 0.51099895000
    brho = 1e9 / 299792458.0
    assert abs(maps.lens_k_from_gradient(1000.0, bg) / (1000.0 / brho) - 1) < 1e-9
