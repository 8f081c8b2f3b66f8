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
