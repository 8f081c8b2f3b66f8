"""Pins of the oracle's adjoint dJ/dk (not GPU): central finite differences of
the oracle's forward tracking and the single-quadrupole closed form."""
import math

import numpy as np
import pytest

from oracle import adjoint, maps, mlp, moments
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init

KEYS = ("x", "px", "y", "py", "t", "pt")


def _bunch(n, seed=0):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return [z[k] for k in KEYS], g


def _fd(z, g, els, which, qi, h_rel=1e-6):
    idx = [i for i, e in enumerate(els) if e["kind"] == "quad"][qi]
    k = els[idx]["k"]
    h = h_rel * abs(k)
    out = []
    for s in (+1, -1):
        e2 = [dict(e) for e in els]
        e2[idx]["k"] = k + s * h
        out.append(adjoint.track_objective(z, g, e2, which))
    return (out[0] - out[1]) / (2 * h)


def test_single_quad_closed_form():
    z, g = _bunch(2000)
    bg = math.sqrt(g * g - 1)
    els = [{"kind": "quad", "L": 0.1, "k": 31.67}]
    J, grad = adjoint.track_grad(z, g, els, "sigma_x")
    S = moments.sigma_matrix(moments.moments28(z))
    M, D = maps.quad(0.1, 31.67, bg), maps.dquad_dk(0.1, 31.67, bg)
    dS = D @ S @ M.T + M @ S @ D.T
    J2 = math.sqrt((M @ S @ M.T)[0, 0])
    assert abs(J / J2 - 1) < 1e-13
    assert abs(grad[0] / (dS[0, 0] / (2 * J2)) - 1) < 1e-11


@pytest.mark.parametrize("which", ["sigma_x", "sigma_y"])
def test_linear_section_vs_finite_differences(which):
    z, g = _bunch(2000, seed=1)
    els = lattice.matching_section()
    J, grad = adjoint.track_grad(z, g, els, which)
    fd = np.array([_fd(z, g, els, which, qi) for qi in range(4)])
    assert np.max(np.abs(grad - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_emittance_gradient_vanishes_without_coupling():
    # emittance is invariant under uncoupled symplectic maps, so dJ/dk = 0
    z, g = _bunch(2000, seed=1)
    els = [e for e in lattice.matching_section() if e["kind"] != "sbend"]
    for which in ("eps_n_x", "eps_n_y"):
        J, grad = adjoint.track_grad(z, g, els, which)
        assert np.max(np.abs(grad)) < 1e-12 * J


def _surrogate(seed, z):
    Ws, bs = mlp_init([6, 32, 32, 6], seed)
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    return mlp.Surrogate(Ws, bs, mu, sd, mu, sd)


@pytest.mark.parametrize("which", ["eps_n_x", "sigma_x"])
def test_surrogate_beamline_vs_finite_differences(which):
    z, g = _bunch(1000, seed=2)
    els = []
    for s in range(2):
        st = lattice.plasma(400)
        st["surrogate"] = _surrogate(10 + s, z)
        els.append(st)
        els.extend(lattice.matching_section())
    J, grad = adjoint.track_grad(z, g, els, which)
    assert grad.shape == (8,)
    fd = np.array([_fd(z, g, els, which, qi) for qi in range(8)])
    assert np.max(np.abs(grad - fd)) <= 1e-6 * np.max(np.abs(fd))
