"""Pins of the oracle's beamline sequencing and of the surrogate's
normalisation wrap (not GPU).

* Surrogate.apply on an identity-path GELU network equals the closed-form
  affine ((z - mu_in) / sd_in) sd_out + mu_out (Sec. 3, data preparation),
  with mu_out != mu_in and sd_out != sd_in; a scaled-and-shifted path checks
  the output bias and the order of the two affines.
* beamline.track through a plasma stage and a transport section: the
  reference energy handed from the stage to the section is the stage-exit
  energy, fixed independently by a quadrature of ds = dgamma / (g cos phi);
  a drift after the stage moves t by L pt / (beta gamma)_exit^2 and x by
  L px exactly; the section acts as the ordered product of its elements; the
  snapshots are the moments of the particles after each element.
* A surrogate stage with a training domain maps the particles inside the box
  and hands the others to the plain push.

The network weights below are built so that gelu(a) - gelu(-a) = a, which
holds exactly for the tanh form because tanh is odd: a hidden pair
(+a, -a) carries a coordinate through any number of GELU layers.
"""
import math

import numpy as np
from scipy.integrate import quad as integrate
from scipy.optimize import brentq

from oracle import beamline, maps, mlp, moments, wake
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch

KEYS = ("x", "px", "y", "py", "t", "pt")
H = 128


def _identity_path(scale=1.0, shift=None):
    """6-128^4-6 GELU network whose FP64 forward is F(x) = scale x + shift."""
    W0 = np.zeros((H, 6))
    for j in range(6):
        W0[2 * j, j], W0[2 * j + 1, j] = 1.0, -1.0
    Wh = np.zeros((H, H))
    for j in range(6):
        Wh[2 * j, 2 * j], Wh[2 * j, 2 * j + 1] = 1.0, -1.0
        Wh[2 * j + 1, 2 * j], Wh[2 * j + 1, 2 * j + 1] = -1.0, 1.0
    W4 = np.zeros((6, H))
    for j in range(6):
        W4[j, 2 * j], W4[j, 2 * j + 1] = scale, -scale
    Ws = [W0, Wh, Wh.copy(), Wh.copy(), W4]
    bs = [np.zeros(H)] * 4 + [np.zeros(6) if shift is None else np.asarray(shift, float)]
    return Ws, bs


def _bunch(n, seed):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return [np.asarray(z[k], dtype=np.float64) for k in KEYS], g


def test_gelu_pair_identity_is_exact():
    a = np.linspace(-9.0, 9.0, 1001)
    assert np.max(np.abs(mlp.gelu(a) - mlp.gelu(-a) - a)) < 1e-14


def test_surrogate_apply_is_the_closed_form_affine():
    z, _ = _bunch(500, 3)
    mu_in = np.array([1e-7, -2e-6, 3e-7, 4e-6, -5e-7, 2e-3])
    sd_in = np.array([2e-6, 5e-4, 3e-6, 4e-4, 3e-6, 1e-2])
    mu_out = np.array([-4e-7, 1e-5, 2e-7, -3e-5, 1e-6, -6e-3])
    sd_out = np.array([7e-6, 2e-3, 5e-6, 9e-4, 2e-6, 3e-2])
    Ws, bs = _identity_path()
    got = mlp.Surrogate(Ws, bs, mu_in, sd_in, mu_out, sd_out).apply(z)
    for c in range(6):
        want = (z[c] - mu_in[c]) / sd_in[c] * sd_out[c] + mu_out[c]
        assert np.max(np.abs(got[c] - want)) <= 1e-13 * sd_out[c] * (1 + np.max(np.abs(z[c] - mu_in[c])) / sd_in[c])
    # F(x) = 2x + c: the output bias enters before the de-normalisation
    c = np.array([0.5, -1.0, 0.25, 2.0, -0.75, 1.5])
    Ws, bs = _identity_path(scale=2.0, shift=c)
    got = mlp.Surrogate(Ws, bs, mu_in, sd_in, mu_out, sd_out).apply(z)
    for j in range(6):
        want = (2.0 * (z[j] - mu_in[j]) / sd_in[j] + c[j]) * sd_out[j] + mu_out[j]
        assert np.max(np.abs(got[j] - want)) <= 1e-12 * sd_out[j] * (1 + np.max(np.abs(want - mu_out[j])) / sd_out[j])


def _gamma_exit_by_quadrature(st, g0):
    """Stage-exit gamma of the on-axis reference from the ODE's invariant and
    a quadrature of ds = dgamma / (g cos phi(gamma))."""
    I0 = (st.g / st.kp) * math.sin(st.kp * st.zeta0) - (g0 - math.sqrt(g0 * g0 - 1))

    def cosphi(gam):
        s = (st.kp / st.g) * (I0 + gam - math.sqrt(gam * gam - 1))
        return math.sqrt(1 - s * s)

    def s_of(gam):
        return integrate(lambda q: 1.0 / (st.g * cosphi(q)), g0, gam,
                         epsabs=1e-13, epsrel=1e-13, limit=200)[0]

    return brentq(lambda q: s_of(q) - st.L, g0 + 1, g0 + 2 * st.g * st.L, xtol=1e-12, rtol=1e-15)


def test_track_hands_the_stage_exit_reference_to_the_section():
    z, g0 = _bunch(64, 5)
    stage = lattice.plasma(400)
    L1 = 0.5
    section = [lattice.drift(L1), lattice.quad(0.1, 30.0), lattice.sbend(0.2, 1e-3),
               lattice.drift(0.3)]
    g_exit = _gamma_exit_by_quadrature(beamline.stage_of(stage), g0)
    bg = math.sqrt(g_exit * g_exit - 1)

    z_st, g_st, snaps_st = beamline.track(z, g0, [stage])
    assert abs(g_st / g_exit - 1) < 1e-11
    z_out, g_out, snaps = beamline.track(z, g0, [stage] + section)
    assert g_out == g_st
    assert [s[1] for s in snaps] == [g_st] * 5

    # the first drift, closed form at the exit reference
    z_d, _, _ = beamline.track(z, g0, [stage, section[0]])
    assert np.max(np.abs(z_d[0] - (z_st[0] + L1 * z_st[1]))) < 1e-15
    shift = z_d[4] - z_st[4]
    want = L1 * z_st[5] / (bg * bg)
    assert np.max(np.abs(shift - want)) < 1e-8 * np.max(np.abs(want))
    # with the entry reference instead the shift would be ~10x larger
    bg0 = math.sqrt(g0 * g0 - 1)
    assert np.max(np.abs(want)) < 0.2 * np.max(np.abs(L1 * z_st[5] / (bg0 * bg0)))

    # the section is the ordered product of its element maps (right to left)
    M = np.eye(6)
    for e in section:
        M = maps.element_matrix(e, bg) @ M
    want = M @ np.stack(z_st)
    assert np.max(np.abs(np.stack(z_out) - want) / (np.std(want, axis=1, keepdims=True))) < 1e-12
    Mrev = np.eye(6)
    for e in reversed(section):
        Mrev = maps.element_matrix(e, bg) @ Mrev
    assert np.max(np.abs(np.stack(z_out) - Mrev @ np.stack(z_st))) > 1e-9

    # each snapshot is the moments of the particles after its element
    zs = z_st
    for j, e in enumerate(section):
        zs = [r for r in maps.element_matrix(e, bg) @ np.stack(zs)]
        m = snaps[1 + j][0]
        assert m[0] == 64
        for a in range(6):
            assert abs(m[1 + a] - math.fsum(zs[a]) / 64) <= 1e-14 * np.std(zs[a]) + 1e-300
        mx = math.fsum(zs[0]) / 64
        sxx = math.fsum((zs[0] - mx) ** 2) / 64
        assert abs(m[7] - sxx) <= 1e-12 * sxx


def test_surrogate_stage_maps_inside_and_pushes_outside():
    z, g0 = _bunch(200, 7)
    stage = dict(lattice.plasma(400))
    mu_in = np.array([np.mean(c) for c in z])
    sd_in = np.array([np.std(c) for c in z])
    Ws, bs = _identity_path()
    # a box that leaves out the particles with x above its 80th percentile
    lo = np.array([np.min(c) for c in z]) - 1.0
    hi = np.array([np.max(c) for c in z]) + 1.0
    hi[0] = np.quantile(z[0], 0.8)
    sur = mlp.Surrogate(Ws, bs, mu_in, sd_in, 2 * mu_in, 3 * sd_in, domain=(lo, hi))
    stage["surrogate"] = sur
    z_out, g_out, snaps = beamline.track(z, g0, [stage])
    assert g_out == wake.reference_exit(beamline.stage_of(stage), g0)[0]
    inside = z[0] <= hi[0]
    assert 0 < inside.sum() < len(inside)
    pushed, _ = wake.push_stage([c[~inside] for c in z], g0, beamline.stage_of(stage))
    for c in range(6):
        mapped = (z[c][inside] - mu_in[c]) / sd_in[c] * (3 * sd_in[c]) + 2 * mu_in[c]
        assert np.max(np.abs(z_out[c][inside] - mapped)) <= 1e-12 * sd_in[c] * 10
        assert np.array_equal(z_out[c][~inside], pushed[c])
    assert np.array_equal(snaps[0][0], moments.moments28(z_out))
