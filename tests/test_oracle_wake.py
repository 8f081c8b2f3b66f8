"""Pins of the oracle's prescribed-wake RK4 stage (not GPU).

* on-axis invariant (g/k_p) sin(k_p zeta) - (gamma - u_z) of the ODE;
* gamma at the stage exit from an independent quadrature of ds = dgamma / (g cos phi);
* the RK4 routine on a linear system equals the degree-4 Taylor polynomial of
  exp(hA) to the n-th power;
* the RK4 push of the full system against an independent adaptive integrator,
  and its fourth-order convergence;
* adiabatic invariance of the betatron action (gamma K)^(1/2) x^2 + u_x^2 (gamma K)^(-1/2)
  and the WKB phase advance of a small-amplitude particle.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad as integrate, solve_ivp
from scipy.optimize import brentq

from oracle import wake
from synth.bunch import BunchRecipe, gaussian_bunch

ST = wake.Stage(L=0.3, nsteps=400)
G0 = 1957.9511835591836


def _f(st):
    return lambda Y: wake.rhs(Y, st.g, st.K0, st.kp)


def _invariant(st, zeta, uz):
    gamma = np.sqrt(1 + uz * uz)
    return (st.g / st.kp) * np.sin(st.kp * zeta) - (gamma - uz)


def test_on_axis_invariant_conserved():
    zeta0 = ST.zeta0 + np.array([-2e-6, 0.0, 3e-6, 5e-6])
    uz0 = np.sqrt(np.array([1900.0, 1957.95, 2100.0, 6000.0]) ** 2 - 1)
    zero = np.zeros(4)
    Y = wake.rk4(_f(ST), (zero, zero, zero, zero, zeta0, uz0), ST.L / ST.nsteps, ST.nsteps)
    I0 = _invariant(ST, zeta0, uz0)
    I1 = _invariant(ST, Y[4], Y[5])
    assert np.max(np.abs(I1 - I0)) < 1e-12
    assert np.all(Y[5] > uz0 + 1000)        # accelerated


def test_reference_gamma_matches_quadrature():
    g_out, zeta_out, uz_out = wake.reference_exit(ST, G0)
    I0 = _invariant(ST, ST.zeta0, math.sqrt(G0 * G0 - 1))

    def cosphi(gam):
        s = (ST.kp / ST.g) * (I0 + gam - math.sqrt(gam * gam - 1))
        return math.sqrt(1 - s * s)

    def s_of(gam):
        return integrate(lambda q: 1.0 / (ST.g * cosphi(q)), G0, gam,
                         epsabs=1e-13, epsrel=1e-13, limit=200)[0]

    g_quad = brentq(lambda q: s_of(q) - ST.L, G0 + 1, G0 + 2 * ST.g * ST.L, xtol=1e-12, rtol=1e-15)
    assert abs(g_out / g_quad - 1) < 1e-11
    assert abs(g_out - 6111.3828298) < 1e-6


def test_rk4_linear_system_closed_form():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(6, 6))
    Y0 = rng.normal(size=(6, 3))
    h, n = 0.05, 37
    f = lambda Y: tuple(A @ np.stack(Y))
    Y = np.stack(wake.rk4(f, tuple(Y0), h, n))
    hA = h * A
    T4 = np.eye(6) + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
    ref = np.linalg.matrix_power(T4, n) @ Y0
    assert np.max(np.abs(Y - ref)) < 1e-12 * np.max(np.abs(ref))


def _sample(n=4):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=11))
    return [z[k] for k in ("x", "px", "y", "py", "t", "pt")], g


def test_rk4_push_matches_adaptive_integrator():
    z, g = _sample(3)
    Y0 = wake.to_absolute(z, g, ST.zeta0)
    f = _f(ST)

    def ode(s, y):
        return np.concatenate(f(tuple(y.reshape(6, -1))))

    ref = solve_ivp(ode, (0.0, ST.L), np.concatenate(Y0), method="DOP853",
                    rtol=1e-13, atol=1e-30).y[:, -1].reshape(6, -1)
    scale = np.array([2e-6, 1.0, 2e-6, 1.0, 3e-6, 100.0])[:, None]
    err = lambda n: np.max(np.abs(np.stack(wake.rk4(f, Y0, ST.L / n, n)) - ref) / scale)
    e1, e2, e3 = err(1500), err(3000), err(12000)
    # fourth order: halving the step divides the error by about 16, down to
    # the truncation error of the finest run (the adaptive result is ~1e-12)
    assert 12 < e1 / e2 < 20
    assert e3 < 3e-8 and e3 < 1.5 * e1 / 16 ** 3


def test_betatron_action_and_wkb_phase():
    st = ST
    x0 = 1e-8
    uz0 = math.sqrt(G0 * G0 - 1)
    one = np.ones(1)
    Y0 = (x0 * one, 0 * one, 0 * one, 0 * one, st.zeta0 * one, uz0 * one)
    n = 4000
    h = st.L / n
    f = _f(st)
    Y = Y0
    psi = 0.0
    xs, us, gs, ks = [], [], [], []
    for i in range(n):
        gam = float(np.sqrt(1 + Y[5][0] ** 2))
        K = st.K0 * math.sin(st.kp * Y[4][0])
        xs.append(Y[0][0]); us.append(Y[1][0]); gs.append(gam); ks.append(K)
        Y = wake.rk4(f, Y, h, 1)
    gam = float(np.sqrt(1 + Y[5][0] ** 2))
    K = st.K0 * math.sin(st.kp * Y[4][0])
    gs.append(gam); ks.append(K); xs.append(Y[0][0]); us.append(Y[1][0])
    gs, ks = np.array(gs), np.array(ks)
    w = np.sqrt(ks / gs)
    psi_wkb = float(np.sum(0.5 * (w[1:] + w[:-1])) * h)

    def action(x, u, gK):
        return math.sqrt(gK) * x * x + u * u / math.sqrt(gK)

    J0 = action(xs[0], us[0], gs[0] * ks[0])
    J1 = action(xs[-1], us[-1], gs[-1] * ks[-1])
    assert abs(J1 / J0 - 1) < 2e-2
    # final phase of the oscillation versus the WKB phase integral
    ang = math.atan2(-us[-1] / math.sqrt(gs[-1] * ks[-1]), xs[-1])
    d = (ang - psi_wkb + math.pi) % (2 * math.pi) - math.pi
    assert abs(d) < 0.05
    assert 80 < psi_wkb < 120


def test_entry_exit_roundtrip():
    z, g = _sample(50)
    Y = wake.to_absolute(z, g, 1.3e-5)
    back = wake.to_relative(Y, g, 1.3e-5)
    for a, b in zip(z, back):
        assert np.max(np.abs(np.asarray(a) - b)) <= 1e-12 * max(1e-30, np.max(np.abs(a)))
