"""Plasma stage with a prescribed linear-regime wake, classical RK4 in s (FP64).

The paper's plasma stages are nonlinear per-particle phase-space maps
(Sec. 4 and Sec. 1: an element is a map f: R^6 -> R^6) obtained from PIC.
Here the stage is the plain method the surrogate learns from: each particle
is pushed independently through a prescribed wake of the plasma density n0,

    E_z = E0 cos(k_p zeta),   focusing  E0 k_p r sin(k_p zeta) / 2,

with zeta = z - c t the co-moving position (the paper's xi, Sec. 4.1) and the
lattice position s as independent variable (Sec. 1). With u = p/(m_e c),
gamma = sqrt(1 + |u|^2), g = e E0/(m_e c^2), K0 = g k_p / 2, phi = k_p zeta:

    dx/ds   = u_x / u_z                   dy/ds   = u_y / u_z
    du_x/ds = -(gamma/u_z) K0 sin(phi) x  du_y/ds = -(gamma/u_z) K0 sin(phi) y
    dzeta/ds = 1 - gamma/u_z              du_z/ds = (gamma/u_z) g cos(phi)

(d/ds = (gamma/(c u_z)) d/dt; the last two follow from v_z = c u_z/gamma.)
Relative coordinates map to this absolute state with the stage-entry
reference (gamma_r, (beta gamma)_r, zeta_r):
u_x = px (beta gamma)_r, gamma = gamma_r - pt (beta gamma)_r,
u_z = sqrt(gamma^2 - 1 - u_x^2 - u_y^2), zeta = zeta_r - t; and back at the
exit with the exit reference. The reference particle is the on-axis particle
entering at phase phi0, pushed by the same RK4; the next stage re-phases it
to phi0 (identical repeated stages, Sec. 4).

Parity: pinned by the on-axis invariant (g/k_p) sin(k_p zeta) - (gamma - u_z),
by gamma(L) from an independent quadrature, by RK4 on a linear system against
the degree-4 Taylor polynomial of exp(hA), by an independent adaptive
integrator on the full system, and by the adiabatic gamma^(-1/4) amplitude law.
"""
import math

import numpy as np

from .constants import plasma_kp, field_g


class Stage:
    """Parameters of one prescribed-wake plasma stage."""

    def __init__(self, L=0.3, nsteps=400, n0_cm3=1.0e17, E0_Vpm=10.0e9,
                 phi0=math.pi / 4.0):
        self.L = float(L)
        self.nsteps = int(nsteps)
        self.kp = plasma_kp(n0_cm3)
        self.g = field_g(E0_Vpm)
        self.K0 = 0.5 * self.g * self.kp
        self.phi0 = float(phi0)
        self.zeta0 = self.phi0 / self.kp


def rhs(Y, g, K0, kp):
    """Right-hand side of the stage ODE; Y = (x, ux, y, uy, zeta, uz) arrays."""
    x, ux, y, uy, zeta, uz = Y
    gamma = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    r = gamma / uz
    phi = kp * zeta
    sphi = np.sin(phi)
    return (ux / uz,
            -r * K0 * sphi * x,
            uy / uz,
            -r * K0 * sphi * y,
            1.0 - r,
            r * g * np.cos(phi))


def rk4(f, Y, h, n):
    """Classical fourth-order Runge-Kutta, n uniform steps of size h."""
    Y = tuple(np.array(c, dtype=np.float64, copy=True) for c in Y)
    for _ in range(n):
        k1 = f(Y)
        k2 = f(tuple(a + 0.5 * h * b for a, b in zip(Y, k1)))
        k3 = f(tuple(a + 0.5 * h * b for a, b in zip(Y, k2)))
        k4 = f(tuple(a + h * b for a, b in zip(Y, k3)))
        Y = tuple(a + (h / 6.0) * (b1 + 2.0 * b2 + 2.0 * b3 + b4)
                  for a, b1, b2, b3, b4 in zip(Y, k1, k2, k3, k4))
    return Y


def reference_exit(stage: Stage, gamma_in):
    """On-axis reference through the stage: returns (gamma_out, zeta_out, uz_out)."""
    uz0 = math.sqrt(gamma_in * gamma_in - 1.0)
    Y0 = tuple(np.array([v]) for v in (0.0, 0.0, 0.0, 0.0, stage.zeta0, uz0))
    f = lambda Y: rhs(Y, stage.g, stage.K0, stage.kp)
    Y = rk4(f, Y0, stage.L / stage.nsteps, stage.nsteps)
    uz = float(Y[5][0])
    return math.sqrt(1.0 + uz * uz), float(Y[4][0]), uz


def to_absolute(z, gamma_r, zeta_r):
    """Relative (x, px, y, py, t, pt) -> absolute (x, ux, y, uy, zeta, uz)."""
    bg = math.sqrt(gamma_r * gamma_r - 1.0)
    ux = z[1] * bg
    uy = z[3] * bg
    gamma = gamma_r - z[5] * bg
    uz = np.sqrt(gamma * gamma - 1.0 - ux * ux - uy * uy)
    return (np.asarray(z[0], dtype=np.float64), ux, np.asarray(z[2], dtype=np.float64),
            uy, zeta_r - z[4], uz)


def to_relative(Y, gamma_r, zeta_r):
    """Absolute (x, ux, y, uy, zeta, uz) -> relative (x, px, y, py, t, pt)."""
    bg = math.sqrt(gamma_r * gamma_r - 1.0)
    x, ux, y, uy, zeta, uz = Y
    gamma = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    return [x, ux / bg, y, uy / bg, zeta_r - zeta, -(gamma - gamma_r) / bg]


def push_stage(z, gamma_in, stage: Stage):
    """Push relative coordinates through one stage; returns (z_out, gamma_out)."""
    gamma_out, zeta_out, _ = reference_exit(stage, gamma_in)
    Y = to_absolute(z, gamma_in, stage.zeta0)
    f = lambda Yv: rhs(Yv, stage.g, stage.K0, stage.kp)
    Y = rk4(f, Y, stage.L / stage.nsteps, stage.nsteps)
    return to_relative(Y, gamma_out, zeta_out), gamma_out
