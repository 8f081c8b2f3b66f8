"""Linear transfer maps of the conventional beamline elements (FP64).

Each element is a per-particle map f: R^6 -> R^6 (Sec. 1: elements as
transfer maps when collective effects are negligible), here linear, acting on
the relative coordinates (x, px, y, py, t, pt) of s-based tracking relative to
a reference trajectory (Sec. 1, s as the independent variable). The paper
does not print the element maps; they are the solutions of the linear
equations of motion of the Hamiltonian

    H = px^2/2 + py^2/2 + pt^2 / (2 beta^2 gamma^2)
        + h^2 x^2 / 2 + h x pt / beta + k (x^2 - y^2) / 2

for a drift (h = k = 0), a quadrupole (h = 0; k > 0 focuses x) and a sector
bend without edge focusing (k = 0, curvature h = angle / L). An active plasma
lens (Sec. 4: the lenses between stages) focuses both planes alike: its
Hamiltonian has k (x^2 + y^2) / 2 in place of the quadrupole's
k (x^2 - y^2) / 2, with k = e g / p_ref for the azimuthal field gradient
g = dB/dr.

Parity: pinned by the matrix exponential of the generator of H (scipy
expm), by symplecticity, emittance invariance and the chicane R56 closed form.
"""
import math

import numpy as np

J6 = np.zeros((6, 6))
for _p in range(3):
    J6[2 * _p, 2 * _p + 1] = 1.0
    J6[2 * _p + 1, 2 * _p] = -1.0


def beta_from_bg(bg):
    return bg / math.sqrt(1.0 + bg * bg)


def drift(L, bg):
    """Drift of length L for reference beta*gamma = bg."""
    M = np.eye(6)
    M[0, 1] = L
    M[2, 3] = L
    M[4, 5] = L / (bg * bg)
    return M


def _plane(L, k):
    """2x2 map of x'' = -k x over length L."""
    if k > 0.0:
        w = math.sqrt(k)
        c, s = math.cos(w * L), math.sin(w * L)
        return np.array([[c, s / w], [-w * s, c]])
    if k < 0.0:
        w = math.sqrt(-k)
        c, s = math.cosh(w * L), math.sinh(w * L)
        return np.array([[c, s / w], [w * s, c]])
    return np.array([[1.0, L], [0.0, 1.0]])


def quad(L, k, bg):
    """Quadrupole of length L and strength k [1/m^2]; k > 0 focuses x."""
    M = np.eye(6)
    M[0:2, 0:2] = _plane(L, k)
    M[2:4, 2:4] = _plane(L, -k)
    M[4, 5] = L / (bg * bg)
    return M


def plasma_lens(L, k, bg):
    """Active plasma lens of length L and strength k [1/m^2] in both planes."""
    M = np.eye(6)
    M[0:2, 0:2] = _plane(L, k)
    M[2:4, 2:4] = _plane(L, k)
    M[4, 5] = L / (bg * bg)
    return M


E_CHARGE = 1.602176634e-19      # C
M_E = 9.1093837015e-31          # kg
C_LIGHT = 299792458.0           # m/s


def lens_k_from_gradient(grad_T_per_m, bg):
    """k = e g / p_ref with p_ref = bg m_e c."""
    return E_CHARGE * grad_T_per_m / (bg * M_E * C_LIGHT)


def _dplane_dk(L, k):
    """d/dk of the 2x2 map of x'' = -k x (k != 0)."""
    if k > 0.0:
        w = math.sqrt(k)
        c, s = math.cos(w * L), math.sin(w * L)
        dw = 0.5 / w
        # d/dw of [[c, s/w], [-w s, c]]
        dM = np.array([[-L * s, L * c / w - s / (w * w)],
                       [-s - w * L * c, -L * s]])
        return dM * dw
    if k < 0.0:
        w = math.sqrt(-k)
        c, s = math.cosh(w * L), math.sinh(w * L)
        dw = -0.5 / w
        dM = np.array([[L * s, L * c / w - s / (w * w)],
                       [s + w * L * c, L * s]])
        return dM * dw
    # k = 0: series limit d/dk at 0 of [[1 - k L^2/2, L - k L^3/6], [-k L, 1 - k L^2/2]]
    return np.array([[-L * L / 2.0, -L ** 3 / 6.0], [-L, -L * L / 2.0]])


def dquad_dk(L, k, bg):
    """Derivative of the quadrupole matrix with respect to k."""
    D = np.zeros((6, 6))
    D[0:2, 0:2] = _dplane_dk(L, k)
    D[2:4, 2:4] = -_dplane_dk(L, -k)
    return D


def sbend(L, angle, bg):
    """Sector bend of arc length L and bending angle `angle` (no edge focusing)."""
    if angle == 0.0:
        return drift(L, bg)
    h = angle / L
    b = beta_from_bg(bg)
    C, S = math.cos(angle), math.sin(angle)
    M = np.eye(6)
    M[0, 0] = C
    M[0, 1] = S / h
    M[0, 5] = -(1.0 - C) / (h * b)
    M[1, 0] = -h * S
    M[1, 1] = C
    M[1, 5] = -S / b
    M[2, 3] = L
    M[4, 0] = S / b
    M[4, 1] = (1.0 - C) / (h * b)
    M[4, 5] = L / (bg * bg) - (angle - S) / (h * b * b)
    return M


def element_matrix(e, bg):
    """Matrix of a linear element given as a dict with 'kind' and parameters."""
    kind = e["kind"]
    if kind == "drift":
        return drift(e["L"], bg)
    if kind == "quad":
        return quad(e["L"], e["k"], bg)
    if kind == "sbend":
        return sbend(e["L"], e["angle"], bg)
    if kind == "plasma_lens":
        return plasma_lens(e["L"], e["k"], bg)
    raise ValueError("not a linear element: %r" % kind)


def generator(e, bg):
    """Coefficient matrix A of dz/ds = A z for the element's Hamiltonian.

    Used only to pin the element maps (M = expm(L A)).
    """
    b = beta_from_bg(bg)
    A = np.zeros((6, 6))
    A[0, 1] = 1.0
    A[2, 3] = 1.0
    A[4, 5] = 1.0 / (bg * bg)
    k = e.get("k", 0.0) if e["kind"] in ("quad", "plasma_lens") else 0.0
    h = e["angle"] / e["L"] if e["kind"] == "sbend" else 0.0
    A[1, 0] = -(h * h + k)
    A[3, 2] = -k if e["kind"] == "plasma_lens" else k
    A[1, 5] = -h / b
    A[4, 0] = h / b
    return A
