"""Beam moments (FP64): count, means and central second moments.

Follows the statistical beam moments of Sec. 4: the weighted average
<q> = sum w_i q_i / sum w_i (unit weights here), the beam width
sigma_x = sqrt(<x^2>), and the normalised emittance
eps_x = sqrt(<x^2><p_x^2> - <x p_x>^2) with momenta in units of m_e c. The
second moments are taken about the mean (reading: the paper writes them
about zero for a centred beam) with normalisation 1/N, and momenta are
px = p_x/p_ref, so eps_n,x = (beta gamma)_ref sqrt(S_xx S_pxpx - S_xpx^2).

Summation: two passes, each sum evaluated by math.fsum (correctly rounded).
The 28-vector is [N, 6 means, 21 central moments S_ab for a <= b in row-major
order of the coordinates (x, px, y, py, t, pt)].

Parity: pinned by exact rational arithmetic on small inputs, shift
invariance, invariance of the emittance under symplectic uncoupled maps and
the sample moments of the generator.
"""
import math

import numpy as np

PAIRS = [(a, b) for a in range(6) for b in range(a, 6)]


def moments28(z):
    """28 FP64 moments of the particles z (sequence of 6 arrays)."""
    cols = [np.asarray(c, dtype=np.float64) for c in z]
    n = cols[0].size
    out = np.zeros(28)
    out[0] = n
    if n == 0:
        return out
    mean = [math.fsum(c) / n for c in cols]
    out[1:7] = mean
    d = [c - m for c, m in zip(cols, mean)]
    for j, (a, b) in enumerate(PAIRS):
        out[7 + j] = math.fsum(d[a] * d[b]) / n
    return out


def sigma_matrix(m28):
    """6x6 central second-moment matrix from the 28-vector."""
    S = np.zeros((6, 6))
    for j, (a, b) in enumerate(PAIRS):
        S[a, b] = S[b, a] = m28[7 + j]
    return S


def derived(m28, gamma_ref):
    """Beam quantities of the moments for reference Lorentz factor gamma_ref."""
    bg = math.sqrt(gamma_ref * gamma_ref - 1.0)
    S = sigma_matrix(m28)
    mean_pt = m28[6]
    ex = bg * math.sqrt(max(S[0, 0] * S[1, 1] - S[0, 1] ** 2, 0.0))
    ey = bg * math.sqrt(max(S[2, 2] * S[3, 3] - S[2, 3] ** 2, 0.0))
    mean_gamma = gamma_ref - bg * mean_pt
    return {
        "eps_n_x": ex,
        "eps_n_y": ey,
        "sigma_x": math.sqrt(S[0, 0]),
        "sigma_y": math.sqrt(S[2, 2]),
        "mean_gamma": mean_gamma,
        "rel_energy_spread": bg * math.sqrt(S[5, 5]) / mean_gamma,
    }
