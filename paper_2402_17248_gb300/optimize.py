"""Moment-driven transport between stages and gradient-based lens optimisation.

Matching (Sec. 4: the transport between accelerator stages is set from the
beam the previous stage delivers): a plasma stage focuses linearly with
k_beta^2 = K0 sin(phi0) / gamma (K0 = g k_p / 2, g = e E0 / (m_e c^2)), so a
beam enters it matched when beta = beta_m = 1 / k_beta and alpha = 0 in both
planes. `match_section` solves the strengths of a section's quadrupoles for
that target from the moments *measured* at the previous stage's exit (FP64
least squares on the host, with the library's own transfer matrices), and
`track_matched` tracks stage by stage, re-matching every section from the
moments the library just reduced.

Optimisation (Sec. 4.4 minimises the final emittance with Nelder-Mead over
repeated simulations): here the objective's exact gradient comes from the
adjoint (grad.beam_objective), so a quasi-Newton method (L-BFGS) drives the
quadrupole strengths.
"""
import math

import numpy as np
import torch
from scipy.optimize import least_squares

from . import bl
from .grad import beam_objective

E_CHARGE = 1.602176634e-19
M_E = 9.1093837015e-31
C_LIGHT = 299792458.0
EPS0 = 8.8541878128e-12

# 28-vector layout: N, 6 means, then the 21 central second moments
# S[a][b], a <= b, row by row
_PAIRS = [(a, b) for a in range(6) for b in range(a, 6)]


def sigma_matrix(m28):
    S = np.zeros((6, 6))
    for j, (a, b) in enumerate(_PAIRS):
        S[a, b] = S[b, a] = m28[7 + j]
    return S


def twiss(S, plane):
    """(beta, alpha, geometric emittance) of plane 0 (x) or 1 (y) from the
    central second-moment matrix S."""
    i = 2 * plane
    sxx, sxp, spp = S[i, i], S[i, i + 1], S[i + 1, i + 1]
    eps = math.sqrt(max(sxx * spp - sxp * sxp, 0.0))
    return sxx / eps, -sxp / eps, eps


def matched_beta(stage, gamma):
    """beta_m = 1 / k_beta of a prescribed-wake stage for reference gamma."""
    n0 = stage["n0_cm3"] * 1e6
    kp = math.sqrt(n0 * E_CHARGE ** 2 / (EPS0 * M_E)) / C_LIGHT
    g = E_CHARGE * stage["E0_Vpm"] / (M_E * C_LIGHT ** 2)
    k_beta2 = 0.5 * g * kp * math.sin(stage["phi0"]) / gamma
    return 1.0 / math.sqrt(k_beta2)


def _with_quads(section, k):
    out, q = [], 0
    for e in section:
        e = dict(e)
        if e["kind"] == "quad":
            e["k"] = float(k[q])
            q += 1
        out.append(e)
    return out


def match_section(S, gamma, section, beta_target, k0):
    """Quadrupole strengths (in section order) that take the beam with
    central second moments S at the section entrance to beta = beta_target,
    alpha = 0 in x and y at its exit. Returns (k, residual vector)."""
    def residual(k):
        M = bl.bl_segment_matrix(_with_quads(section, k), gamma)
        So = M @ S @ M.T
        bx, ax, _ = twiss(So, 0)
        by, ay, _ = twiss(So, 1)
        return np.array([bx / beta_target - 1.0, ax, by / beta_target - 1.0, ay])

    sol = least_squares(residual, np.asarray(k0, dtype=np.float64), xtol=1e-14, ftol=1e-14,
                        gtol=1e-14, max_nfev=2000)
    return sol.x, residual(sol.x)


def track_matched(bunch, stages, section, k0):
    """Track `bunch` through stage 1, section, stage 2, section, ... where
    each section's quadrupoles are matched, from the moments measured at the
    preceding stage's exit, to the next stage (the last section to a copy of
    the last stage). `stages`: plasma element dicts (with or without
    surrogates); `section`: linear element dicts whose quads are re-solved.
    Returns a list of per-stage records."""
    k = np.asarray(k0, dtype=np.float64)
    log = []
    for i, st in enumerate(stages):
        g_in = bunch.gamma_ref
        bl.bl_track(bunch, bl.Lattice([st]), moments=False)
        m_exit = bl.bl_moments(bunch)[0]
        g_out = bunch.gamma_ref
        nxt = stages[i + 1] if i + 1 < len(stages) else st
        beta_t = matched_beta(nxt, g_out)
        k, res = match_section(sigma_matrix(m_exit), g_out, section, beta_t, k)
        bl.bl_track(bunch, bl.Lattice(_with_quads(section, k)), moments=False)
        m_next = bl.bl_moments(bunch)[0]
        log.append({"stage": i, "gamma_in": g_in, "gamma_out": g_out, "k": k.copy(),
                    "residual": res, "beta_target": beta_t, "moments_exit": m_exit,
                    "moments_next_entry": m_next})
    return log


def minimize_objective(bunch, elements, objective="eps_n_x", iters=10, k_init=None):
    """L-BFGS over the quadrupole strengths of `elements` for the objective of
    the final moments (the bunch is not modified). Returns (k, history of J)."""
    k0 = np.array([e["k"] for e in elements if e["kind"] == "quad"] if k_init is None else k_init,
                  dtype=np.float64)
    # optimise the relative change of k; J is scaled by its starting value
    scale = np.where(np.abs(k0) > 0, np.abs(k0), 1.0)
    u = torch.zeros(len(k0), dtype=torch.float64, requires_grad=True)
    kt, st = torch.tensor(k0), torch.tensor(scale)
    with torch.no_grad():
        J0 = float(beam_objective(kt, bunch, elements, objective).sum())
    hist = [J0]
    opt = torch.optim.LBFGS([u], lr=1.0, max_iter=iters, history_size=10,
                            line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        J = beam_objective(kt + st * u, bunch, elements, objective).sum() / J0
        J.backward()
        hist.append(float(J.detach()) * J0)
        return J

    opt.step(closure)
    return (kt + st * u).detach().numpy(), hist
