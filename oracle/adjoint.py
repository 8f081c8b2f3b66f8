"""Reverse-mode gradient of final beam quantities w.r.t. quadrupole strengths.

The paper tunes the transport between stages by optimising lens strengths
against final beam moments (Sec. 4.4, emittance as the figure of merit). This
module gives the exact gradient of such an objective for a beamline of
linear elements and surrogate stages, in FP64, by hand-derived reverse mode:

* objective J of the final central moments (eps_n,x or sigma_x, and the y
  analogues), seeded per particle as lambda_i = dJ/dz_i;
* linear element z_out = M z_in: lambda_in = M^T lambda_out and, for a
  quadrupole, dJ/dk += sum_i lambda_out,i^T (dM/dk) z_in,i;
* surrogate stage: lambda_in = J_F(z_in)^T lambda_out through the MLP
  (normalisation, layers, GELU) by oracle.mlp.backward.

Parity: pinned by central finite differences of the oracle's own forward
tracking (whose parts are pinned separately) and by the closed form
dSigma/dk = M' Sigma M^T + M Sigma M'^T for a single quadrupole.
"""
import math

import numpy as np

from . import maps, mlp, moments, wake
from .beamline import apply_matrix

OBJECTIVES = ("eps_n_x", "sigma_x", "eps_n_y", "sigma_y")


def objective(m28, gamma_ref, which):
    return moments.derived(m28, gamma_ref)[which]


def seed(z, gamma_ref, which):
    """(J, lambda) with lambda_i = dJ/dz_i for the final particles z."""
    m = moments.moments28(z)
    S = moments.sigma_matrix(m)
    n = m[0]
    bg = math.sqrt(gamma_ref * gamma_ref - 1.0)
    lam = [np.zeros_like(np.asarray(c, dtype=np.float64)) for c in z]
    a = 0 if which.endswith("_x") else 2
    b = a + 1
    da = np.asarray(z[a], dtype=np.float64) - m[1 + a]
    db = np.asarray(z[b], dtype=np.float64) - m[1 + b]
    if which.startswith("eps"):
        D = S[a, a] * S[b, b] - S[a, b] ** 2
        J = bg * math.sqrt(D)
        c = bg / (2.0 * math.sqrt(D)) * (2.0 / n)
        lam[a] = c * (S[b, b] * da - S[a, b] * db)
        lam[b] = c * (S[a, a] * db - S[a, b] * da)
    else:
        J = math.sqrt(S[a, a])
        lam[a] = da / (n * J)
    return J, lam


def track_grad(z, gamma_ref, elements, which, bf16=False):
    """J and dJ/dk for every quadrupole (in element order) of the beamline."""
    z = [np.asarray(c, dtype=np.float64).copy() for c in z]
    tape = []
    for e in elements:
        if e["kind"] == "plasma":
            sur = e.get("surrogate")
            if sur is None:
                raise ValueError("the adjoint covers surrogate stages only")
            st = wake.Stage(L=e["L"], nsteps=e["nsteps"], n0_cm3=e["n0_cm3"],
                            E0_Vpm=e["E0_Vpm"], phi0=e["phi0"])
            gamma_out, _, _ = wake.reference_exit(st, gamma_ref)
            X = (np.stack(z, axis=1) - sur.mu_in) / sur.sd_in
            Yn, cache = mlp.forward(sur.Ws, sur.bs, X, bf16=bf16, keep=True)
            Y = Yn * sur.sd_out + sur.mu_out
            tape.append(("stage", sur, cache))
            z = [Y[:, j].copy() for j in range(6)]
            gamma_ref = gamma_out
        else:
            bg = math.sqrt(gamma_ref * gamma_ref - 1.0)
            M = maps.element_matrix(e, bg)
            dM = maps.dquad_dk(e["L"], e["k"], bg) if e["kind"] == "quad" else None
            tape.append(("linear", M, dM, z))
            z = apply_matrix(M, z)
    J, lam = seed(z, gamma_ref, which)
    grads = []
    for rec in reversed(tape):
        if rec[0] == "linear":
            _, M, dM, zin = rec
            if dM is not None:
                dz = apply_matrix(dM, zin)
                grads.append(math.fsum(np.concatenate([l * d for l, d in zip(lam, dz)])))
            L = np.stack(lam)
            lam = list(M.T @ L)
        else:
            _, sur, cache = rec
            dYn = np.stack(lam, axis=1) * sur.sd_out
            dX, _, _ = mlp.backward(sur.Ws, cache, dYn)
            lin = dX / sur.sd_in
            lam = [lin[:, j].copy() for j in range(6)]
    grads.reverse()
    return J, np.array(grads)


def track_objective(z, gamma_ref, elements, which, bf16=False):
    """J of the final particles (forward only), for finite differences."""
    from .beamline import track
    zo, go, _ = track(z, gamma_ref, elements, snapshots=False, bf16=bf16)
    return objective(moments.moments28(zo), go, which)
