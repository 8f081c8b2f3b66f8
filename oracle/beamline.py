"""Tracking through a beamline of linear elements and plasma stages (FP64).

The beamline is a sequence of elements, each a per-particle map applied in
turn (Sec. 2: conventional elements and plasma elements combined in one
s-based simulation; Sec. 4: repeated plasma stages joined by transport).
Plasma stages are either the prescribed-wake RK4 push or an MLP surrogate of
that stage (Sec. 4.3: surrogates incorporated into the tracking loop).
Moments are taken from the particles after every element (Sec. 4: moments
after each stage; here after every element).

Elements are dicts: {'kind': 'drift'|'quad'|'sbend'|'plasma_lens', 'L', 'k',
'angle'} or {'kind': 'plasma', 'L', 'nsteps', 'n0_cm3', 'E0_Vpm', 'phi0',
'surrogate': oracle.mlp.Surrogate or None}.

A surrogate with a training domain maps only the particles inside it; the
others are pushed through the stage by the plain RK4 method, the surrogate's
fallback (the learned map is trusted only where it was trained).
"""
import numpy as np

from . import maps, moments, wake


def stage_of(e):
    return wake.Stage(L=e["L"], nsteps=e["nsteps"], n0_cm3=e["n0_cm3"],
                      E0_Vpm=e["E0_Vpm"], phi0=e["phi0"])


def apply_matrix(M, z):
    """z_out = M z for every particle."""
    Zo = M @ np.stack(z)
    return [Zo[i].copy() for i in range(6)]


def track(z, gamma_ref, elements, snapshots=True, bf16=False):
    """Track particles z (6 arrays) starting at reference gamma_ref.

    Returns (z_out, gamma_out, list of (moments28, gamma_ref) after each element).
    """
    z = [np.asarray(c, dtype=np.float64).copy() for c in z]
    snaps = []
    for e in elements:
        if e["kind"] == "plasma":
            st = stage_of(e)
            sur = e.get("surrogate")
            gamma_out, _, _ = wake.reference_exit(st, gamma_ref)
            if sur is None:
                z, gamma_ref = wake.push_stage(z, gamma_ref, st)
            else:
                inside = sur.in_domain(z)
                zs = sur.apply(z, bf16=bf16)
                if not inside.all():
                    out = ~inside
                    zp, _ = wake.push_stage([c[out] for c in z], gamma_ref, st)
                    for c in range(6):
                        zs[c][out] = zp[c]
                z = zs
                gamma_ref = gamma_out
        else:
            bg = np.sqrt(gamma_ref * gamma_ref - 1.0)
            z = apply_matrix(maps.element_matrix(e, bg), z)
        if snapshots:
            snaps.append((moments.moments28(z), gamma_ref))
    return z, gamma_ref, snaps
