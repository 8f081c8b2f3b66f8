"""Beamline recipes of the tracked workloads, as plain element lists.

Element dicts: {'kind': 'drift', 'L'}, {'kind': 'quad', 'L', 'k'} (k > 0
focuses x), {'kind': 'sbend', 'L', 'angle'}, {'kind': 'plasma', 'L',
'nsteps', 'n0_cm3', 'E0_Vpm', 'phi0'}. Lengths in m, k in 1/m^2, angles in
rad, density in 1/cm^3, field in V/m.
"""
import math

PHI0 = math.pi / 4.0
N0_CM3 = 1.0e17
E0_VPM = 10.0e9
STAGE_L = 0.3

# Quadrupole strengths of the matching section (x-focusing positive), from an
# FP64 least-squares match of the stage-exit Twiss functions back to the
# matched beta of the next stage.
DESIGN_K = (-35.52, 31.67, -31.75, 35.70)
CHICANE_ANGLE = 1.0e-3
DIPOLE_L = 0.2


def plasma(nsteps, L=STAGE_L):
    return {"kind": "plasma", "L": L, "nsteps": nsteps, "n0_cm3": N0_CM3,
            "E0_Vpm": E0_VPM, "phi0": PHI0}


def drift(L):
    return {"kind": "drift", "L": L}


def quad(L, k):
    return {"kind": "quad", "L": L, "k": k}


def sbend(L, angle):
    return {"kind": "sbend", "L": L, "angle": angle}


def plasma_lens(L, k):
    return {"kind": "plasma_lens", "L": L, "k": k}


def single_stage_transport(nsteps=200):
    """One plasma stage, then drift 0.5 m, four 0.1 m quads (k = +-50), drift 0.5 m."""
    return [plasma(nsteps), drift(0.5), quad(0.1, 50.0), quad(0.1, -50.0),
            quad(0.1, 50.0), quad(0.1, -50.0), drift(0.5)]


def chicane(angle=CHICANE_ANGLE, Lb=DIPOLE_L, gap=0.25):
    return [sbend(Lb, angle), drift(gap), sbend(Lb, -angle), drift(gap),
            sbend(Lb, -angle), drift(gap), sbend(Lb, angle)]


def matching_section(k=DESIGN_K):
    """Drift, two quads, four-dipole chicane, two quads, drift (17 elements)."""
    return ([drift(0.5), quad(0.1, k[0]), drift(0.1), quad(0.1, k[1]), drift(0.1)]
            + chicane()
            + [drift(0.1), quad(0.1, k[2]), drift(0.1), quad(0.1, k[3]), drift(0.5)])


def staged_beamline(n_stages=8, nsteps=400, k=DESIGN_K):
    """n_stages x (plasma stage + matching section)."""
    out = []
    for _ in range(n_stages):
        out.append(plasma(nsteps))
        out.extend(matching_section(k))
    return out
