"""Physical constants (CODATA 2018) and derived plasma-wake scales.

The wake scales follow the plasma-stage model of the method: the plasma
wavenumber k_p = omega_p / c of a plasma of electron density n0 (Sec. 4,
staged laser-plasma accelerator), and the field amplitude expressed as an
inverse length g = e E0 / (m_e c^2).
"""
import math

C = 299792458.0                      # m/s
E_CHARGE = 1.602176634e-19           # C
EPS0 = 8.8541878128e-12              # F/m
M_E = 9.1093837015e-31               # kg
MEC2_MEV = 0.51099895000             # electron rest energy [MeV]
MEC2_EV = MEC2_MEV * 1.0e6


def plasma_kp(n0_cm3):
    """Plasma wavenumber [1/m] for electron density n0 [1/cm^3]."""
    n0 = n0_cm3 * 1.0e6
    omega_p = math.sqrt(n0 * E_CHARGE * E_CHARGE / (EPS0 * M_E))
    return omega_p / C


def field_g(E0_Vpm):
    """Field amplitude as an inverse length, e E0 / (m_e c^2) [1/m]."""
    return E0_Vpm / MEC2_EV
