"""Bunch recipes of the tracked workloads, drawn from Philox normals.

Coordinates are the six relative phase-space coordinates used throughout the
library: x, y [m]; px = p_x/p_ref, py = p_y/p_ref; t = c * (arrival-time
offset) [m]; pt = -(gamma - gamma_ref)/(beta*gamma)_ref. The recipe only
fixes the distribution (independent Gaussians at a waist, zero means unless a
centroid shift is requested, t truncated at +-3 sigma by resampling); it does
no tracking arithmetic.
"""
from dataclasses import dataclass

import numpy as np

from .philox import normal_pairs, uniforms

ELECTRON_REST_MEV = 0.51099895000        # CODATA 2018
C_LIGHT = 299792458.0


def gamma_from_kinetic_gev(e_kin_gev):
    """Lorentz factor of an electron with the given kinetic energy."""
    return 1.0 + e_kin_gev * 1.0e3 / ELECTRON_REST_MEV


@dataclass
class BunchRecipe:
    """A 6D Gaussian bunch at a waist, relative to the reference particle."""
    n: int = 10_000
    e_kin_gev: float = 1.0          # reference kinetic energy
    eps_n: float = 1.0e-6           # normalised emittance, both planes [m]
    sigma_x: float = 2.0e-6         # both planes [m]
    sigma_t_s: float = 10.0e-15     # rms duration [s]
    rel_energy_spread: float = 0.01
    t_cut_sigma: float = 3.0        # |t| truncation in units of sigma_t
    seed: int = 0
    first_index: int = 0            # Philox index of the first particle (for shards)

    @property
    def gamma_ref(self):
        return gamma_from_kinetic_gev(self.e_kin_gev)


def _truncated_pair(seed, idx, stream, cut):
    """Normal pair for (seed, idx, stream) with |first| <= cut by resampling."""
    a, b = normal_pairs(seed, idx, stream, 0)
    bad = np.abs(a) > cut
    attempt = 1
    while bad.any():
        if attempt > 64:
            raise RuntimeError("truncated normal did not converge")
        ra, rb = normal_pairs(seed, idx[bad], stream, attempt)
        a[bad] = ra
        b[bad] = rb
        bad = np.abs(a) > cut
        attempt += 1
    return a, b


def _draw(n, seed, first_index, sx, spx, st, spt, cut, t_shift=None, chunk=1 << 21):
    out = {k: np.empty(n, dtype=np.float64) for k in ("x", "px", "y", "py", "t", "pt")}
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        idx = np.arange(first_index + lo, first_index + hi, dtype=np.uint64)
        zx, zpx = normal_pairs(seed, idx, 0)
        zy, zpy = normal_pairs(seed, idx, 1)
        zt, zpt = _truncated_pair(seed, idx, 2, cut)
        sl = slice(lo, hi)
        out["x"][sl] = zx * (sx[sl] if np.ndim(sx) else sx)
        out["px"][sl] = zpx * (spx[sl] if np.ndim(spx) else spx)
        out["y"][sl] = zy * (sx[sl] if np.ndim(sx) else sx)
        out["py"][sl] = zpy * (spx[sl] if np.ndim(spx) else spx)
        out["t"][sl] = zt * (st[sl] if np.ndim(st) else st)
        out["pt"][sl] = zpt * (spt[sl] if np.ndim(spt) else spt)
        if t_shift is not None:
            out["t"][sl] += t_shift[sl]
    return out


def gaussian_bunch(recipe: BunchRecipe):
    """Draw the recipe's bunch; returns (dict of float64 arrays, gamma_ref)."""
    g = recipe.gamma_ref
    bg = np.sqrt(g * g - 1.0)
    spx = recipe.eps_n / (recipe.sigma_x * bg)
    st = C_LIGHT * recipe.sigma_t_s
    spt = recipe.rel_energy_spread * g / bg
    z = _draw(recipe.n, recipe.seed, recipe.first_index, recipe.sigma_x, spx, st, spt,
              recipe.t_cut_sigma)
    return z, g


def training_population(n_bunches, per_bunch, gamma_ref, t_shift_max, seed=1000,
                        eps_range=(0.5e-6, 2.0e-6), spread_range=(0.005, 0.02),
                        sigma_x=2.0e-6, sigma_t_s=10.0e-15, t_cut_sigma=3.0):
    """Bunches with randomised emittance, energy spread and centroid in t.

    Per bunch b: eps ~ U(eps_range), relative energy spread ~ U(spread_range),
    centroid shift in t ~ U(-t_shift_max, t_shift_max) (the caller converts an
    injection-phase jitter into a length). Particles of bunch b occupy
    indices [b*per_bunch, (b+1)*per_bunch). Returns (dict of arrays, params).
    """
    bg = np.sqrt(gamma_ref * gamma_ref - 1.0)
    bidx = np.arange(n_bunches, dtype=np.uint64)
    u0, u1 = uniforms(seed, bidx, 100)
    u2, _ = uniforms(seed, bidx, 101)
    eps = eps_range[0] + (eps_range[1] - eps_range[0]) * u0
    spread = spread_range[0] + (spread_range[1] - spread_range[0]) * u1
    shift = t_shift_max * (2.0 * u2 - 1.0)
    n = n_bunches * per_bunch
    rep = lambda a: np.repeat(a, per_bunch)
    spx = rep(eps / (sigma_x * bg))
    spt = rep(spread * gamma_ref / bg)
    st = C_LIGHT * sigma_t_s
    z = _draw(n, seed, 0, sigma_x, spx, st, spt, t_cut_sigma, t_shift=rep(shift))
    return z, {"eps_n": eps, "rel_energy_spread": spread, "t_shift": shift}


def uneven_counts(n_bunches=256, lo=1.0e4, hi=1.0e6, seed=0):
    """Particle counts floor(exp(U[ln lo, ln hi])) per bunch."""
    u, _ = uniforms(seed, np.arange(n_bunches, dtype=np.uint64), 200)
    return np.floor(np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)).astype(np.int64)


def random_quad_magnitudes(n_bunches, n_quads, lo=20.0, hi=80.0, seed=0):
    """|k| ~ U[lo, hi] per (bunch, quad); signs are the lattice's business."""
    idx = np.arange(n_bunches * n_quads, dtype=np.uint64)
    u, _ = uniforms(seed, idx, 300)
    return (lo + (hi - lo) * u).reshape(n_bunches, n_quads)


def mlp_init(widths, seed, first_layer_scale=None, first_bias_range=None):
    """Weights W[l] (out x in) and biases b[l] ~ U(+-1/sqrt(fan_in)), float64.

    first_layer_scale: optional per-input scale factors for W[0]'s columns;
    first_bias_range: optional r for b[0] ~ U(+-r) (its own Philox stream).
    Together they spread the first layer's units over a wider range of an
    input, e.g. so that a map oscillating in that input is resolvable."""
    Ws, bs = [], []
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        bound = 1.0 / np.sqrt(fi)
        idx = np.arange(fo * fi + fo, dtype=np.uint64)
        u, _ = uniforms(seed, idx, 400 + l)
        v = bound * (2.0 * u - 1.0)
        Ws.append(v[: fo * fi].reshape(fo, fi))
        bs.append(v[fo * fi:])
    if first_layer_scale is not None:
        Ws[0] = Ws[0] * np.asarray(first_layer_scale, dtype=np.float64)[None, :]
    if first_bias_range is not None:
        u, _ = uniforms(seed, np.arange(widths[1], dtype=np.uint64), 450)
        bs[0] = first_bias_range * (2.0 * u - 1.0)
    return Ws, bs
