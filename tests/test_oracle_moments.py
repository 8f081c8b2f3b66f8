"""Pins of the oracle's beam moments (not GPU)."""
import math
from fractions import Fraction

import numpy as np

from oracle import maps, moments
from synth.bunch import BunchRecipe, gaussian_bunch


def _exact28(z):
    cols = [[Fraction(float(v)) for v in c] for c in z]
    n = len(cols[0])
    mean = [sum(c) / n for c in cols]
    out = [Fraction(n)] + mean
    for a, b in moments.PAIRS:
        out.append(sum((cols[a][i] - mean[a]) * (cols[b][i] - mean[b]) for i in range(n)) / n)
    return out


def test_moments_exact_rational():
    rng = np.random.default_rng(0)
    z = [rng.normal(size=41).astype(np.float32) * 10.0 ** e for e in (-6, -4, -6, -4, -6, -2)]
    z[4] += np.float32(3e-5)          # offset mean: central moments must still be exact
    m = moments.moments28(z)
    ex = _exact28(z)
    for a, b in zip(m[:7], ex[:7]):
        assert abs(a - float(b)) <= 2e-16 * abs(float(b))
    diag = {a: float(ex[7 + j]) for j, (a, b) in enumerate(moments.PAIRS) if a == b}
    for j, (a, b) in enumerate(moments.PAIRS):
        scale = math.sqrt(diag[a] * diag[b])
        assert abs(m[7 + j] - float(ex[7 + j])) <= 1e-15 * scale


def test_shift_invariance():
    rng = np.random.default_rng(1)
    z = [rng.normal(size=1000) for _ in range(6)]
    m0 = moments.moments28(z)
    m1 = moments.moments28([c + 5.0 for c in z])
    assert np.max(np.abs(m1[7:] - m0[7:])) < 1e-13
    assert np.max(np.abs(m1[1:7] - m0[1:7] - 5.0)) < 1e-14


def test_generator_moments_and_derived_quantities():
    r = BunchRecipe(n=200_000, seed=2)
    z, g = gaussian_bunch(r)
    zz = [z[k] for k in ("x", "px", "y", "py", "t", "pt")]
    d = moments.derived(moments.moments28(zz), g)
    n = r.n
    assert abs(d["eps_n_x"] / 1e-6 - 1) < 10 / math.sqrt(n)
    assert abs(d["eps_n_y"] / 1e-6 - 1) < 10 / math.sqrt(n)
    assert abs(d["sigma_x"] / 2e-6 - 1) < 5 / math.sqrt(n)
    assert abs(d["rel_energy_spread"] / 0.01 - 1) < 5 / math.sqrt(n)
    # energy spread and emittance from per-particle absolute quantities
    bg = math.sqrt(g * g - 1)
    gam = g - zz[5] * bg
    assert abs(d["rel_energy_spread"] - gam.std() / gam.mean()) < 1e-12
    ux = zz[1] * bg
    x = zz[0]
    e = math.sqrt(np.mean((x - x.mean()) ** 2) * np.mean((ux - ux.mean()) ** 2)
                  - np.mean((x - x.mean()) * (ux - ux.mean())) ** 2)
    assert abs(d["eps_n_x"] / e - 1) < 1e-10


def test_empty_bunch():
    m = moments.moments28([np.zeros(0)] * 6)
    assert m[0] == 0 and np.all(m == 0)


def test_sigma_propagation_equals_direct():
    z, g = gaussian_bunch(BunchRecipe(n=3000, seed=4))
    Z = np.stack([z[k] for k in ("x", "px", "y", "py", "t", "pt")])
    bg = math.sqrt(g * g - 1)
    M = maps.quad(0.1, 31.67, bg) @ maps.sbend(0.2, 1e-3, bg) @ maps.drift(0.5, bg)
    m0 = moments.moments28(Z)
    m1 = moments.moments28(M @ Z)
    S1 = M @ moments.sigma_matrix(m0) @ M.T
    assert np.max(np.abs(moments.sigma_matrix(m1) - S1) / np.sqrt(np.outer(np.diag(S1), np.diag(S1)))) < 1e-12
    assert np.max(np.abs(m1[1:7] - M @ m0[1:7])) < 1e-18
