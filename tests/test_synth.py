"""Seeded input generators: Philox known answers and the bunch recipes."""
import os

import numpy as np

from synth.philox import philox4x32_10, normal_pairs
from synth.bunch import BunchRecipe, gaussian_bunch, training_population, uneven_counts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        out = philox4x32_10(*v[:4], v[4], v[5])
        assert [int(o) for o in out] == v[6:]


def test_normals_statistics():
    a, b = normal_pairs(7, np.arange(200_000, dtype=np.uint64), 3)
    for z in (a, b):
        assert abs(z.mean()) < 5 / np.sqrt(z.size)
        assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert abs(np.mean(a * b)) < 5 / np.sqrt(a.size)


def test_design_bunch_recipe():
    r = BunchRecipe(n=100_000, seed=0)
    z, g = gaussian_bunch(r)
    bg = np.sqrt(g * g - 1)
    assert abs(g - 1957.9511835591836) < 1e-9
    n = r.n
    tol = lambda s: 6 * s / np.sqrt(n)
    assert abs(z["x"].std() - 2e-6) < 2 * tol(2e-6)
    assert abs(z["px"].std() - 1e-6 / (2e-6 * bg)) < 2 * tol(1e-6 / (2e-6 * bg))
    assert abs(z["pt"].std() - 0.01 * g / bg) < 2 * tol(0.01 * g / bg)
    st = 299792458.0 * 10e-15
    assert np.abs(z["t"]).max() <= 3 * st * (1 + 1e-15)
    # truncation at 3 sigma leaves 0.9733 of the variance
    assert abs(z["t"].std() / st - 0.98658) < 0.01


def test_subsets_regenerate_identically():
    a, _ = normal_pairs(3, np.arange(10, 20, dtype=np.uint64), 1)
    b, _ = normal_pairs(3, np.arange(0, 30, dtype=np.uint64), 1)
    assert np.array_equal(a, b[10:20])


def test_training_population_and_counts():
    z, p = training_population(4, 1000, 2000.0, 3e-6, seed=5)
    assert z["x"].size == 4000
    assert np.all((p["eps_n"] >= 0.5e-6) & (p["eps_n"] <= 2e-6))
    for b in range(4):
        tb = z["t"][b * 1000:(b + 1) * 1000]
        assert abs(tb.mean() - p["t_shift"][b]) < 1e-6
    c = uneven_counts(256, seed=0)
    assert c.min() >= 10_000 and c.max() <= 1_000_000
