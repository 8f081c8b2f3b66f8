"""Pins of the oracle's surrogate-with-fallback stage: particles outside a
surrogate's training-input box are pushed by the plain RK4 stage, the others
mapped by the network, and the box test is inclusive at its edges."""
import numpy as np

from oracle import beamline, mlp, wake
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init

KEYS = ("x", "px", "y", "py", "t", "pt")


def _setup(n=400):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=21))
    z = [z[k] for k in KEYS]
    Ws, bs = mlp_init([6, 16, 16, 6], 3)
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    return z, g, Ws, bs, mu, sd


def test_outside_particles_take_the_plain_push():
    z, g, Ws, bs, mu, sd = _setup()
    lo, hi = mu - 1.5 * sd, mu + 1.5 * sd
    sur = mlp.Surrogate(Ws, bs, mu, sd, mu, sd, domain=(lo, hi))
    st = lattice.plasma(50)
    st["surrogate"] = sur
    zo, go, _ = beamline.track(z, g, [st], snapshots=False)
    inside = sur.in_domain(z)
    assert 0 < inside.sum() < len(inside)
    want_in = mlp.Surrogate(Ws, bs, mu, sd, mu, sd).apply([c[inside] for c in z])
    want_out, _ = wake.push_stage([c[~inside] for c in z], g, beamline.stage_of(st))
    for c in range(6):
        assert np.array_equal(zo[c][inside], want_in[c])
        assert np.array_equal(zo[c][~inside], want_out[c])
    # the reference energy follows the stage either way
    assert go == wake.reference_exit(beamline.stage_of(st), g)[0]


def test_no_domain_is_the_plain_surrogate_and_edges_are_inside():
    z, g, Ws, bs, mu, sd = _setup(50)
    st = lattice.plasma(50)
    st["surrogate"] = mlp.Surrogate(Ws, bs, mu, sd, mu, sd)
    zo, _, _ = beamline.track(z, g, [st], snapshots=False)
    want = mlp.Surrogate(Ws, bs, mu, sd, mu, sd).apply(z)
    assert all(np.array_equal(a, b) for a, b in zip(zo, want))
    lo = np.array([np.min(c) for c in z])
    hi = np.array([np.max(c) for c in z])
    assert mlp.Surrogate(Ws, bs, mu, sd, mu, sd, domain=(lo, hi)).in_domain(z).all()
    assert not mlp.Surrogate(Ws, bs, mu, sd, mu, sd, domain=(lo, np.nextafter(hi, -np.inf))).in_domain(z).all()
