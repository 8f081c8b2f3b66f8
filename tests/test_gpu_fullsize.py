"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the 2^24-particle bunch through the 8-stage pusher and surrogate
beamlines (sampled particles against the oracle tracking the same particles
one by one, and the full final moments against the oracle's moments of the
same FP32 arrays), the 2^22-particle adjoint against central differences of
the GPU path itself, and 256 uneven bunches with per-bunch quads (sampled
particles of sampled bunches against the oracle with each bunch's own
strengths)."""
import numpy as np
import pytest

from gpu_util import KEYS, as_f32, from_bunch, to_bunch
from oracle import beamline, moments
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch, random_quad_magnitudes, uneven_counts

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
N_FULL = 1 << 24


@pytest.fixture(scope="module")
def full_bunch():
    from paper_2402_17248_gb300 import bl
    bl.lib()
    z, g = gaussian_bunch(BunchRecipe(n=N_FULL, seed=0))
    return as_f32([z[k] for k in KEYS]), g


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def test_fullsize_pusher_beamline(full_bunch):
    from paper_2402_17248_gb300 import bl
    z, g = full_bunch
    els = lattice.staged_beamline(8, 400)
    b = to_bunch(z, g)
    mom, nf = bl.bl_track(b, bl.Lattice(els))
    assert nf == 0
    got = from_bunch(b)
    idx = _sample(N_FULL, 512, 1)
    zo, go, _ = beamline.track([c[idx] for c in z], g, els, snapshots=False)
    assert abs(b.gamma_ref / go - 1) < 1e-12
    for a, w in zip(got, zo):
        err = np.max(np.abs(a[idx] - w)) / np.std(w)
        print("pusher beamline, sampled particles: max err / rms %.3e" % err)
        # FP32 deviation-form RK4: the per-stage phase error budget of the
        # 400-step test (1.3e-4 rms) over 8 stages, 1e-3 (measured 4.8e-4)
        assert err < 1.5e-3
    # moments of the whole final bunch: the library's reduction against the
    # oracle's moments of the same FP32 particles (1e-10), and bl_track's last
    # snapshot (entry reduction propagated in FP64 through the last segment)
    # against them (differs by the FP32 rounding of the map applied to the
    # particles)
    want = moments.moments28(got)
    S = moments.sigma_matrix(want)
    sd = np.sqrt(np.diag(S))

    def worst(m):
        return max(abs(m[7 + j] - want[7 + j]) / (sd[a] * sd[c])
                   for j, (a, c) in enumerate(moments.PAIRS))
    red = bl.bl_moments(b)[0]
    print("final second moments: reduction %.3e, propagated snapshot %.3e" %
          (worst(red), worst(mom[-1][0])))
    assert worst(red) < 1e-10
    assert worst(mom[-1][0]) < 1e-6


def test_fullsize_surrogate_beamline(full_bunch):
    from paper_2402_17248_gb300 import bl
    import test_gpu_beamline as tb
    z, g = full_bunch
    gpu, ora = tb._nets([c[:100000] for c in z], 8, 200)
    b = to_bunch(z, g)
    mom, nf = bl.bl_track(b, bl.Lattice(tb._beamline(8, gpu)))
    assert nf == 0
    got = from_bunch(b)
    idx = _sample(N_FULL, 512, 2)
    zo, go, _ = beamline.track([c[idx] for c in z], g, tb._beamline(8, ora), snapshots=False, bf16=True)
    for a, w in zip(got, zo):
        s_ = np.std(w)
        d = np.abs(a[idx] - w)
        print("surrogate beamline, sampled particles: median %.2e max %.2e of rms" %
              (np.median(d) / s_, np.max(d) / s_))
        # a BF16 rounding flip on the identity path moves a particle by one
        # BF16 ulp of its value; the rest agree to accumulation order
        assert np.mean(d <= 2e-3 * s_) > 0.99
        assert np.all(d <= 2e-3 * s_ + 8 * 2.0 ** -8 * np.abs(w))


def test_fullsize_adjoint_against_gpu_central_differences(full_bunch):
    from paper_2402_17248_gb300 import bl
    import test_gpu_beamline as tb
    z, g = full_bunch
    n = 1 << 22
    za = [c[:n] for c in z]
    gpu, _ = tb._nets(za[:6], 8, 300)
    els = tb._beamline(8, gpu)
    J, grad = bl.bl_track_grad(to_bunch(za, g), bl.Lattice(els), "sigma_x")
    g_out = bl.bl_reference_exit(lattice.plasma(400), g)
    for _ in range(7):
        g_out = bl.bl_reference_exit(lattice.plasma(400), g_out)
    qpos = [i for i, e in enumerate(els) if e["kind"] == "quad"]
    fd = []
    for qi in (0, 5, 18, 31):
        k = els[qpos[qi]]["k"]
        # two effects bound the agreement: the GPU forward rounds activations
        # to BF16, so J(k) is piecewise smooth at the scale of single-particle
        # rounding flips (noise ~1e-3 of the difference at this step), and the
        # O(h^2) truncation of the central difference (~4e-4 here: sigma_x
        # changes by ~0.6 % for a 1e-4 change of one k). The adjoint's
        # precision is pinned by the 10^4-particle oracle comparisons.
        h = 1e-4 * abs(k)
        v = []
        for sgn in (1, -1):
            e2 = [dict(e) for e in els]
            e2[qpos[qi]]["k"] = k + sgn * h
            m, _ = bl.bl_track(to_bunch(za, g), bl.Lattice(e2))
            v.append(bl.bl_beam_quantities(m[-1][0], g_out)["sigma_x"])
        fd.append((v[0] - v[1]) / (2 * h))
    fd = np.array(fd)
    ad = grad[0][[0, 5, 18, 31]]
    rel = np.max(np.abs(ad - fd)) / np.max(np.abs(fd))
    print("2^22 particles, dsigma_x/dk: adjoint vs GPU central differences %.3e" % rel)
    assert rel < 5e-3


def test_fullsize_batched_bunches(full_bunch):
    from paper_2402_17248_gb300 import bl
    import test_gpu_beamline as tb
    z, g = full_bunch
    nbunch = 256
    counts = uneven_counts(nbunch, 1.0e4, 1.0e6, seed=0)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    starts = np.random.default_rng(0).integers(0, N_FULL, size=nbunch)
    gidx = np.concatenate([(st + np.arange(c)) % N_FULL for st, c in zip(starts, counts)])
    zb = [c[gidx] for c in z]
    kmag = random_quad_magnitudes(nbunch, 32, 20.0, 80.0, seed=0)
    signs = np.array([-1.0, 1.0, -1.0, 1.0] * 8)
    gpu, ora = tb._nets([c[:100000] for c in z], 8, 400)

    def with_k(nets, per_bunch=None, b=None):
        out = tb._beamline(8, nets)
        q = 0
        for e in out:
            if e["kind"] == "quad":
                if per_bunch:
                    e["per_bunch_k"] = (signs[q] * kmag[:, q]).copy()
                else:
                    e["k"] = float(signs[q] * kmag[b, q])
                q += 1
        return out

    b = to_bunch(zb, g, offsets=off)
    mom, nf = bl.bl_track(b, bl.Lattice(with_k(gpu, per_bunch=True), n_bunch_k=nbunch))
    got = from_bunch(b)
    worst = 0.0
    for bi in (0, 17, 128, 255):
        rows = off[bi] + _sample(counts[bi], 64, bi)
        zo, _, _ = beamline.track([c[rows] for c in zb], g, with_k(ora, b=bi), snapshots=False,
                                  bf16=True)
        for a, w in zip(got, zo):
            s_ = max(np.std(w), 1e-300)
            d = np.abs(a[rows] - w)
            worst = max(worst, float(np.median(d) / s_))
            assert np.mean(d <= 2e-3 * s_) > 0.95
    print("batched, sampled bunches: worst median error %.3e of rms" % worst)
    assert worst < 1e-4
