"""GPU parity: moments, linear segment maps, stage pusher and full tracking
against the FP64 oracle on identical seeded inputs."""
import math

import numpy as np
import pytest

from gpu_util import KEYS, as_f32, from_bunch, to_bunch
from oracle import beamline, maps, moments, wake
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_17248_gb300 import bl
    bl.lib()


def _bunch(n, seed=0):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return [z[k] for k in KEYS], g


def _cmp_moments(got, want, tol):
    """Moments agree to tol relative to the beam's own scales."""
    assert got[0] == want[0]
    if want[0] == 0:
        assert np.all(got == 0)
        return 0.0
    S = moments.sigma_matrix(want)
    sd = np.sqrt(np.maximum(np.diag(S), 1e-300))
    err = 0.0
    for a in range(6):
        err = max(err, abs(got[1 + a] - want[1 + a]) / sd[a])
    for j, (a, b) in enumerate(moments.PAIRS):
        err = max(err, abs(got[7 + j] - want[7 + j]) / (sd[a] * sd[b]))
    assert err <= tol, err
    return err


@pytest.mark.parametrize("n", [1, 2, 127, 128, 129, 2047, 2048, 2049, 4095, 4096, 4097, 8191,
                               8192, 8193, 10000, (1 << 18) + 3])
def test_moments_fp32(n):
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(n, seed=n)
    z32 = as_f32(z)
    b = to_bunch(z32, g)
    got = bl.bl_moments(b)[0]
    want = moments.moments28(z32)
    if n > 1:
        _cmp_moments(got, want, 1e-10)
    else:
        assert got[0] == 1 and np.allclose(got[1:7], want[1:7], rtol=1e-12, atol=0)


def test_moments_fp64_and_offset_mean():
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(30001, seed=5)
    z[4] = z[4] + 4e-5   # large centroid offset relative to sigma_t
    b = to_bunch(z, g, dtype="f64")
    _cmp_moments(bl.bl_moments(b)[0], moments.moments28(z), 1e-10)
    z32 = as_f32(z)
    _cmp_moments(bl.bl_moments(to_bunch(z32, g))[0], moments.moments28(z32), 1e-10)


def test_moments_many_bunches_with_empty_and_tiny():
    from paper_2402_17248_gb300 import bl
    counts = [0, 1, 5000, 0, 3, 4096, 12345, 0, 2, 70000, 1]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    z, g = _bunch(int(off[-1]), seed=9)
    z32 = as_f32(z)
    got = bl.bl_moments(to_bunch(z32, g, offsets=off))
    for i, c in enumerate(counts):
        want = moments.moments28([a[off[i]:off[i + 1]] for a in z32])
        if c > 1:
            _cmp_moments(got[i], want, 1e-10)
        else:
            assert got[i][0] == c


def test_moments_growing_scale_and_outliers():
    """The FP32 sums keep per-coordinate power-of-two bounds that start at
    zero and are raised when a larger particle arrives: particles whose size
    grows 1e4-fold along the array, with outliers at ~1000 sigma and a
    centroid offset, still match the oracle."""
    from paper_2402_17248_gb300 import bl
    n = 300007
    z, g = _bunch(n, seed=21)
    rng = np.random.default_rng(21)
    grow = np.geomspace(1e-4, 1.0, n)
    z = [a * grow for a in z]
    for a in z:
        idx = rng.choice(n, 7, replace=False)
        a[idx] *= 1e3 * rng.choice([-1.0, 1.0], 7)
    z[1] = z[1] + 3.0 * z[1].std()
    z32 = as_f32(z)
    _cmp_moments(bl.bl_moments(to_bunch(z32, g))[0], moments.moments28(z32), 1e-10)


def test_moments_bunches_of_very_different_size():
    """Bounds restart at every bunch: a bunch 1e6 times smaller than the one
    before it is summed at its own scale."""
    from paper_2402_17248_gb300 import bl
    counts = [40000, 9000, 40000, 3, 20000]
    scale = [1.0, 1e-6, 1e3, 1.0, 1e-3]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    z, g = _bunch(int(off[-1]), seed=33)
    for i in range(len(counts)):
        for a in z:
            a[off[i]:off[i + 1]] *= scale[i]
    z32 = as_f32(z)
    got = bl.bl_moments(to_bunch(z32, g, offsets=off))
    for i in range(len(counts)):
        want = moments.moments28([a[off[i]:off[i + 1]] for a in z32])
        _cmp_moments(got[i], want, 1e-10)


def _segment(bg, k=lattice.DESIGN_K):
    M = np.eye(6)
    for e in lattice.matching_section(k):
        M = maps.element_matrix(e, bg) @ M
    return M


@pytest.mark.parametrize("dtype,n", [("f32", 129), ("f32", 100003), ("f64", 4097)])
def test_linear_segment(dtype, n):
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(n, seed=3)
    if dtype == "f32":
        z = as_f32(z)
    bg = math.sqrt(g * g - 1)
    M = _segment(bg)
    b = to_bunch(z, g, dtype=dtype)
    bl.bl_apply_linear(b, M)
    got = from_bunch(b)
    want = list(M @ np.stack(z))
    scale = [np.std(w) for w in want]
    err = max(float(np.max(np.abs(a - w))) / s for a, w, s in zip(got, want, scale))
    tol = 1e-5 if dtype == "f32" else 1e-12
    assert err < tol, err


def test_linear_per_bunch_matrices():
    from paper_2402_17248_gb300 import bl
    counts = [1000, 0, 4097, 3]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    z, g = _bunch(int(off[-1]), seed=4)
    z = as_f32(z)
    bg = math.sqrt(g * g - 1)
    Ms = np.stack([_segment(bg, (-20 - 10 * i, 30.0, -40.0 + i, 50.0)) for i in range(4)])
    b = to_bunch(z, g, offsets=off)
    bl.bl_apply_linear(b, Ms)
    got = from_bunch(b)
    for i in range(4):
        sl = slice(off[i], off[i + 1])
        want = Ms[i] @ np.stack([c[sl] for c in z])
        for a in range(6):
            if counts[i]:
                s = max(np.std(want[a]), np.max(np.abs(want[a])))
                assert np.max(np.abs(got[a][sl] - want[a])) <= 1e-5 * s


def test_pusher_fp64_config1_stage():
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(10000)
    st = lattice.plasma(200)
    b = to_bunch(z, g, dtype="f64")
    bl.bl_push_stage(b, st)
    got = from_bunch(b)
    want, g_out = wake.push_stage(z, g, wake.Stage(nsteps=200))
    assert abs(b.gamma_ref / g_out - 1) < 1e-13
    scale = [np.std(w) for w in want]
    errs = [float(np.max(np.abs(a - w))) / s for a, w, s in zip(got, want, scale)]
    print("fp64 pusher per-coordinate max err / rms:", errs)
    assert max(errs) < 1e-10


def test_pusher_fp32_400_steps():
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(20000, seed=1)
    z = as_f32(z)
    b = to_bunch(z, g)
    bl.bl_push_stage(b, lattice.plasma(400))
    got = from_bunch(b)
    want, g_out = wake.push_stage(z, g, wake.Stage(nsteps=400))
    scale = [np.std(w) for w in want]
    errs = [float(np.max(np.abs(a - w))) / s for a, w, s in zip(got, want, scale)]
    dg = moments.derived(moments.moments28(got), g_out)
    dw = moments.derived(moments.moments28(want), g_out)
    rel = {k: abs(dg[k] / dw[k] - 1) for k in dw}
    print("fp32 pusher per-coordinate max err / rms:", errs, "moments:", rel)
    assert max(rel.values()) < 1e-5
    # Per particle the FP32 error is a betatron phase error: each step turns
    # the particle by mu/N ~ 0.4 rad (mu up to ~160 rad over the stage), and
    # FP32 evaluation of that turn (plus the rounding of the wake phase
    # k_p t) is off by ~1e-7 relative, i.e. ~8e-8 rad per step. Over 400
    # steps that is at most ~3e-5 rad if every step erred the same way, and a
    # particle of betatron amplitude <= 4 rms then moves by <= 1.3e-4 rms
    # (measured: 1.1e-4). Hence 3e-4; the moments are held to 1e-5.
    assert max(errs) < 3e-4


def test_track_config1_fp64_moments_every_element():
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(10000)
    els = lattice.single_stage_transport(200)
    L = bl.Lattice(els)
    b = to_bunch(z, g, dtype="f64")
    mom, nonfin = bl.bl_track(b, L)
    assert nonfin == 0
    zo, go, snaps = beamline.track(z, g, els)
    assert abs(b.gamma_ref / go - 1) < 1e-13
    for e, (want, gr) in enumerate(snaps):
        _cmp_moments(mom[e][0], want, 1e-10)
    got = from_bunch(b)
    for a, w in zip(got, zo):
        assert np.max(np.abs(a - w)) <= 1e-10 * np.std(w)


def test_track_two_stage_beamline_fp32():
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(20000, seed=2)
    z = as_f32(z)
    els = lattice.staged_beamline(2, 400)
    L = bl.Lattice(els)
    b = to_bunch(z, g)
    mom, nonfin = bl.bl_track(b, L)
    zo, go, snaps = beamline.track(z, g, els)
    worst = 0.0
    for e, (want, gr) in enumerate(snaps):
        dg = moments.derived(mom[e][0], gr)
        dw = moments.derived(want, gr)
        for k in ("eps_n_x", "eps_n_y", "sigma_x", "sigma_y", "rel_energy_spread"):
            worst = max(worst, abs(dg[k] / dw[k] - 1))
    print("fp32 two-stage beamline worst relative moment error:", worst)
    assert worst < 1e-5


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_track_plasma_lens_section(dtype):
    """Stage, then drift + active plasma lens (k from a field gradient of
    3 kT/m) + drift + defocusing lens + drift: particles and moments after
    every element against the oracle (the lens map comes from the library's
    own element matrices)."""
    from paper_2402_17248_gb300 import bl, workflow
    z, g = _bunch(20001, seed=8)
    if dtype == "f32":
        z = as_f32(z)
    st = lattice.plasma(200)
    g1 = bl.bl_reference_exit(st, g)
    k_lens = workflow.plasma_lens_k(3000.0, g1)
    els = [st, lattice.drift(0.05), lattice.plasma_lens(0.03, k_lens), lattice.drift(0.1),
           lattice.plasma_lens(0.01, -0.3 * k_lens), lattice.drift(0.2)]
    b = to_bunch(z, g, dtype=dtype)
    mom, nonfin = bl.bl_track(b, bl.Lattice(els))
    assert nonfin == 0
    zo, go, snaps = beamline.track(z, g, els)
    tol = 1e-10 if dtype == "f64" else 1e-5
    for e, (want, gr) in enumerate(snaps):
        _cmp_moments(mom[e][0], want, tol)
    got = from_bunch(b)
    ptol = 1e-10 if dtype == "f64" else 3e-4  # FP32: phase error budget as the pusher test
    for a, w in zip(got, zo):
        assert np.max(np.abs(a - w)) <= ptol * np.std(w)


def test_nonfinite_particles_are_counted_and_kept():
    """NaN/inf-poisoned particles: bl_track reports them through the
    non-finite count at every reduction point, leaves them non-finite, and
    every other particle is tracked exactly as in a clean run."""
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(20000, seed=14)
    z = as_f32(z)
    bad = [5, 1234, 19999]
    zp = [c.copy() for c in z]
    zp[0][bad[0]] = np.nan
    zp[5][bad[1]] = np.inf
    zp[4][bad[2]] = -np.inf
    els = lattice.single_stage_transport(200)
    L = bl.Lattice(els)
    b = to_bunch(zp, g)
    mom, nf = bl.bl_track(b, L)
    R = bl.lib().bl_track_num_reductions(L.handle)
    assert nf == len(bad) * R
    got = from_bunch(b)
    assert all(not np.all(np.isfinite([c[i] for c in got])) for i in bad)
    c_ = to_bunch(z, g)
    bl.bl_track(c_, L)
    clean = from_bunch(c_)
    keep = np.ones(len(z[0]), dtype=bool)
    keep[bad] = False
    assert all(np.array_equal(a[keep], w[keep]) for a, w in zip(got, clean))


def test_injected_allocation_failure_is_reported_and_recovered():
    """A workspace allocation that fails (host-side injection) surfaces as
    BL_ERR_OOM from bl_track, and the library works normally afterwards."""
    import torch
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(5000, seed=15)
    z = as_f32(z)
    L = bl.Lattice(lattice.matching_section())
    s = torch.cuda.Stream()  # a stream whose work buffers do not exist yet
    with torch.cuda.stream(s):
        b = to_bunch(z, g)
        bl.bl_debug_fail_allocations(1)
        with pytest.raises(bl.BlError) as e:
            bl.bl_track(b, L, stream=s)
        assert e.value.status == bl.BL_ERR_OOM
        bl.bl_debug_fail_allocations(0)
        b = to_bunch(z, g)
        mom, nf = bl.bl_track(b, L, stream=s)
        s.synchronize()
    assert nf == 0
    ref = to_bunch(z, g)
    mref, _ = bl.bl_track(ref, L)
    assert np.array_equal(mom, mref)
    assert all(np.array_equal(a, w) for a, w in zip(from_bunch(b), from_bunch(ref)))


def test_fp32_stage_push_rejects_low_reference_energy():
    """The FP32 deviation form of the pusher expands gamma/u_z to second order
    in (1 + u_perp^2)/u_z^2; below gamma_ref = 400 at the stage entry the host
    refuses the FP32 push (an FP64 bunch takes it instead)."""
    import torch
    from paper_2402_17248_gb300 import bl
    z32 = [torch.zeros(64, dtype=torch.float32, device="cuda") for _ in range(6)]
    b = bl.Bunch(z32, 300.0)
    with pytest.raises(bl.BlError) as e:
        bl.bl_push_stage(b, lattice.plasma(10))
    assert e.value.status == bl.BL_ERR_INVALID_ARG
    z64 = [torch.zeros(64, dtype=torch.float64, device="cuda") for _ in range(6)]
    b64 = bl.Bunch(z64, 300.0)
    bl.bl_push_stage(b64, lattice.plasma(10))
    assert b64.gamma_ref > 300.0
