"""bl_track_host: a bunch held in host memory, streamed through the GPU in
chunks (copies on their own streams, two compute streams), against bl_track
on a device copy of the same bunch. The particles must agree bit for bit
(same kernels, particle by particle); the whole-bunch moments are pooled from
the chunks' moments in FP64 and agree with bl_track's up to rounding order."""
import numpy as np
import pytest

from gpu_util import KEYS, from_bunch, to_bunch
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init

pytestmark = pytest.mark.gpu
WIDTHS = [6, 128, 128, 128, 128, 6]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_17248_gb300 import bl
    bl.lib()


def _bunch(n, seed):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return [np.asarray(z[k], dtype=np.float32) for k in KEYS], g


def _beamline(z, single_stage=False, lead_section=False):
    """surrogate stage (with a training box that leaves ~10 % of the
    particles to the fallback pusher) + matching section + pusher stage +
    matching section; single_stage: the surrogate stage and its section only
    (bl_track_host then streams every chunk through the whole lattice
    instead of keeping the bunch on the device between the first and the
    last stage)"""
    from paper_2402_17248_gb300 import bl
    Z = np.stack(z, axis=1).astype(np.float64)
    mu, sd = np.nanmean(Z, axis=0), np.nanstd(Z, axis=0)
    Ws, bs = mlp_init(WIDTHS, 5)
    sur = bl.Surrogate(Ws, bs, mu, sd, mu, sd)
    sur.set_domain(mu - 2.5 * sd, mu + 2.5 * sd)
    st = lattice.plasma(100)
    st["surrogate"] = sur
    els = [st] + lattice.matching_section()
    if not single_stage:
        els += [lattice.plasma(100)] + lattice.matching_section()
    if lead_section:  # linear elements before the first stage: a segment in the chunked head
        # (millimetres: the beam's beta function at the entrance is ~4 mm)
        els = [lattice.drift(0.001), lattice.quad(0.001, 5.0), lattice.drift(0.001)] + els
    lat = bl.Lattice(els)
    lat.elements = els
    return lat, sur


def _device_reference(z, g, lat):
    from paper_2402_17248_gb300 import bl
    b = to_bunch([c.astype(np.float64) for c in z], g)
    m, nf = bl.bl_track(b, lat)
    return [c.astype(np.float32) for c in from_bunch(b)], m, nf, b.gamma_ref


def _moments_close(a, b, lat, g, m_entry):
    """|a - b| <= 2e-10 x the entry's natural scale. Each side reduces the
    particles at a segment entry within the library's moment tolerance of
    1e-10 of the exact moments (float-float sums, grouped differently on the
    two sides), so the two reductions differ by at most 2e-10 sigma_a sigma_b
    there (N for the count, sigma_a for a mean). Both sides then propagate
    the reduced moments through the same FP64 element maps, so after
    elements with cumulative map M the difference is M dS M^T, bounded by
    2e-10 v_i v_j with v = |M| s (elementwise absolute value of M). The
    reductions accumulate raw sums of z_a z_b, whose float-float rounding is
    relative to |<z_a z_b>| <= (sigma_a + |mu_a|)(sigma_b + |mu_b|), so s is
    sigma + |mu| at the segment entry. m_entry: moments of the bunch at the
    lattice entrance (the reduction of a leading segment)."""
    from paper_2402_17248_gb300 import bl
    a, b = np.asarray(a)[:, 0], np.asarray(b)[:, 0]
    els = lat.elements
    diag = [7, 13, 18, 22, 25, 27]
    scale = np.empty_like(b)
    entry = np.asarray(m_entry)
    gam, first = g, 0
    for e, el in enumerate(els):
        if el["kind"] == "plasma":
            gam = bl.bl_reference_exit(el, gam)
            M = np.eye(6)
            entry, first = b[e], e + 1
        else:
            M = bl.bl_segment_matrix(els[first:e + 1], gam)
        v = np.abs(M) @ (np.sqrt(np.abs(entry[diag])) + np.abs(entry[1:7]))
        scale[e, 0] = b[e, 0]
        scale[e, 1:7] = v
        j = 7
        for p in range(6):
            for q in range(p, 6):
                scale[e, j] = v[p] * v[q]
                j += 1
    err = np.abs(a - b) / (scale + 1e-300)
    e, j = np.unravel_index(np.argmax(err), err.shape)
    print("pooled vs whole-bunch moments: max scaled difference %.2e (element %d, entry %d)"
          % (np.max(err), e, j))
    return np.all(err <= 2e-10)


# (n, chunk, single-stage lattice, linear elements before the first stage):
# whole-bunch mode with a ragged last chunk, with even chunks and with a
# segment in the chunked head; one chunk; the chunk-through mode
@pytest.mark.parametrize("n,chunk,single,lead", [(300_001, 65536, False, False),
                                                 (131_072, 32768, False, False),
                                                 (200_003, 65536, False, True),
                                                 (50_000, 0, False, False),
                                                 (300_001, 65536, True, False)])
def test_host_stream_matches_device(n, chunk, single, lead):
    import torch
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(n, seed=21)
    lat, _sur = _beamline(z, single, lead)
    want, m_dev, nf_dev, g_dev = _device_reference(z, g, lat)
    hin = [torch.from_numpy(c.copy()).pin_memory() for c in z]
    hout = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(6)]
    m, nf, g_out = bl.bl_track_host(hin, hout, g, lat, chunk=chunk)
    assert nf == nf_dev
    assert g_out == g_dev
    for a, w in zip(hout, want):
        assert np.array_equal(a.numpy(), w, equal_nan=True)
    finite = np.isfinite(m_dev)
    assert np.array_equal(np.isfinite(m), finite)
    assert _moments_close(np.where(finite, m, 0.0), np.where(finite, m_dev, 0.0), lat, g,
                          bl.bl_moments(to_bunch(z, g))[0])
    # the inputs are untouched when the output is separate
    assert all(np.array_equal(a.numpy(), c) for a, c in zip(hin, z))


def test_host_stream_in_place_pageable_and_nonfinite():
    """out aliasing in, plain (pageable) numpy arrays, and a planted NaN
    counted like bl_track counts it"""
    from paper_2402_17248_gb300 import bl
    n = 70_003
    z, g = _bunch(n, seed=22)
    z[3][12345] = np.float32("nan")
    lat, _sur = _beamline(z)
    want, m_dev, nf_dev, _ = _device_reference(z, g, lat)
    arr = [c.copy() for c in z]
    m, nf, _ = bl.bl_track_host(arr, arr, g, lat, chunk=20000)
    assert nf == nf_dev and nf > 0
    for a, w in zip(arr, want):
        assert np.array_equal(a, w, equal_nan=True)
    finite = np.isfinite(m_dev)
    assert np.array_equal(np.isfinite(m), finite)
    zc = [np.where(np.isfinite(c), c, 0.0).astype(np.float32) for c in z]
    assert _moments_close(np.where(finite, m, 0.0), np.where(finite, m_dev, 0.0), lat, g,
                          bl.bl_moments(to_bunch(zc, g))[0])


def test_host_stream_without_moments_and_repeat():
    """no moments requested; two calls in a row give the same particles"""
    import torch
    from paper_2402_17248_gb300 import bl
    n = 200_000
    z, g = _bunch(n, seed=23)
    lat, _sur = _beamline(z)
    want, _, _, g_dev = _device_reference(z, g, lat)
    hin = [torch.from_numpy(c.copy()).pin_memory() for c in z]
    for _ in range(2):
        hout = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(6)]
        m, nf, g_out = bl.bl_track_host(hin, hout, g, lat, chunk=40000, moments=False)
        assert m is None and nf is None and g_out == g_dev
        for a, w in zip(hout, want):
            assert np.array_equal(a.numpy(), w)
