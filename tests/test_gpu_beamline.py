"""GPU parity of the surrogate beamline paths: the adjoint bl_track_grad
against the FP64 oracle's reverse mode and finite differences, batched uneven
bunches with per-bunch quadrupoles through surrogate stages, and what a
network trained on the GPU gains over the plain pusher it replaces."""
import math
import time

import numpy as np
import pytest

from gpu_util import KEYS, as_f32, from_bunch, to_bunch
from oracle import adjoint, beamline, mlp, moments
from synth import lattice
from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init, training_population

pytestmark = pytest.mark.gpu
WIDTHS = [6, 128, 128, 128, 128, 6]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_17248_gb300 import bl
    bl.lib()


def _bunch(n, seed=0):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return as_f32([z[k] for k in KEYS]), g


def _near_identity(seed, eps):
    """Weights of F(z) = z + eps * (a random smooth map), exactly representable
    in BF16 on the identity path: hidden units 0..5 carry GELU(x) and 6..11
    carry GELU(-x), and GELU(x) - GELU(-x) = x for the tanh form as well."""
    Ws, bs = mlp_init(WIDTHS, seed)
    Ws = [eps * W for W in Ws]
    bs = [eps * b for b in bs]
    I6 = np.eye(6)
    Ws[0][:12, :] = np.vstack([I6, -I6])
    bs[0][:12] = 0.0
    for l in (1, 2, 3):
        Ws[l][:12, :] = 0.0
        Ws[l][:12, :12] = np.block([[I6, -I6], [-I6, I6]])
        bs[l][:12] = 0.0
    Ws[4][:, :12] = np.hstack([I6, -I6])
    return Ws, bs


def _nets(z, n_stages, seed, eps=0.05):
    """Test surrogates F(z) = z + eps * (random smooth map) (GPU handles and
    matching oracle objects)."""
    from paper_2402_17248_gb300 import bl
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    gpu, ora = [], []
    for s in range(n_stages):
        Ws, bs = _near_identity(seed + s, eps)
        gpu.append(bl.Surrogate(Ws, bs, mu, sd, mu, sd))
        Wr = [mlp.bf16_round(np.asarray(W, np.float32).astype(np.float64)) for W in Ws]
        br = [np.asarray(b, np.float32).astype(np.float64) for b in bs]
        ora.append(mlp.Surrogate(Wr, br, mu, sd, mu, sd))
    return gpu, ora


def _beamline(n_stages, nets, k=lattice.DESIGN_K):
    els = []
    for s in range(n_stages):
        st = lattice.plasma(400)
        st["surrogate"] = nets[s]
        els.append(st)
        els.extend(lattice.matching_section(k))
    return els


# (objective, network nonlinearity eps, tolerance on dJ/dk). Through a
# near-symplectic transport the normalised emittance is almost stationary in
# the focusing strengths: with eps = 0.05 networks its gradient is a residual
# set by the BF16 rounding of the hidden activations (the BF16 and FP64
# oracles differ in it by a factor 3.6), i.e. by individual rounding
# decisions, which FP32 accumulation order and tanh.approx move. With eps = 1
# the emittance gradient is the network's own nonlinearity (BF16 and FP64
# oracles agree to 2 %), and a 2^-16 relative perturbation of tanh moves it by
# at most 3.3e-3, hence 1e-2; sigma_x is well conditioned at both strengths.
ADJOINT_CASES = [("sigma_x", 0.05, 5e-3), ("sigma_x", 1.0, 5e-3),
                 ("eps_n_x", 1.0, 1e-2), ("eps_n_y", 1.0, 1e-2)]


@pytest.mark.parametrize("which,eps,tol", ADJOINT_CASES)
def test_adjoint_matches_oracle(which, eps, tol):
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(10000, seed=3)
    gpu, ora = _nets(z, 2, 40, eps)
    L = bl.Lattice(_beamline(2, gpu))
    b = to_bunch(z, g)
    J, grad = bl.bl_track_grad(b, L, which)
    Jo, go = adjoint.track_grad(z, g, _beamline(2, ora), which, bf16=True)
    rel = np.max(np.abs(grad[0] - go)) / np.max(np.abs(go))
    print("%s (eps %.2f): J gpu %.6e oracle %.6e; dJ/dk normwise rel err %.3e"
          % (which, eps, J[0], Jo, rel))
    assert abs(J[0] / Jo - 1) < 1e-5
    # the device VJP differentiates GELU through tanh.approx (relative error
    # ~2^-11 per evaluation) over 8 layers; the oracle uses exact tanh
    assert rel < tol


def test_adjoint_matches_finite_differences():
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(10000, seed=4)
    gpu, ora = _nets(z, 1, 60)
    els_o = _beamline(1, ora)
    L = bl.Lattice(_beamline(1, gpu))
    J, grad = bl.bl_track_grad(to_bunch(z, g), L, "sigma_x")
    fd = []
    for qi in range(4):
        idx = [i for i, e in enumerate(els_o) if e["kind"] == "quad"][qi]
        k = els_o[idx]["k"]
        h = 1e-6 * abs(k)
        vals = []
        for sgn in (1, -1):
            e2 = [dict(e) for e in els_o]
            e2[idx]["k"] = k + sgn * h
            vals.append(adjoint.track_objective(z, g, e2, "sigma_x", bf16=True))
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    rel = np.max(np.abs(grad[0] - fd)) / np.max(np.abs(fd))
    print("dJ/dk vs central differences of the oracle: normwise rel err %.3e" % rel)
    assert rel < 2e-3


def test_autograd_objective_matches_adjoint():
    """beam_objective (torch.autograd.Function over bl_track_grad): J and
    dJ/dk equal a direct bl_track_grad call, the caller's bunch is left
    untouched, a small step against the gradient lowers J, and per-bunch
    strengths give one gradient row per bunch."""
    import torch
    from paper_2402_17248_gb300 import bl
    from paper_2402_17248_gb300.grad import beam_objective
    z, g = _bunch(10000, seed=6)
    gpu, _ = _nets(z, 2, 40)
    els = _beamline(2, gpu)
    k0 = np.array([e["k"] for e in els if e["kind"] == "quad"])
    k = torch.tensor(k0, dtype=torch.float64, requires_grad=True)
    b = to_bunch(z, g)
    J = beam_objective(k, b, els, "sigma_x")
    J.sum().backward()
    J2, g2 = bl.bl_track_grad(to_bunch(z, g), bl.Lattice(els), "sigma_x")
    assert J.shape == (1,) and float(J.detach()[0]) == J2[0]
    assert np.array_equal(k.grad.numpy(), g2[0])
    assert all(np.array_equal(a, c) for a, c in zip(from_bunch(b), z))
    gk = k.grad.numpy()
    alpha = 0.01 * J2[0] / float(gk @ gk)
    with torch.no_grad():
        J_step = beam_objective(k - alpha * k.grad, b, els, "sigma_x")
    print("sigma_x %.6e -> %.6e after a step of 1%% predicted decrease" % (J2[0], float(J_step[0])))
    assert float(J_step[0]) < J2[0]
    # per-bunch strengths: two bunches, each with its own k
    off = np.array([0, 4000, 10000], dtype=np.int64)
    kb = torch.tensor(np.vstack([k0, 1.05 * k0]), dtype=torch.float64, requires_grad=True)
    Jb = beam_objective(kb, to_bunch(z, g, offsets=off), els, "eps_n_x")
    Jb.sum().backward()
    assert Jb.shape == (2,) and kb.grad.shape == (2, len(k0))
    for i in range(2):
        zi = [c[off[i]:off[i + 1]] for c in z]
        ei = [dict(e) for e in els]
        q = 0
        for e in ei:
            if e["kind"] == "quad":
                e["k"] = float(kb.detach()[i, q])
                q += 1
        Ji, gi = bl.bl_track_grad(to_bunch(zi, g), bl.Lattice(ei), "eps_n_x")
        assert abs(float(Jb.detach()[i]) / Ji[0] - 1) < 1e-9
        assert np.allclose(kb.grad[i].numpy(), gi[0], rtol=1e-6, atol=1e-9 * np.abs(gi[0]).max())


def test_batched_beamline_in_a_cuda_graph():
    """The batched uneven-bunch beamline (per-bunch quads, surrogate stages,
    per-bunch moments after every element) captured once as a CUDA graph with
    bl_track_async and replayed twice on fresh copies of the input: particles
    and moments bit-identical to eager bl_track."""
    import torch
    from paper_2402_17248_gb300 import bl
    counts = [30000, 7, 0, 12345, 4096, 1]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    z, g = _bunch(int(off[-1]), seed=9)
    gpu, _ = _nets(z, 2, 90)
    rng = np.random.default_rng(1)
    kq = rng.uniform(20, 80, size=(len(counts), 8)) * np.array([-1, 1, -1, 1] * 2)
    els = _beamline(2, gpu)
    qi = 0
    for e in els:
        if e["kind"] == "quad":
            e["per_bunch_k"] = kq[:, qi].copy()
            qi += 1
    L = bl.Lattice(els, n_bunch_k=len(counts))
    b_eager = to_bunch(z, g, offsets=off)
    m_eager, nf = bl.bl_track(b_eager, L)
    z_eager = from_bunch(b_eager)
    b = to_bunch(z, g, offsets=off)
    src = [c.clone() for c in b.coords]
    tg = bl.TrackGraph(b, L)
    for _ in range(2):
        for w, s0 in zip(b.coords, src):
            w.copy_(s0)
        tg.replay()
        m_graph, nf_graph = tg.moments()
        assert nf_graph == nf == 0
        assert np.array_equal(m_graph, m_eager)
        assert all(np.array_equal(a, c) for a, c in zip(from_bunch(b), z_eager))
    assert b.gamma_ref == b_eager.gamma_ref


def test_surrogate_domain_fallback_to_pusher():
    """A surrogate stage with a training-input box: particles inside are
    mapped by the network, the others pushed by the plain RK4 stage (the
    surrogate's fallback), against the oracle's hybrid stage."""
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(20000, seed=13)
    gpu, ora = _nets(z, 1, 95)
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    lo = (mu - 2.0 * sd).astype(np.float32).astype(np.float64)
    hi = (mu + 2.0 * sd).astype(np.float32).astype(np.float64)
    gpu[0].set_domain(lo, hi)
    ora[0].domain = (lo, hi)
    st_g = lattice.plasma(200)
    st_g["surrogate"] = gpu[0]
    st_o = dict(st_g, surrogate=ora[0])
    b = to_bunch(z, g)
    mom, nf = bl.bl_track(b, bl.Lattice([st_g]))
    got = from_bunch(b)
    zo, go, snaps = beamline.track(z, g, [st_o], bf16=True)
    inside = ora[0].in_domain(z)
    print("fallback particles: %d of %d" % ((~inside).sum(), len(inside)))
    assert 0.1 < (~inside).mean() < 0.5
    for a, w in zip(got, zo):
        s_ = np.std(w)
        # network side: the identity path of this test network carries the
        # input through BF16 activations, so a rare rounding flip moves a
        # particle by one BF16 ulp of its value (2^-8 relative)
        d_in = np.abs(a[inside] - w[inside])
        assert np.mean(d_in <= 2e-3 * s_) > 0.999
        assert np.all(d_in <= 2e-3 * s_ + 2.0 ** -7 * np.abs(w[inside]))
        assert np.max(np.abs(a[~inside] - w[~inside])) <= 1e-3 * s_  # FP32 vs FP64 RK4
    # the same stage without the domain maps everything with the network
    gpu[0].set_domain(None, None)
    b2 = to_bunch(z, g)
    bl.bl_track(b2, bl.Lattice([st_g]))
    got2 = from_bunch(b2)
    assert np.array_equal(got2[0][inside], got[0][inside])
    assert not np.allclose(got2[0][~inside], got[0][~inside], rtol=0, atol=1e-3 * np.std(zo[0]))


def test_batched_uneven_bunches_per_bunch_quads():
    """Bunches of uneven size stored back to back, each with its own quad
    strengths, through two surrogate stages in one bl_track call: bit-identical
    to tracking each bunch alone, and per-bunch moments after every element
    close to the oracle's."""
    from paper_2402_17248_gb300 import bl
    counts = [20000, 3, 0, 4097, 15000, 1]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    z, g = _bunch(int(off[-1]), seed=5)
    gpu, ora = _nets(z, 2, 80)
    rng = np.random.default_rng(0)
    kq = rng.uniform(20, 80, size=(len(counts), 8)) * np.array([-1, 1, -1, 1] * 2)

    def els_for(nets, per_bunch=None, b=None):
        out = _beamline(2, nets)
        qi = 0
        for e in out:
            if e["kind"] == "quad":
                if per_bunch is not None:
                    e["per_bunch_k"] = kq[:, qi].copy()
                else:
                    e["k"] = float(kq[b, qi])
                qi += 1
        return out

    L = bl.Lattice(els_for(gpu, per_bunch=True), n_bunch_k=len(counts))
    bb = to_bunch(z, g, offsets=off)
    mom, nonfin = bl.bl_track(bb, L)
    assert nonfin == 0
    got = from_bunch(bb)
    worst = worst_small = 0.0
    rms0, dpart = None, [[] for _ in range(6)]
    for b in range(len(counts)):
        sl = slice(off[b], off[b + 1])
        zb = [c[sl] for c in z]
        # the same bunch alone, scalar strengths: identical particles
        if counts[b]:
            single = to_bunch(zb, g)
            ms, _ = bl.bl_track(single, bl.Lattice(els_for(gpu, b=b)))
            alone = from_bunch(single)
            for a, w in zip(got, alone):
                assert np.array_equal(a[sl], w)
        # per-bunch moments after every element versus the FP64 oracle
        zo, go, snaps = beamline.track(zb, g, els_for(ora, b=b), bf16=True)
        for e, (want, gr) in enumerate(snaps):
            m = mom[e][b]
            assert m[0] == counts[b]
            if counts[b] > 1:
                S = moments.sigma_matrix(want)
                sd = np.sqrt(np.diag(S))
                for j, (p, q) in enumerate(moments.PAIRS):
                    d = abs(m[7 + j] - want[7 + j]) / (sd[p] * sd[q])
                    if counts[b] > 1000:
                        worst = max(worst, d)
                    else:
                        worst_small = max(worst_small, d)
        # and the particles themselves, one by one, scaled by the bunch's own
        # output rms (each bunch has its own quadrupoles); bunches of a few
        # particles take the first bunch's rms, having none of their own
        if counts[b]:
            if rms0 is None:
                rms0 = [np.std(c) for c in zo]
            for c in range(6):
                rms = np.std(zo[c]) if counts[b] >= 100 else rms0[c]
                d = np.abs(got[c][sl] - zo[c])
                dpart[c].append(d / rms)
    # a rounding flip of a BF16 activation moves a particle by a few BF16
    # ulps of a value of the order of the coordinate's spread (2^-8 x 4 sigma
    # per flip), and a flip in the first stage is carried through the second
    dall = [np.concatenate(v) for v in dpart]
    worst_particle = max(float(np.median(v)) for v in dall)
    largest = max(float(np.max(v)) for v in dall)
    within = min(float(np.mean(v <= 2e-3)) for v in dall)
    print("batched vs oracle: worst second-moment difference / (sd_a sd_b) %.3e (bunches "
          "> 1000 particles), %.3e (smaller); particles: worst median difference / rms %.3e, "
          "fraction within 2e-3 rms %.5f, largest %.2e" % (worst, worst_small, worst_particle,
                                                           within, largest))
    assert within >= 0.999
    assert largest <= 0.1
    # downstream stages quantise their inputs to BF16; particles whose FP32
    # input lies within rounding of a BF16 midpoint move by one BF16 ulp, so
    # a bunch of a few particles can move by a sizeable part of its spread
    # (measured 2e-5 on the large bunches)
    assert worst < 2e-4
    assert worst_small < 2e-3
    assert worst_particle < 1e-4


def test_trained_surrogate_gain_over_pusher():
    """A surrogate of a 15 GeV plasma stage, trained on the GPU from pusher
    pairs, replaces the 400-step RK4 push at a fraction of its cost, with the
    held-out exit beam's moments close to the pusher's."""
    import torch
    from paper_2402_17248_gb300 import bl, workflow
    kp = 59507.379801365234
    g0 = 1.0 + 15000.0 / 0.51099895
    zt, _ = training_population(16, 65536, g0, 0.2 / kp, seed=1001)
    pairs = workflow.stage_pairs(workflow.device_bunch(zt, g0), lattice.staged_beamline(1, 400))
    xin, xout, gin = pairs[0]
    sur, info = workflow.fit_surrogate(xin, xout, steps=6000, batch=4096, lr=2e-3, seed=5)
    print("15 GeV stage surrogate test loss %.3e" % info["test_loss"])
    ntrain = info["train_pairs"]
    test_in = xin[:, ntrain:].contiguous()
    st = lattice.plasma(400)
    def run(push):
        b = bl.Bunch([test_in[i].clone() for i in range(6)], gin)
        torch.cuda.synchronize()
        t = time.perf_counter()
        if push:
            bl.bl_push_stage(b, st)
        else:
            bl.bl_surrogate_apply(sur, b)
        torch.cuda.synchronize()
        return b, time.perf_counter() - t
    run(True), run(False)
    bp, tp = run(True)
    bs, ts = run(False)
    g_out = bl.bl_reference_exit(st, gin)
    qp = bl.bl_beam_quantities(bl.bl_moments(bp)[0], g_out)
    qs = bl.bl_beam_quantities(bl.bl_moments(bs)[0], g_out)
    err = {k: abs(qs[k] / qp[k] - 1) for k in ("eps_n_x", "eps_n_y", "rel_energy_spread", "sigma_x")}
    print("speedup %.1fx; relative moment differences %s" % (tp / ts, err))
    assert tp / ts > 5
    assert info["test_loss"] < 0.05
    # measured 6e-3 (emittances) and 4e-4 (energy spread) after this short
    # fit; the 8-stage beamline at the benchmark's training length is held
    # to 2e-3 in test_gpu_learned.py
    assert err["eps_n_x"] < 2e-2 and err["eps_n_y"] < 2e-2
    assert err["rel_energy_spread"] < 2e-3


@pytest.mark.parametrize("width", [3.5, 2.0, 0.7])
def test_fused_fallback_equals_plain_pusher(width):
    """Particles outside a surrogate's training box are pushed inside the
    surrogate kernel by its fallback warp (past a CTA's 256-entry queue, by
    the list-mode pusher) with the plain FP32 pusher's arithmetic, so they
    equal bl_push_stage's result bit for bit; the others equal the
    domain-free network's output. Box half-widths of 3.5, 2 and 0.7 sigma
    put ~0.3 %, ~25 % and ~98 % of a 10^6-particle bunch outside: the queue
    alone, the queue plus the list, and nearly all through the list."""
    from paper_2402_17248_gb300 import bl
    n = 1_000_000
    z, g = _bunch(n, seed=31)
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    Ws, bs = mlp_init(WIDTHS, 7)
    sur = bl.Surrogate(Ws, bs, mu, sd, mu, sd)
    sur.set_domain(mu - width * sd, mu + width * sd)
    # the FP32 box the kernel compares with (the library widens the FP64
    # bounds outward to FP32)
    import ctypes
    lo64, hi64, has = np.zeros(6), np.zeros(6), ctypes.c_int32(0)
    assert bl.lib().bl_surrogate_get_domain(sur.handle, lo64.ctypes.data, hi64.ctypes.data,
                                            ctypes.byref(has)) == bl.BL_OK and has.value
    lo, hi = lo64.astype(np.float32), hi64.astype(np.float32)
    z32 = np.stack([np.asarray(c, dtype=np.float32) for c in z])
    inside = np.all((z32 >= lo[:, None]) & (z32 <= hi[:, None]), axis=0)
    st = lattice.plasma(400)
    st["surrogate"] = sur
    b1 = to_bunch(z, g)
    bl.bl_track(b1, bl.Lattice([st]), moments=False)
    got = from_bunch(b1)
    b2 = to_bunch(z, g)
    bl.bl_push_stage(b2, lattice.plasma(400))
    push = from_bunch(b2)
    sur.set_domain(None, None)
    b3 = to_bunch(z, g)
    bl.bl_track(b3, bl.Lattice([st]), moments=False)
    net = from_bunch(b3)
    print("box +-%.1f sigma: %.4f of the particles outside" % (width, 1.0 - inside.mean()))
    assert 0 < (~inside).sum() < n
    for a, p_, q in zip(got, push, net):
        assert np.array_equal(a[~inside], p_[~inside])
        assert np.array_equal(a[inside], q[inside])
