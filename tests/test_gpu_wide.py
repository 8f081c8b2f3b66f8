"""GPU parity of the paper-shaped wide PReLU surrogates (five hidden layers of
900 units, three of 700) against the FP64 oracle with the same BF16-valued
weights and BF16 rounding points, including chunked application and ragged
particle counts."""
import numpy as np
import pytest

from gpu_util import KEYS, as_f32, from_bunch, to_bunch
from oracle import mlp, moments
from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_17248_gb300 import bl
    bl.lib()


def _bunch(n, seed=0):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return as_f32([z[k] for k in KEYS]), g


def _net(widths, seed, z):
    Ws, bs = mlp_init(widths, seed)
    slopes = [0.25 - 0.05 * l for l in range(len(widths) - 2)]
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    return Ws, bs, slopes, mu, sd, mu + 0.2 * sd, 1.3 * sd


@pytest.mark.parametrize("widths,n,chunk", [
    ([6, 900, 900, 900, 900, 900, 6], 20001, 8192),
    ([6, 700, 700, 700, 6], 20001, 0),
    ([6, 700, 700, 700, 6], 127, 0),
    ([6, 96, 130, 6], 1, 0),
])
def test_wide_matches_oracle(widths, n, chunk):
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(max(n, 2), seed=len(widths) + n)
    z = [c[:n] for c in z]
    Ws, bs, slopes, mu, sd, mo, so = _net(widths, 17, _bunch(4000, 3)[0])
    net = bl.WideSurrogate(Ws, bs, slopes, mu, sd, mo, so)
    b = to_bunch(z, g)
    bl.bl_wide_mlp_apply(net, b, chunk=chunk)
    got = from_bunch(b)
    bl.bl_poll_device_errors()
    Wr = [mlp.bf16_round(np.asarray(W, np.float32).astype(np.float64)) for W in Ws]
    br = [np.asarray(v, np.float32).astype(np.float64) for v in bs]
    osur = mlp.Surrogate(Wr, br, mu, sd, mo, so, slopes=np.asarray(slopes, np.float32))
    want = osur.apply(z, bf16=True)
    err = max(float(np.max(np.abs(a - w))) / s for a, w, s in zip(got, want, so))
    print("widths %s n=%d: max |gpu - oracle| / sd_out %.3e" % (widths[1:-1], n, err))
    assert err < 2e-3
    if n > 10000:
        Sg = moments.sigma_matrix(moments.moments28(got))
        Sw = moments.sigma_matrix(moments.moments28(osur.apply(z, bf16=False)))
        rel = np.max(np.abs(np.diag(Sg) / np.diag(Sw) - 1))
        print("  output second moments vs the FP64 network: %.3e" % rel)
        assert rel < 2e-3


def test_wide_rejects_bad_descriptors():
    from paper_2402_17248_gb300 import bl
    Ws, bs = mlp_init([6, 64, 6], 1)
    one = np.ones(6)
    with pytest.raises(bl.BlError):
        bl.WideSurrogate(Ws, bs, [0.25], one, -one, one, one)  # negative sd
    Ws2, bs2 = mlp_init([5, 64, 6], 1)
    with pytest.raises(bl.BlError):
        bl.WideSurrogate(Ws2, bs2, [0.25], np.ones(6), one, one, one)  # input width 5


def _pairs(n, seed):
    """(input, target) pairs of a smooth 6D map on design-bunch inputs."""
    rng = np.random.default_rng(seed)
    zin, _ = _bunch(n, seed)
    Zi = np.stack(zin).astype(np.float64)
    sd = Zi.std(axis=1, keepdims=True)
    A = rng.normal(size=(6, 6)) * 0.3 + np.eye(6)
    Zo = (A @ (Zi / sd)) * sd + 0.1 * np.sin(Zi / sd) * sd
    return Zi.astype(np.float32), Zo.astype(np.float32)


def _flat_oracle_grad(Ws, bs, slopes, Zi, Zo, mu_i, sd_i, mu_o, sd_o):
    """Loss and flat gradient [W0, b0, ..., slopes] of the oracle's MSE on
    normalised data with the BF16-valued weights and BF16 rounding points."""
    Wr = [mlp.bf16_round(np.asarray(W, np.float32).astype(np.float64)) for W in Ws]
    br = [np.asarray(b, np.float32).astype(np.float64) for b in bs]
    sl = [float(np.float32(a)) for a in slopes]
    X = (Zi.T.astype(np.float64) - mu_i) / sd_i
    Y = (Zo.T.astype(np.float64) - mu_o) / sd_o
    P, cache = mlp.forward(Wr, br, X, bf16=True, keep=True, slopes=sl)
    L = mlp.mse(P, Y)
    _, dW, db, dsl = mlp.backward(Wr, cache, mlp.mse_grad(P, Y), slopes=sl)
    flat = []
    for l in range(len(Ws)):
        flat += [dW[l].ravel(), db[l].ravel()]
    flat.append(np.asarray(dsl))
    return L, np.concatenate(flat)


@pytest.mark.parametrize("widths,batch", [([6, 700, 700, 700, 6], 1000),
                                          ([6, 900, 900, 900, 900, 900, 6], 777),
                                          ([6, 96, 130, 6], 1)])
def test_wide_gradient_matches_oracle(widths, batch):
    """Minibatch MSE loss and gradient (every weight, bias and PReLU slope)
    of the wide network's training path against the oracle's reverse mode
    with the same BF16-valued weights; inputs gathered through an index
    vector."""
    import torch
    from paper_2402_17248_gb300 import bl
    Zi, Zo = _pairs(max(batch, 2000), 31)
    mu_i, sd_i = Zi.mean(axis=1), Zi.std(axis=1)
    mu_o, sd_o = Zo.mean(axis=1), Zo.std(axis=1)
    Ws, bs = mlp_init(widths, 9)
    slopes = [0.25 - 0.05 * l for l in range(len(widths) - 2)]
    net = bl.WideSurrogate(Ws, bs, slopes, mu_i, sd_i, mu_o, sd_o)
    sel = np.random.default_rng(batch).permutation(Zi.shape[1])[:batch]
    din, dout = torch.tensor(Zi, device="cuda"), torch.tensor(Zo, device="cuda")
    idx = torch.tensor(sel, device="cuda", dtype=torch.int64)
    grad = torch.zeros(net.num_params, device="cuda")
    loss = torch.zeros(1, device="cuda")
    bl.bl_wide_mlp_grad(net, din, dout, grad, idx=idx, loss_out=loss)
    torch.cuda.synchronize()
    bl.bl_poll_device_errors()
    L, flat = _flat_oracle_grad(Ws, bs, slopes, Zi[:, sel], Zo[:, sel], mu_i, sd_i, mu_o, sd_o)
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - flat) / np.linalg.norm(flat)
    nsl = len(widths) - 2
    rel_s = np.max(np.abs(g[-nsl:] - flat[-nsl:])) / np.max(np.abs(flat[-nsl:]))
    print("widths %s batch %d: loss gpu %.6e oracle %.6e; gradient normwise rel err %.3e, "
          "slopes %.3e" % (widths[1:-1], batch, loss.item(), L, rel, rel_s))
    assert abs(loss.item() / L - 1) < 1e-3
    assert rel < 5e-3
    assert rel_s < 5e-3


def test_wide_training_on_pusher_pairs_and_as_a_lattice_stage():
    """A 3 x 700 PReLU network trained on the GPU (Adam on every weight, bias
    and slope) on one plasma stage's pusher pairs lowers its held-out loss
    and moves its slopes; as the stage of a lattice it tracks exactly like
    bl_wide_mlp_apply followed by the section, and matches the oracle's
    PReLU surrogate with its trained parameters."""
    import torch
    from paper_2402_17248_gb300 import bl, workflow
    from oracle import beamline
    from synth import lattice
    from synth.bunch import training_population
    g0 = BunchRecipe().gamma_ref
    zt, _ = training_population(4, 65536, g0, 0.2 / workflow.plasma_wavenumber(), seed=1001)
    els = lattice.staged_beamline(1, 400)
    xin, xout, gin = workflow.stage_pairs(workflow.device_bunch(zt, g0), els)[0]
    net, info = workflow.fit_wide_surrogate(xin, xout, [6, 700, 700, 700, 6], steps=1500,
                                            batch=4096, lr=1e-3, seed=3, log_every=1)
    h = info["history"]
    print("3x700 on pusher pairs: held-out loss %.3e -> %.3e, slopes %s (%.1fs)"
          % (h[0][1], info["test_loss"], np.round(info["slopes"], 4), info["seconds"]))
    # 1500 steps of 4096 take the held-out loss of a fresh 3 x 700 network
    # from ~1 to ~0.27 on these pairs; the paper trains for far longer
    assert info["test_loss"] < 0.5 * h[0][1]
    assert info["test_loss"] < h[len(h) // 2][1]
    assert np.max(np.abs(np.asarray(info["slopes"]) - 0.25)) > 1e-3
    # the trained network as the stage of a lattice
    z, g = _bunch(30001, seed=5)
    st = dict(els[0], surrogate=net)
    b1 = to_bunch(z, g)
    m1, nf = bl.bl_track(b1, bl.Lattice([st] + els[1:]))
    b2 = to_bunch(z, g)
    bl.bl_wide_mlp_apply(net, b2)
    b2.struct.gamma_ref = bl.bl_reference_exit(els[0], g)
    bl.bl_track(b2, bl.Lattice(els[1:]), moments=False)
    for a, w in zip(from_bunch(b1), from_bunch(b2)):
        assert np.array_equal(a, w)
    assert b1.gamma_ref == b2.gamma_ref
    Ws, bs, sl = net.params()
    Wr = [mlp.bf16_round(W.astype(np.float64)) for W in Ws]
    osur = mlp.Surrogate(Wr, [b.astype(np.float64) for b in bs], net.mu_in, net.sd_in,
                         net.mu_out, net.sd_out, slopes=sl)
    lat_o = [dict(els[0], surrogate=osur)] + els[1:]
    zo, go, _ = beamline.track(z, g, lat_o, bf16=True)
    z64, _, _ = beamline.track(z, g, lat_o, bf16=False)
    got = from_bunch(b1)
    # Per particle the device and the BF16-emulating oracle differ where a
    # hidden activation lies within FP32 accumulation error of a BF16
    # rounding midpoint and the two round it to neighbouring values. A
    # trained network amplifies such a flip by its Jacobian, which is large
    # in t (the exit coordinates oscillate across the bunch in t), so single
    # particles can move by percents of the rms. The differences that flips
    # cause are bounded by what rounding every activation does: per
    # coordinate, the rms of (device - BF16 oracle) stays below the rms of
    # (BF16 oracle - FP64 network); the beam's moments agree to 2e-3.
    for c, (a, w, v) in enumerate(zip(got, zo, z64)):
        sd = np.std(w)
        d = np.abs(a - w) / sd
        flip = np.sqrt(np.mean((a - w) ** 2)) / sd
        rnd = np.sqrt(np.mean((w - v) ** 2)) / sd
        print("  %s: |gpu - oracle| / rms median %.2e, 99%% %.2e, max %.2e; rms %.2e "
              "(BF16 rounding itself: %.2e)" % (KEYS[c], np.median(d), np.quantile(d, 0.99),
                                                d.max(), flip, rnd))
        assert flip <= rnd, (KEYS[c], flip, rnd)
    Sg = moments.sigma_matrix(moments.moments28(got))
    So = moments.sigma_matrix(moments.moments28(zo))
    sdv = np.sqrt(np.diag(So))
    rel = float(np.max(np.abs(Sg - So) / np.outer(sdv, sdv)))
    print("  exit second moments vs oracle: %.3e of sigma_a sigma_b" % rel)
    assert rel < 2e-3
