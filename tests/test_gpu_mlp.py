"""GPU parity of the MLP surrogate: tcgen05 inference and the training /
gradient kernels against the FP64 oracle with the same BF16-valued weights."""
import math

import numpy as np
import pytest

from gpu_util import KEYS, as_f32, from_bunch, to_bunch
from oracle import mlp, moments
from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init

pytestmark = pytest.mark.gpu
WIDTHS = [6, 128, 128, 128, 128, 6]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_17248_gb300 import bl
    bl.lib()


def _bunch(n, seed=0):
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=seed))
    return as_f32([z[k] for k in KEYS]), g


def _net(seed, z, out_shift=0.0):
    Ws, bs = mlp_init(WIDTHS, seed)
    Z = np.stack(z, axis=1)
    mu, sd = Z.mean(axis=0), Z.std(axis=0)
    return Ws, bs, mu, sd, mu + out_shift * sd, sd * 1.5


def _oracle_surrogate(Ws, bs, mu, sd, mo, so):
    Wr = [mlp.bf16_round(np.asarray(W, dtype=np.float32).astype(np.float64)) for W in Ws]
    br = [np.asarray(b, dtype=np.float32).astype(np.float64) for b in bs]
    return mlp.Surrogate(Wr, br, mu, sd, mo, so)


@pytest.mark.parametrize("n", [1, 127, 128, 129, 257, 10000, 300001])
def test_inference_matches_oracle(n):
    from paper_2402_17248_gb300 import bl
    z, g = _bunch(max(n, 2), seed=n)
    z = [c[:n] for c in z]
    Ws, bs, mu, sd, mo, so = _net(3, _bunch(5000, 1)[0], 0.3)
    sur = bl.Surrogate(Ws, bs, mu, sd, mo, so)
    b = to_bunch(z, g)
    bl.bl_surrogate_apply(sur, b)
    got = from_bunch(b)
    bl.bl_poll_device_errors()
    osur = _oracle_surrogate(Ws, bs, mu, sd, mo, so)
    want_bf = osur.apply(z, bf16=True)
    want_64 = osur.apply(z, bf16=False)
    e_bf = max(float(np.max(np.abs(a - w))) / s for a, w, s in zip(got, want_bf, so))
    e_64 = max(float(np.max(np.abs(a - w))) / s for a, w, s in zip(got, want_64, so))
    print("n=%d max |gpu - oracle| / sd_out: bf16-emulating %.3e, fp64 %.3e" % (n, e_bf, e_64))
    assert e_bf < 2e-3
    if n >= 10000:
        dg = moments.moments28(got)
        dw = moments.moments28(want_64)
        Sg, Sw = moments.sigma_matrix(dg), moments.sigma_matrix(dw)
        rel = np.max(np.abs(np.diag(Sg) / np.diag(Sw) - 1))
        print("  output second moments, relative to the FP64 network: %.3e" % rel)
        assert rel < 2e-3


def test_inference_repeatable_and_inplace_tail():
    from paper_2402_17248_gb300 import bl
    import torch
    z, g = _bunch(1000, seed=4)
    Ws, bs, mu, sd, mo, so = _net(5, z)
    sur = bl.Surrogate(Ws, bs, mu, sd, mo, so)
    # a 997-particle view into a longer buffer: the 3 trailing values stay intact
    coords = [torch.tensor(c, dtype=torch.float32, device="cuda") for c in z]
    views = [c[:997] for c in coords]
    b = bl.Bunch(views, g)
    bl.bl_surrogate_apply(sur, b)
    torch.cuda.synchronize()
    for c, orig in zip(coords, z):
        assert np.array_equal(c[997:].cpu().numpy().astype(np.float64), orig[997:])
    first = [c[:997].cpu().numpy().copy() for c in coords]
    coords2 = [torch.tensor(c, dtype=torch.float32, device="cuda") for c in z]
    b2 = bl.Bunch([c[:997] for c in coords2], g)
    bl.bl_surrogate_apply(sur, b2)
    torch.cuda.synchronize()
    for a, c in zip(first, coords2):
        assert np.array_equal(a, c[:997].cpu().numpy())


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    zin, g = _bunch(n, seed)
    A = rng.normal(size=(6, 6)) * 0.3 + np.eye(6)
    Zi = np.stack(zin)
    sd = Zi.std(axis=1, keepdims=True)
    Zo = (A @ (Zi / sd)) * sd + 0.1 * np.sin(Zi / sd) * sd
    return Zi.astype(np.float32), Zo.astype(np.float32)


def _oracle_grad(Ws, bs, Zi, Zo, mu_i, sd_i, mu_o, sd_o):
    osur = _oracle_surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    X = (Zi.T.astype(np.float64) - mu_i) / sd_i
    Y = (Zo.T.astype(np.float64) - mu_o) / sd_o
    P, cache = mlp.forward(osur.Ws, osur.bs, X, bf16=True, keep=True)
    L = mlp.mse(P, Y)
    _, dW, db = mlp.backward(osur.Ws, cache, mlp.mse_grad(P, Y))
    flat = []
    for l in range(5):
        flat += [dW[l].ravel(), db[l].ravel()]
    return L, np.concatenate(flat)


@pytest.fixture(params=["tensor_core", "simt"])
def train_kernel(request):
    from paper_2402_17248_gb300 import bl
    prev = bl.bl_debug_train_kernel(request.param == "simt")
    yield request.param
    bl.bl_debug_train_kernel(prev)


# batch sizes: one sample, ragged tiles of the 128-sample tensor-core kernel,
# several tiles, and more tiles than SMs (tiles looped per CTA)
@pytest.mark.parametrize("batch", [1, 127, 129, 1200, 40000])
def test_gradient_matches_oracle(train_kernel, batch):
    """Minibatch MSE loss and gradient (all weights and biases, flat layout)
    of both gradient kernels against the FP64 oracle's reverse mode with the
    same BF16-valued weights; inputs gathered through an index vector."""
    import torch
    from paper_2402_17248_gb300 import bl
    Zi, Zo = _pairs(max(1200, batch), 11)
    mu_i, sd_i = Zi.mean(axis=1), Zi.std(axis=1)
    mu_o, sd_o = Zo.mean(axis=1), Zo.std(axis=1)
    Ws, bs = mlp_init(WIDTHS, 2)
    sur = bl.Surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    din = torch.tensor(Zi, device="cuda")
    dout = torch.tensor(Zo, device="cuda")
    sel = np.random.default_rng(batch).permutation(Zi.shape[1])[:batch]
    idx = torch.tensor(sel, device="cuda", dtype=torch.int64)
    grad = torch.zeros(bl.BL_MLP_NPARAM, device="cuda")
    loss = torch.zeros(1, device="cuda")
    bl.bl_surrogate_grad(sur, din, dout, grad, idx=idx, loss_out=loss)
    torch.cuda.synchronize()
    L, flat = _oracle_grad(Ws, bs, Zi[:, sel], Zo[:, sel], mu_i, sd_i, mu_o, sd_o)
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - flat) / np.linalg.norm(flat)
    print("%s batch %d: loss gpu %.6e oracle %.6e; gradient normwise rel err %.3e"
          % (train_kernel, batch, loss.item(), L, rel))
    assert abs(loss.item() / L - 1) < 1e-3
    # tanh.approx (relative error 2^-11) in the forward's GELU is the
    # largest term; measured 1e-5 .. 2e-4
    assert rel < 1e-3
    # per layer: every block of the flat vector is filled, not only the large ones
    offs = [0, 768, 896, 17280, 17408, 33792, 33920, 50304, 50432, 51200, 51206]
    for a, b in zip(offs[:-1], offs[1:]):
        ra = np.linalg.norm(g[a:b] - flat[a:b]) / np.linalg.norm(flat[a:b])
        assert ra < 5e-3, (a, b, ra)


def test_gradient_kernels_agree():
    """The tensor-core and SIMT gradient kernels evaluate the same minibatch
    gradient independently; they agree to the tolerance of their BF16
    operands."""
    import torch
    from paper_2402_17248_gb300 import bl
    Zi, Zo = _pairs(20000, 13)
    mu_i, sd_i = Zi.mean(axis=1), Zi.std(axis=1)
    mu_o, sd_o = Zo.mean(axis=1), Zo.std(axis=1)
    Ws, bs = mlp_init(WIDTHS, 4)
    sur = bl.Surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    din = torch.tensor(Zi, device="cuda")
    dout = torch.tensor(Zo, device="cuda")
    out = []
    for simt in (False, True):
        prev = bl.bl_debug_train_kernel(simt)
        try:
            g = torch.zeros(bl.BL_MLP_NPARAM, device="cuda")
            bl.bl_surrogate_grad(sur, din, dout, g)
            torch.cuda.synchronize()
        finally:
            bl.bl_debug_train_kernel(prev)
        out.append(g.cpu().numpy().astype(np.float64))
    rel = np.linalg.norm(out[0] - out[1]) / np.linalg.norm(out[1])
    print("tensor-core vs SIMT gradient: normwise rel diff %.3e" % rel)
    assert rel < 1e-2


def test_training_reduces_loss_and_adam_step():
    import torch
    from paper_2402_17248_gb300 import bl
    Zi, Zo = _pairs(24000, 12)
    mu_i, sd_i = Zi.mean(axis=1), Zi.std(axis=1)
    mu_o, sd_o = Zo.mean(axis=1), Zo.std(axis=1)
    Ws, bs = mlp_init(WIDTHS, 3)
    sur = bl.Surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    din = torch.tensor(Zi, device="cuda")
    dout = torch.tensor(Zo, device="cuda")
    # first Adam step moves every parameter by lr * sign(g) (bias-corrected)
    grad = torch.zeros(bl.BL_MLP_NPARAM, device="cuda")
    idx = torch.arange(0, 1200, device="cuda", dtype=torch.int64)
    bl.bl_surrogate_grad(sur, din, dout, grad, idx=idx)
    bl.bl_surrogate_train_step(sur, din, dout, idx=idx, lr=1e-3)
    torch.cuda.synchronize()
    W1, b1 = sur.params()
    g = grad.cpu().numpy()
    moved = np.concatenate([(W1[l] - np.asarray(Ws[l], np.float32)).ravel().astype(np.float64)
                            for l in range(5)])
    gw = np.concatenate([g[o:o + WIDTHS[l] * WIDTHS[l + 1]] for l, o in
                         enumerate([0, 896, 17408, 33920, 50432])])
    big = np.abs(gw) > 1e-5
    assert np.allclose(moved[big], -1e-3 * np.sign(gw[big]), rtol=1e-3, atol=2e-7)
    # a few hundred steps lower the held-out loss
    loss = torch.zeros(1, device="cuda", dtype=torch.float64)
    test_in, test_out = din[:, 20000:].contiguous(), dout[:, 20000:].contiguous()
    bl.bl_surrogate_loss(sur, test_in, test_out, loss)
    torch.cuda.synchronize()
    l0 = loss.item()
    gen = torch.Generator(device="cuda").manual_seed(0)
    for step in range(300):
        idx = torch.randint(0, 20000, (1200,), device="cuda", generator=gen)
        bl.bl_surrogate_train_step(sur, din, dout, idx=idx, lr=1e-3)
    bl.bl_surrogate_loss(sur, test_in, test_out, loss)
    torch.cuda.synchronize()
    print("held-out loss %.4e -> %.4e" % (l0, loss.item()))
    assert loss.item() < 0.2 * l0


def test_surrogate_file_round_trip_and_resume(tmp_path):
    """save -> load gives the same parameters, normalisation, domain and
    inference bit for bit; training resumed from the file follows the same
    trajectory (parameters and Adam state) as training that never stopped."""
    import torch
    from paper_2402_17248_gb300 import bl
    Zi, Zo = _pairs(8000, 21)
    mu_i, sd_i = Zi.mean(axis=1), Zi.std(axis=1)
    mu_o, sd_o = Zo.mean(axis=1), Zo.std(axis=1)
    Ws, bs = mlp_init(WIDTHS, 9)
    din = torch.tensor(Zi, device="cuda").contiguous()
    dout = torch.tensor(Zo, device="cuda").contiguous()
    gen = torch.Generator(device="cuda").manual_seed(3)
    idx = torch.randint(0, 8000, (60, 1024), device="cuda", generator=gen)
    a = bl.Surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    for j in range(30):
        bl.bl_surrogate_train_step(a, din, dout, idx=idx[j], lr=1e-3)
    lo, hi = Zi.min(axis=1).astype(np.float64), Zi.max(axis=1).astype(np.float64)
    a.set_domain(lo, hi)
    torch.cuda.synchronize()
    path = tmp_path / "stage.blsurr"
    a.save(path)
    b = bl.Surrogate.load(path)
    for x, y in zip(a.params(), b.params()):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))
    assert np.array_equal(b.mu_in, a.mu_in) and np.array_equal(b.sd_out, a.sd_out)
    assert b.domain is not None and np.all(b.domain[0] <= lo) and np.all(b.domain[1] >= hi)
    z, g = _bunch(3000, seed=8)
    o1, o2 = to_bunch(z, g), to_bunch(z, g)
    bl.bl_surrogate_apply(a, o1)
    bl.bl_surrogate_apply(b, o2)
    assert all(np.array_equal(u, v) for u, v in zip(from_bunch(o1), from_bunch(o2)))
    for j in range(30, 60):  # resume: same steps on both
        bl.bl_surrogate_train_step(a, din, dout, idx=idx[j], lr=1e-3)
        bl.bl_surrogate_train_step(b, din, dout, idx=idx[j], lr=1e-3)
    torch.cuda.synchronize()
    for x, y in zip(a.params(), b.params()):
        assert all(np.array_equal(u, v) for u, v in zip(x, y))


def _read_surrogate_file(path):
    """FP32 masters, Adam m and v and the step count of a surrogate file
    (layout of bl_surrogate_save: magic, version, widths, FP64 normalisation,
    domain flag and box, step, then the three flat FP32 vectors)."""
    raw = open(path, "rb").read()
    off = 8 + 4 + 6 * 4 + 4 * 6 * 8 + 4 + 2 * 6 * 4
    step = int(np.frombuffer(raw, dtype=np.int32, count=1, offset=off)[0])
    off += 4
    n = 51206
    P = np.frombuffer(raw, dtype=np.float32, count=n, offset=off)
    M = np.frombuffer(raw, dtype=np.float32, count=n, offset=off + 4 * n)
    V = np.frombuffer(raw, dtype=np.float32, count=n, offset=off + 8 * n)
    return step, P.astype(np.float64), M.astype(np.float64), V.astype(np.float64)


def test_adam_over_many_steps_matches_oracle(tmp_path):
    """50 Adam steps of bl_surrogate_train_step on fixed index batches: the
    FP32 masters and the first and second moments m, v read back from the
    surrogate file agree with the oracle's FP64 Adam (bias-corrected,
    Kingma and Ba Alg. 1) fed the same minibatch gradients, so the m and v
    recurrences and the bias corrections for t > 1 are checked, not only
    the first step."""
    import torch
    from paper_2402_17248_gb300 import bl
    Zi, Zo = _pairs(20000, 17)
    mu_i, sd_i = Zi.mean(axis=1), Zi.std(axis=1)
    mu_o, sd_o = Zo.mean(axis=1), Zo.std(axis=1)
    Ws, bs = mlp_init(WIDTHS, 5)
    sur = bl.Surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    din = torch.tensor(Zi, device="cuda")
    dout = torch.tensor(Zo, device="cuda")
    rng = np.random.default_rng(6)
    steps, batch, lr, b1, b2, eps = 50, 1024, 2e-3, 0.9, 0.999, 1e-8
    path = str(tmp_path / "s.blsur")
    sur.save(path)
    t0, p0, m0, v0 = _read_surrogate_file(path)
    assert t0 == 0 and not m0.any() and not v0.any()
    grads = []
    g = torch.zeros(bl.BL_MLP_NPARAM, device="cuda")
    for t in range(steps):
        idx = torch.tensor(rng.permutation(20000)[:batch], device="cuda", dtype=torch.int64)
        bl.bl_surrogate_grad(sur, din, dout, g, idx=idx)
        grads.append(g.cpu().numpy().astype(np.float64))
        bl.bl_surrogate_train_step(sur, din, dout, idx=idx, lr=lr, beta1=b1, beta2=b2, eps=eps)
    torch.cuda.synchronize()
    sur.save(path)
    t1, p1, m1, v1 = _read_surrogate_file(path)
    assert t1 == steps
    opt = mlp.Adam([p0], lr=lr, b1=b1, b2=b2, eps=eps)
    p = [p0]
    for gr in grads:
        p = opt.step(p, [gr])
    rm = np.linalg.norm(m1 - opt.m[0]) / np.linalg.norm(opt.m[0])
    rv = np.linalg.norm(v1 - opt.v[0]) / np.linalg.norm(opt.v[0])
    disp = p[0] - p0
    rp = np.linalg.norm((p1 - p0) - disp) / np.linalg.norm(disp)
    print("after %d Adam steps: m %.2e, v %.2e, displacement of the masters %.2e (normwise rel)"
          % (steps, rm, rv, rp))
    assert rm < 1e-6 and rv < 1e-6
    assert rp < 1e-5


def _split_grad(sur, din, dout, idx, nA):
    """Gradient and loss of the whole batch and of its first nA samples and
    the rest, each from its own bl_surrogate_grad call."""
    import torch
    from paper_2402_17248_gb300 import bl
    out = []
    parts = [(None, None)]
    parts.append((0, nA))
    parts.append((nA, None))
    for a, b in parts:
        g = torch.zeros(bl.BL_MLP_NPARAM, device="cuda")
        loss = torch.zeros(1, device="cuda")
        if idx is not None:
            sel = idx if a is None else idx[a:b].contiguous()
            bl.bl_surrogate_grad(sur, din, dout, g, idx=sel, loss_out=loss)
            n = sel.numel()
        else:
            i_ = din if a is None else din[:, a:b].contiguous()
            o_ = dout if a is None else dout[:, a:b].contiguous()
            bl.bl_surrogate_grad(sur, i_, o_, g, loss_out=loss)
            n = i_.shape[1]
        torch.cuda.synchronize()
        out.append((g.double().cpu().numpy(), float(loss.item()), n))
    return out


# a batch just past the 2^17-sample launch chunk (two chunks, the second
# ragged), gathered through an index vector and read as contiguous columns;
# and the API's largest batch, 2^24 samples (128 chunks)
@pytest.mark.parametrize("batch,with_idx", [((1 << 17) + 5003, True),
                                            ((1 << 17) + 5003, False),
                                            (1 << 24, False)])
def test_gradient_large_batch_in_chunks(train_kernel, batch, with_idx):
    """A minibatch larger than one gradient launch (2^17 samples) is taken in
    chunks whose partial rows are added to one running row, each chunk
    scaled as a mean over the whole batch, so the workspace stays bounded.
    Its gradient and loss are the sample-weighted mean of those of two
    sub-batches computed by separate calls, to FP32 summation rounding."""
    import torch
    from paper_2402_17248_gb300 import bl
    if train_kernel == "simt" and batch > (1 << 20):
        pytest.skip("the SIMT kernel is a cross-check at moderate batch sizes")
    g = torch.Generator(device="cuda").manual_seed(batch % 1000)
    din = torch.randn(6, batch, device="cuda", generator=g)
    dout = din + 0.1 * torch.randn(6, batch, device="cuda", generator=g)
    Ws, bs = mlp_init(WIDTHS, 5)
    sur = bl.Surrogate(Ws, bs, np.zeros(6), np.ones(6), np.zeros(6), np.ones(6))
    idx = None
    if with_idx:
        idx = torch.randperm(batch, device="cuda", generator=g)
    nA = (1 << 16) if batch < (1 << 20) else batch // 2
    (ga, La, n), (g1, L1, n1), (g2, L2, n2) = _split_grad(sur, din, dout, idx, nA)
    assert n == batch and n1 + n2 == batch
    want = (n1 * g1 + n2 * g2) / batch
    rel = np.linalg.norm(ga - want) / np.linalg.norm(want)
    print("%s batch %d: whole-batch vs split gradient rel diff %.2e, loss %.8e vs %.8e"
          % (train_kernel, batch, rel, La, (n1 * L1 + n2 * L2) / batch))
    assert rel < 1e-5
    assert abs(La / ((n1 * L1 + n2 * L2) / batch) - 1) < 1e-6
