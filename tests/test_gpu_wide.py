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
