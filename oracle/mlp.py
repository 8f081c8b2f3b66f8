"""Fully connected MLP surrogate, its gradient, MSE loss and Adam (FP64).

Network (Sec. 3, Eq. for F): F = L_l o sigma o ... o sigma o L_0 with
L_i(v) = A_i v + b_i, the same activation sigma after every hidden layer and
equal hidden widths H; n = m = 6 phase-space coordinates. The hidden
activation here is GELU in the tanh form of Hendrycks and Gimpel,
gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (reading: the paper
uses PReLU; the tracked configuration names GELU).

Inputs and outputs are normalised per coordinate to zero mean and unit
standard deviation (Sec. 3, data preparation): x~ = (x - mu_in)/sigma_in,
y = y~ sigma_out + mu_out. Loss: MSE(x, y) = (1/(N n)) sum (x_ij - y_ij)^2
(Sec. 3). Optimiser: Adam (Kingma and Ba, Algorithm 1) with bias correction.

Weights are stored as W[l] with shape (out, in), as in Eq. L_i(v) = A_i v + b_i.

The paper's own networks (Sec. 4.2: five hidden layers of 900 units for the
first stages, three of 700 for the later ones) use PReLU,
prelu(x) = max(x, 0) + a min(x, 0) with one learned slope a per layer (the
single-parameter form; reading). `forward(..., slopes=[a_0, ...])` selects it.

Optional BF16 emulation rounds at the points where a BF16 datapath stores
values: the normalised network input, stored as an FP32 value x32, is
carried as a pair of bfloat16 numbers, hi = bf16(x32) and lo = bf16(x32 - hi)
(16 significant bits; one BF16
value alone would quantise the input to 2^-9, which the exit coordinates'
strong dependence on the arrival time t turns into errors of percents of
their spread), and every hidden activation is rounded to one bfloat16 value
(round to nearest even); all sums stay FP64.

Parity: forward and backward (GELU and PReLU, the PReLU slopes' gradient
included) pinned against an independent float64 autograd implementation
(torch CPU, test only) and central finite differences; GELU special values;
Adam's first step closed form and an independent Adam.
"""
import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def bf16_round(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    bits = x.view(np.uint64).copy()
    # bfloat16 keeps 7 explicit mantissa bits; float64 has 52 -> drop 45
    drop = np.uint64(45)
    lsb = (bits >> drop) & np.uint64(1)
    rnd = (np.uint64(1) << np.uint64(44)) - np.uint64(1) + lsb
    finite = np.isfinite(x)
    out_bits = ((bits + rnd) >> drop) << drop
    return np.where(finite, out_bits.view(np.float64), x)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    u = GELU_C * (x + GELU_A * x ** 3)
    t = np.tanh(u)
    du = GELU_C * (1.0 + 3.0 * GELU_A * x * x)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * du


def prelu(x, a):
    return np.where(x > 0.0, x, a * x)


def bf16_pair(x):
    """x carried as hi + lo: x is first stored as an FP32 value x32 (as the
    normalisation hands it to the network), then hi = bf16(x32) and
    lo = bf16(x32 - hi); returned as float64."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    hi = bf16_round(x32)
    return hi + bf16_round(x32 - hi)


def forward(Ws, bs, X, bf16=False, keep=False, slopes=None):
    """X: (N, n_in) normalised inputs. Returns outputs (N, n_out) [, cache].
    slopes: None for GELU, else one PReLU slope per hidden layer."""
    h = np.asarray(X, dtype=np.float64)
    if bf16:
        h = bf16_pair(h)
    pre, acts = [], [h]
    nl = len(Ws)
    for l in range(nl):
        a = h @ Ws[l].T + bs[l]
        if l < nl - 1:
            pre.append(a)
            h = gelu(a) if slopes is None else prelu(a, slopes[l])
            if bf16:
                h = bf16_round(h)
            acts.append(h)
        else:
            h = a
    if keep:
        return h, (pre, acts)
    return h


def backward(Ws, cache, dY, slopes=None):
    """Reverse mode through the network for upstream gradient dY (N, n_out).

    Returns (dX, dWs, dbs): gradients with respect to the network input, the
    weights and the biases (summed over the batch). Rounding to bfloat16 in an
    emulated forward is treated as the identity. With slopes (a PReLU
    network), returns (dX, dWs, dbs, dslopes): d prelu / d pre = 1 where
    pre > 0 and a otherwise, and d prelu / d a = min(pre, 0), so
    dL/da_l = sum over the batch and the layer's units of min(pre, 0) times
    the gradient with respect to that layer's output.
    """
    pre, acts = cache
    nl = len(Ws)
    dWs = [None] * nl
    dbs = [None] * nl
    dsl = [0.0] * (nl - 1)
    d = np.asarray(dY, dtype=np.float64)
    for l in range(nl - 1, -1, -1):
        dWs[l] = d.T @ acts[l]
        dbs[l] = d.sum(axis=0)
        d = d @ Ws[l]
        if l > 0:
            z = pre[l - 1]
            if slopes is None:
                d = d * gelu_grad(z)
            else:
                dsl[l - 1] = float(np.sum(d * np.minimum(z, 0.0)))
                d = d * np.where(z > 0.0, 1.0, slopes[l - 1])
    if slopes is None:
        return d, dWs, dbs
    return d, dWs, dbs, dsl


def mse(P, Y):
    P = np.asarray(P, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.mean((P - Y) ** 2))


def mse_grad(P, Y):
    """d MSE / d P for MSE = (1/(N n)) sum (P - Y)^2."""
    P = np.asarray(P, dtype=np.float64)
    return 2.0 * (P - np.asarray(Y, dtype=np.float64)) / P.size


class Adam:
    """Adam with bias correction; epsilon is added outside the square root."""

    def __init__(self, params, lr=1.0e-4, b1=0.9, b2=0.999, eps=1.0e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for i, (p, g) in enumerate(zip(params, grads)):
            self.m[i] = self.b1 * self.m[i] + (1.0 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1.0 - self.b2) * g * g
            mhat = self.m[i] / c1
            vhat = self.v[i] / c2
            out.append(p - self.lr * mhat / (np.sqrt(vhat) + self.eps))
        return out


class Surrogate:
    """A trained stage surrogate: weights plus FP64 normalisation constants."""

    def __init__(self, Ws, bs, mu_in, sd_in, mu_out, sd_out, slopes=None, domain=None):
        self.slopes = None if slopes is None else [float(a) for a in slopes]
        # domain: (lo[6], hi[6]) box of the training inputs; a particle outside
        # it is not mapped by the network (see in_domain)
        self.domain = None if domain is None else (np.asarray(domain[0], dtype=np.float64),
                                                   np.asarray(domain[1], dtype=np.float64))
        self.Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
        self.bs = [np.asarray(b, dtype=np.float64) for b in bs]
        self.mu_in = np.asarray(mu_in, dtype=np.float64)
        self.sd_in = np.asarray(sd_in, dtype=np.float64)
        self.mu_out = np.asarray(mu_out, dtype=np.float64)
        self.sd_out = np.asarray(sd_out, dtype=np.float64)

    def in_domain(self, z):
        """Boolean mask of the particles inside the training-input box (all
        True without a domain). Comparisons are made on the coordinates as
        the tracked particles hold them."""
        if self.domain is None:
            return np.ones(len(np.asarray(z[0])), dtype=bool)
        lo, hi = self.domain
        m = np.ones(len(np.asarray(z[0])), dtype=bool)
        for c in range(6):
            v = np.asarray(z[c], dtype=np.float64)
            m &= ~((v < lo[c]) | (v > hi[c]))
        return m

    def apply(self, z, bf16=False):
        """Map relative coordinates at stage entry to those at stage exit."""
        X = (np.stack([np.asarray(c, dtype=np.float64) for c in z], axis=1) - self.mu_in) / self.sd_in
        Yn = forward(self.Ws, self.bs, X, bf16=bf16, slopes=self.slopes)
        Y = Yn * self.sd_out + self.mu_out
        return [Y[:, j].copy() for j in range(6)]
