"""Particle sharding across ranks (one process per GPU).

Particles are independent (paper Sec. 1: per-particle maps without collective
effects; Sec. 2: node-local inference on each subset of the distributed
particles), so rank r simply tracks its own contiguous share of the bunch with
no exchange in the data path. The only cross-rank step is turning per-rank
moments into moments of the whole bunch: each rank contributes its
28-vector [N, means, central second moments] and the pooled values follow
from the parallel-variance combination (counts add; the pooled mean is the
count-weighted mean; pooled central moments add each part's central moments
plus the scatter of its mean about the pooled mean), evaluated in FP64.
"""
import numpy as np

PAIRS = [(a, b) for a in range(6) for b in range(a, 6)]


def shard_range(n_total, rank, world):
    """Contiguous particle range [lo, hi) of `rank` for a bunch of n_total."""
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def combine_moments(parts):
    """Pool a list of 28-vectors (each [N, 6 means, 21 central moments, 1/N])."""
    parts = [np.asarray(p, dtype=np.float64) for p in parts]
    N = sum(p[0] for p in parts)
    out = np.zeros(28)
    out[0] = N
    if N == 0:
        return out
    mean = sum(p[0] * p[1:7] for p in parts) / N
    out[1:7] = mean
    for j, (a, b) in enumerate(PAIRS):
        s = 0.0
        for p in parts:
            if p[0] == 0:
                continue
            da, db = p[1 + a] - mean[a], p[1 + b] - mean[b]
            s += p[0] * (p[7 + j] + da * db)
        out[7 + j] = s / N
    return out


def gather_moments(m, group=None):
    """All-gather per-rank moment arrays [..., 28] and pool them on every rank."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(m, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    bufs = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(bufs, t, group=group)
    arrs = [b.cpu().numpy() for b in bufs]
    flat = [a.reshape(-1, 28) for a in arrs]
    pooled = np.stack([combine_moments([f[i] for f in flat]) for i in range(flat[0].shape[0])])
    return pooled.reshape(np.shape(m))
