"""Multi-rank host logic on CPU: sharding ranges and the pooled moments of a
bunch split across ranks (gloo, world size 2), checked against the moments
of the whole bunch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import moments
from paper_2402_17248_gb300.shard import combine_moments, gather_moments, shard_range
from synth.bunch import BunchRecipe, gaussian_bunch

KEYS = ("x", "px", "y", "py", "t", "pt")


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 1000, 16777216):
        for w in (1, 2, 3, 8):
            r = [shard_range(n, k, w) for k in range(w)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[i][1] == r[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1


def test_combine_equals_whole_bunch():
    z, g = gaussian_bunch(BunchRecipe(n=10007, seed=3))
    zz = [z[k] for k in KEYS]
    zz[4] = zz[4] + 1e-5 * np.arange(10007) / 10007  # structure across shards
    whole = moments.moments28(zz)
    for w in (2, 3, 5):
        parts = [moments.moments28([c[slice(*shard_range(10007, k, w))] for c in zz]) for k in range(w)]
        pooled = combine_moments(parts + [np.zeros(28)])
        S = moments.sigma_matrix(whole)
        sd = np.sqrt(np.diag(S))
        assert pooled[0] == whole[0]
        assert np.max(np.abs(pooled[1:7] - whole[1:7]) / sd) < 1e-13
        for j, (a, b) in enumerate(moments.PAIRS):
            assert abs(pooled[7 + j] - whole[7 + j]) <= 1e-12 * sd[a] * sd[b]


def _worker(rank, world, port, n, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=7))
    lo, hi = shard_range(n, rank, world)
    mine = moments.moments28([z[k][lo:hi] for k in KEYS])
    # two snapshots per rank, as bl_track returns one per element
    m = np.stack([mine, mine * np.array([1.0] + [2.0] * 6 + [4.0] * 21)])
    pooled = gather_moments(m)
    q.put((rank, pooled))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_gloo_two_ranks_pool_moments():
    n = 20001
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=7))
    whole = moments.moments28([z[k] for k in KEYS])
    S = moments.sigma_matrix(whole)
    sd = np.sqrt(np.diag(S))
    for r in (0, 1):
        got = res[r][0]
        assert got[0] == n
        assert np.max(np.abs(got[1:7] - whole[1:7]) / sd) < 1e-13
        for j, (a, b) in enumerate(moments.PAIRS):
            assert abs(got[7 + j] - whole[7 + j]) <= 1e-12 * sd[a] * sd[b]
    assert np.array_equal(res[0], res[1])
