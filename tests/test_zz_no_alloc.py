"""The allocation-free moment entry point (bl_moments_noalloc) gives the same
moments as bl_moments, through the C ABI, on two calls in a row.

It serves callers that may not allocate device memory (a framework's caching
allocator owns it, real-time code reserved it all up front, or an implicit
synchronisation of cudaMalloc/cudaFree is not acceptable); its scratch is a
fixed device array inside the library. This file is collected last on
purpose."""
import math

import numpy as np
import pytest

from synth.bunch import BunchRecipe, gaussian_bunch

pytestmark = pytest.mark.gpu
KEYS = ("x", "px", "y", "py", "t", "pt")


def _agree(got, want, tol):
    assert got[0] == want[0]
    if want[0] < 2:
        return
    sd = np.sqrt([max(want[7 + j], 1e-300) for j in (0, 6, 11, 15, 18, 20)])
    pairs = [(a, b) for a in range(6) for b in range(a, 6)]
    for a in range(6):
        assert abs(got[1 + a] - want[1 + a]) <= tol * sd[a]
    for j, (a, b) in enumerate(pairs):
        assert abs(got[7 + j] - want[7 + j]) <= tol * sd[a] * sd[b]


def test_noalloc_matches_bl_moments_on_two_calls():
    import torch
    from paper_2402_17248_gb300 import bl
    bl.lib()
    counts = [70000, 0, 1, 4096, 250003, 17]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    z, g = gaussian_bunch(BunchRecipe(n=int(off[-1]), seed=21))
    coords = [torch.tensor(z[k], dtype=torch.float32, device="cuda") for k in KEYS]
    b = bl.Bunch(coords, g, off)
    want = bl.bl_moments(b)
    for call in range(2):
        out = torch.full((len(counts) * 28,), float("nan"), dtype=torch.float64, device="cuda")
        bl.bl_moments_noalloc(b, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(len(counts), 28)
        for i in range(len(counts)):
            _agree(got[i], want[i], 1e-10)
    # a second, smaller bunch reuses the same scratch
    small = bl.Bunch([c[:999].clone() for c in coords], g)
    out = torch.zeros(28, dtype=torch.float64, device="cuda")
    bl.bl_moments_noalloc(small, out)
    torch.cuda.synchronize()
    _agree(out.cpu().numpy(), bl.bl_moments(small)[0], 1e-10)


def test_noalloc_rejects_inputs_beyond_the_scratch():
    import torch
    from paper_2402_17248_gb300 import bl
    coords = [torch.zeros(16, dtype=torch.float32, device="cuda") for _ in range(6)]
    b = bl.Bunch(coords, 2000.0)
    b.struct.n = (32768 + 1) * 4096      # larger than the fixed scratch allows
    out = torch.zeros(28, dtype=torch.float64, device="cuda")
    with pytest.raises(bl.BlError) as e:
        bl.bl_moments_noalloc(b, out)
    assert e.value.status == bl.BL_ERR_INVALID_ARG
