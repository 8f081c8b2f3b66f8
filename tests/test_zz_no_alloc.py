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


def test_noalloc_allocates_nothing_on_a_fresh_stream():
    """With every library allocation made to fail (host-side injection) and a
    new stream that has no workspace yet, the call still succeeds and gives
    the same moments: no allocating routine is reached."""
    import torch
    from paper_2402_17248_gb300 import bl
    bl.lib()
    z, g = gaussian_bunch(BunchRecipe(n=123457, seed=22))
    coords = [torch.tensor(z[k], dtype=torch.float32, device="cuda") for k in KEYS]
    b = bl.Bunch(coords, g)
    want = bl.bl_moments(b)
    s = torch.cuda.Stream()
    out = torch.zeros(28, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    bl.bl_debug_fail_allocations(1 << 30)
    try:
        for _ in range(2):
            bl.bl_moments_noalloc(b, out, stream=s)
            s.synchronize()
            _agree(out.cpu().numpy(), want[0], 1e-10)
    finally:
        bl.bl_debug_fail_allocations(0)


def test_noalloc_rejects_inputs_beyond_the_scratch():
    """Too many partial-sum slots: a valid 16-particle bunch split into 32768
    bunches (all but the first empty) needs 1 block + 32768 bunch slots, one
    more than the scratch holds. Every buffer is real, so even a regression in
    the check would launch within bounds."""
    import torch
    from paper_2402_17248_gb300 import bl
    coords = [torch.zeros(16, dtype=torch.float32, device="cuda") for _ in range(6)]
    nb = 32768
    off = np.full(nb + 1, 16, dtype=np.int64)
    off[0] = 0
    b = bl.Bunch(coords, 2000.0, off)
    out = torch.zeros(nb * 28, dtype=torch.float64, device="cuda")
    with pytest.raises(bl.BlError) as e:
        bl.bl_moments_noalloc(b, out)
    assert e.value.status == bl.BL_ERR_INVALID_ARG
    # one bunch fewer fits
    b2 = bl.Bunch(coords, 2000.0, off[:nb])
    bl.bl_moments_noalloc(b2, out)
    torch.cuda.synchronize()


def test_noalloc_rejects_pageable_host_output():
    """A plain host pointer for `out` is refused by the C entry point before
    any work is enqueued (the GPU cannot store to pageable memory)."""
    import ctypes
    import torch
    from paper_2402_17248_gb300 import bl
    coords = [torch.zeros(64, dtype=torch.float32, device="cuda") for _ in range(6)]
    b = bl.Bunch(coords, 2000.0)
    host = np.zeros(28)
    st = bl.lib().bl_moments_noalloc(b.ref(), ctypes.c_void_p(host.ctypes.data),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == bl.BL_ERR_INVALID_ARG
    assert "device-accessible" in bl.lib().bl_last_error_message().decode()
