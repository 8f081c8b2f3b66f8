"""The C-ABI library loads and exports every declared symbol; host-only calls
and argument checks (no GPU needed)."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2402_17248_gb300 import bl
from oracle import wake
from synth import lattice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2402_17248_gb300 import build
    build.build()


def _declared():
    names = set()
    for h in ("bl.h", "bl_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(bl_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", bl.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (bl_[a-z0-9_]+)", out))
    missing = names - exported
    assert not missing, missing
    L = bl.lib()
    for n in names:
        assert hasattr(L, n)


def test_reference_exit_matches_oracle():
    st = lattice.plasma(400)
    for g in (1957.9511835591836, 6111.38, 30000.0):
        want = wake.reference_exit(wake.Stage(nsteps=400), g)[0]
        got = bl.bl_reference_exit(st, g)
        assert abs(got / want - 1) < 1e-12


def test_lattice_create_counts_and_validation():
    L = bl.Lattice(lattice.staged_beamline(2, 10))
    assert L.num_elements == 36
    assert L.num_quads == 8
    with pytest.raises(bl.BlError) as e:
        bl.Lattice([{"kind": "plasma", "L": 0.3, "nsteps": 0, "n0_cm3": 1e17,
                     "E0_Vpm": 1e10, "phi0": 0.7}])
    assert e.value.status == bl.BL_ERR_INVALID_ARG
    with pytest.raises(bl.BlError):
        bl.Lattice([{"kind": "quad", "L": 0.1, "k": float("nan")}])
    with pytest.raises(bl.BlError):
        bl.Lattice([{"kind": "quad", "L": 0.1, "k": 1.0, "per_bunch_k": [1.0, 2.0]}])
    with pytest.raises(bl.BlError):
        bl.bl_reference_exit(lattice.plasma(10), 0.5)
    # plasma lenses: a linear element, not a differentiated strength, no per-bunch k
    L = bl.Lattice([lattice.drift(0.1), lattice.plasma_lens(0.03, 2000.0), lattice.quad(0.1, 5.0)])
    assert L.num_elements == 3 and L.num_quads == 1
    with pytest.raises(bl.BlError):
        bl.Lattice([{"kind": "plasma_lens", "L": 0.03, "k": 1.0, "per_bunch_k": [1.0]}], n_bunch_k=1)
    with pytest.raises(bl.BlError):
        bl.Lattice([{"kind": "plasma_lens", "L": 0.03, "k": float("inf")}])


def test_per_bunch_lattice():
    els = [{"kind": "quad", "L": 0.1, "k": 30.0, "per_bunch_k": [20.0, 40.0, 60.0]},
           {"kind": "drift", "L": 1.0}]
    L = bl.Lattice(els, n_bunch_k=3)
    assert L.num_quads == 1


def test_beam_quantities_match_oracle():
    from oracle import moments
    from synth.bunch import BunchRecipe, gaussian_bunch
    z, g = gaussian_bunch(BunchRecipe(n=5000, seed=8))
    zz = [z[k] for k in ("x", "px", "y", "py", "t", "pt")]
    zz[5] = zz[5] + 0.3 * np.std(zz[5])
    zz[1] = zz[1] + 0.5 * zz[0] / 2e-6 * np.std(zz[1])
    m = moments.moments28(zz)
    want = moments.derived(m, g)
    got = bl.bl_beam_quantities(m, g)
    for k in want:
        assert abs(got[k] / want[k] - 1) < 1e-13, k


def _surrogate_file(tmp_path, widths=(6, 128, 128, 128, 128, 6), checksum_ok=True, cut=0):
    """Bytes in the surrogate file format (see bl_surrogate_save)."""
    import struct
    n = 51206
    body = b"BLSURR01" + struct.pack("<i", 1) + struct.pack("<6i", *widths)
    body += struct.pack("<24d", *([0.0] * 6 + [1.0] * 6 + [0.0] * 6 + [1.0] * 6))
    body += struct.pack("<i", 0) + struct.pack("<12f", *([0.0] * 12)) + struct.pack("<i", 0)
    body += np.zeros(3 * n, dtype=np.float32).tobytes()
    h = 1469598103934665603
    for byte in body:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    if not checksum_ok:
        h ^= 1
    data = body + struct.pack("<Q", h)
    if cut:
        data = data[:-cut]
    p = tmp_path / "s.blsurr"
    p.write_bytes(data)
    return p


def test_surrogate_file_validation_before_allocation(tmp_path):
    """A surrogate file is validated on the host before any device work:
    missing, truncated, corrupted (checksum) or foreign-shaped files are
    rejected with BL_ERR_INVALID_ARG."""
    with pytest.raises(bl.BlError) as e:
        bl.Surrogate.load(tmp_path / "missing.blsurr")
    assert e.value.status == bl.BL_ERR_INVALID_ARG
    for kw in ({"checksum_ok": False}, {"cut": 100}, {"widths": (6, 64, 64, 64, 64, 6)}):
        with pytest.raises(bl.BlError) as e:
            bl.Surrogate.load(_surrogate_file(tmp_path, **kw))
        assert e.value.status == bl.BL_ERR_INVALID_ARG, kw
    bad = tmp_path / "bad.blsurr"
    bad.write_bytes(b"NOTASURR" + bytes(64))
    with pytest.raises(bl.BlError):
        bl.Surrogate.load(bad)


def test_track_host_validation_before_any_work():
    """bl_track_host rejects bad arguments on the host, before touching a GPU
    (stream 0: no CUDA call is made to look one up)"""
    L = bl.Lattice([lattice.drift(0.1), lattice.quad(0.1, 5.0)])
    a = [np.zeros(8, dtype=np.float32) for _ in range(6)]
    for kw in ({"gamma_ref": 1.0}, {"gamma_ref": float("nan")}, {"chunk": -1}):
        args = {"gamma_ref": 2000.0, "chunk": 0}
        args.update(kw)
        with pytest.raises(bl.BlError) as e:
            bl.bl_track_host(a, a, args["gamma_ref"], L, chunk=args["chunk"], stream=0)
        assert e.value.status == bl.BL_ERR_INVALID_ARG
    empty = [np.zeros(0, dtype=np.float32) for _ in range(6)]
    with pytest.raises(bl.BlError) as e:
        bl.bl_track_host(empty, empty, 2000.0, L, stream=0)
    assert e.value.status == bl.BL_ERR_INVALID_ARG
    Lb = bl.Lattice([{"kind": "quad", "L": 0.1, "k": 30.0, "per_bunch_k": [20.0, 40.0, 60.0]}],
                    n_bunch_k=3)
    with pytest.raises(bl.BlError) as e:
        bl.bl_track_host(a, a, 2000.0, Lb, stream=0)
    assert e.value.status == bl.BL_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        bl.bl_track_host(a, [np.zeros(8, dtype=np.float64)] * 6, 2000.0, L, stream=0)


def _moments28(Z):
    """[N, 6 means, 21 central second moments (1/N), a <= b row by row]"""
    out = np.zeros(28)
    if len(Z) == 0:
        return out
    mu = Z.mean(axis=0)
    C = (Z - mu).T @ (Z - mu) / len(Z)
    out[0], out[1:7] = len(Z), mu
    out[7:] = [C[a, b] for a in range(6) for b in range(a, 6)]
    return out


def test_pool_moments_equals_moments_of_the_union():
    """The FP64 pooling bl_track_host applies to chunked reductions (host code
    of the library) equals the moments of the union computed directly: the
    chunks have different sizes (one empty), offsets of several sigma and
    different spreads, so a missing or wrong parallel-axis term fails."""
    rng = np.random.default_rng(5)
    sizes = [1, 7, 1000, 0, 123457, 4096]
    chunks = [rng.normal(loc=3.0 * rng.normal(size=6), scale=rng.uniform(0.5, 2.0, size=6),
                         size=(m, 6)) for m in sizes]
    parts = np.ascontiguousarray(np.stack([_moments28(c) for c in chunks]))
    out = np.zeros(28)
    assert bl.lib().bl_debug_pool_moments(parts.ctypes.data, len(sizes), out.ctypes.data) == 0
    want = _moments28(np.concatenate(chunks))
    sd = np.sqrt(want[[7, 13, 18, 22, 25, 27]])
    scale = np.concatenate([[want[0]], sd, [sd[a] * sd[b] for a in range(6) for b in range(a, 6)]])
    assert np.max(np.abs(out - want) / scale) < 1e-12
    # one set pools to itself; bad arguments are refused
    one = np.zeros(28)
    assert bl.lib().bl_debug_pool_moments(parts[2].ctypes.data, 1, one.ctypes.data) == 0
    assert np.allclose(one, parts[2], rtol=1e-15, atol=0.0)
    assert bl.lib().bl_debug_pool_moments(parts.ctypes.data, 0, out.ctypes.data) == 1


def _prototypes():
    """name -> number of parameters of every function declared in include/*.h"""
    protos = {}
    for h in ("bl.h", "bl_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(bl_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
            params = m.group(2).strip()
            protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return protos


def test_binding_arity_matches_the_header():
    """every function the header declares is bound in bl.py with the same
    number of arguments (a mismatch would silently shift arguments)"""
    protos = _prototypes()
    assert len(protos) >= 20
    for name, n in protos.items():
        assert name in bl._SIGS, name
        assert len(bl._SIGS[name][0]) == n, (name, len(bl._SIGS[name][0]), n)


def test_noalloc_binding_rejects_unusable_output_before_any_call():
    """bl_moments_noalloc's binding refuses a host, wrongly typed, strided or
    short `out` before it reaches the library (its kernel stores
    n_bunch * 28 doubles through that pointer)."""
    import types
    import torch
    fake = types.SimpleNamespace(n_bunch=2)
    bad = [torch.zeros(56, dtype=torch.float64),               # host memory
           np.zeros(56)]                                        # not a tensor
    for out in bad:
        with pytest.raises(bl.BlError) as e:
            bl.bl_moments_noalloc(fake, out)
        assert e.value.status == bl.BL_ERR_INVALID_ARG
    if torch.cuda.is_available():
        for out in (torch.zeros(56, dtype=torch.float32, device="cuda"),
                    torch.zeros(112, dtype=torch.float64, device="cuda")[::2],
                    torch.zeros(55, dtype=torch.float64, device="cuda")):
            with pytest.raises(bl.BlError):
                bl.bl_moments_noalloc(fake, out)
