"""Helpers for the GPU parity tests (marshalling between numpy and device)."""
import numpy as np

KEYS = ("x", "px", "y", "py", "t", "pt")


def lib_ready():
    import torch
    if not torch.cuda.is_available():
        return False
    from paper_2402_17248_gb300 import bl
    bl.lib()
    return True


def to_bunch(z, gamma_ref, dtype="f32", offsets=None):
    import torch
    from paper_2402_17248_gb300 import bl
    tdt = torch.float32 if dtype == "f32" else torch.float64
    coords = [torch.tensor(np.asarray(c), dtype=tdt, device="cuda") for c in z]
    return bl.Bunch(coords, gamma_ref, offsets)


def from_bunch(b):
    import torch
    torch.cuda.synchronize()
    return [c.double().cpu().numpy() for c in b.coords]


def as_f32(z):
    return [np.asarray(c, dtype=np.float32).astype(np.float64) for c in z]


def rel_scale_err(a, b, scale):
    """max |a - b| / scale over particles, per coordinate."""
    return [float(np.max(np.abs(np.asarray(x) - np.asarray(y)))) / s for x, y, s in zip(a, b, scale)]
