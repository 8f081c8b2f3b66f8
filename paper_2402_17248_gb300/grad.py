"""torch.autograd binding of the beamline adjoint.

`beam_objective(k, bunch, elements, objective)` returns the objective J of
the final beam moments (normalised emittance or rms spot size, Sec. 4.4's
figures of merit for the focusing lattice) as a function of the quadrupole
strengths k, and its backward pass is the library's hand-written adjoint
(`bl_track_grad`: one forward pass with stage checkpoints, one reverse pass
through the transposed element maps and the surrogates' vector-Jacobian
products). The forward pass tracks a copy of the bunch, so the caller's
particles are left untouched.

k is a float64 tensor of shape [n_quads] (one set of strengths for every
bunch) or [n_bunch, n_quads] (per-bunch strengths); the quads are taken in
lattice order. J has shape [n_bunch].
"""
import numpy as np
import torch

from . import bl


def _with_strengths(elements, k):
    nq = sum(e["kind"] == "quad" for e in elements)
    if k.shape[-1] != nq:
        raise ValueError("k has %d strengths, the lattice has %d quadrupoles" % (k.shape[-1], nq))
    out, q = [], 0
    for e in elements:
        e = dict(e)
        if e["kind"] == "quad":
            if k.ndim == 1:
                e["k"] = float(k[q])
                e.pop("per_bunch_k", None)
            else:
                e["per_bunch_k"] = np.ascontiguousarray(k[:, q], dtype=np.float64)
            q += 1
        out.append(e)
    return out


class TrackGrad(torch.autograd.Function):
    """J(k) through bl_track_grad; d J / d k from the adjoint."""

    @staticmethod
    def forward(ctx, k, bunch, elements, objective):
        kh = k.detach().to("cpu", torch.float64).numpy()
        if kh.ndim == 2 and kh.shape[0] != bunch.n_bunch:
            raise ValueError("per-bunch k needs one row per bunch")
        lat = bl.Lattice(_with_strengths(elements, kh), n_bunch_k=bunch.n_bunch if kh.ndim == 2 else 0)
        work = bl.Bunch([c.clone() for c in bunch.coords], bunch.gamma_ref,
                        offsets=bunch.offsets_host)
        J, g = bl.bl_track_grad(work, lat, objective)
        ctx.save_for_backward(torch.from_numpy(g).to(k.device))
        ctx.per_bunch = kh.ndim == 2
        return torch.from_numpy(J).to(k.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        gk = gJ[:, None].to(g.dtype) * g
        if not ctx.per_bunch:
            gk = gk.sum(dim=0)
        return gk, None, None, None


def beam_objective(k, bunch, elements, objective="eps_n_x"):
    return TrackGrad.apply(k, bunch, elements, objective)
