"""Host-side orchestration of the learned part over the C ABI.

* stage training pairs: a randomised population is tracked with the plain
  RK4 pusher; the entry and exit states of every plasma stage are recorded
  (Sec. 4.1: in/out phase-space arrays of each stage);
* per-coordinate normalisation constants from the library's moment kernel
  (Sec. 3: subtract the mean, divide by the standard deviation);
* a 70/30 train/test split and minibatch Adam on the MSE (Sec. 3, Sec. 4.2),
  every step one bl_surrogate_train_step call.

Nothing here computes the method: each numerical step is a libbl call.
"""
import math
import time

import numpy as np
import torch

from . import bl

KEYS = ("x", "px", "y", "py", "t", "pt")


def device_bunch(z, gamma_ref, dtype=torch.float32, device="cuda"):
    coords = [torch.as_tensor(np.asarray(z[k] if isinstance(z, dict) else z[i]), dtype=dtype,
                              device=device).contiguous()
              for i, k in enumerate(KEYS)]
    return bl.Bunch(coords, gamma_ref)


def split_beamline(elements):
    """[(stage_element, [segment elements that follow]), ...] for a beamline
    that starts with a plasma stage."""
    out = []
    for e in elements:
        if e["kind"] == "plasma":
            out.append((e, []))
        else:
            if not out:
                raise ValueError("beamline must start with a plasma stage")
            out[-1][1].append(e)
    return out


def stage_pairs(bunch, elements):
    """Track `bunch` (FP32, consumed) through the beamline with the plain
    pusher; returns per stage (inputs [6][n], outputs [6][n], gamma_in)."""
    pairs = []
    for stage, seg in split_beamline(elements):
        g_in = bunch.gamma_ref
        xin = torch.stack([c.clone() for c in bunch.coords])
        bl.bl_push_stage(bunch, stage)
        xout = torch.stack([c.clone() for c in bunch.coords])
        pairs.append((xin, xout, g_in))
        if seg:
            lat = bl.Lattice(seg)
            bl.bl_track(bunch, lat, moments=False)
    torch.cuda.synchronize()
    return pairs


def norm_constants(x6):
    """(mean, std) per coordinate of a [6][n] device array via bl_moments."""
    b = bl.Bunch([x6[i] for i in range(6)], 2.0)
    m = bl.bl_moments(b)[0]
    mean = m[1:7].copy()
    var = np.array([m[7 + j] for j in (0, 6, 11, 15, 18, 20)])
    return mean, np.sqrt(np.maximum(var, 1e-300))


def fit_surrogate(xin, xout, steps=20000, batch=1200, lr=1e-3, lr_final=1e-5, seed=0,
                  init_seed=None, test_frac=0.3, log_every=0, widths=bl.WIDTHS, t_scale=1.0,
                  domain=True):
    """Train one stage surrogate on device pairs; returns (surrogate, info).

    t_scale > 1 draws the first layer's weights on the arrival-time input t
    t_scale times wider and the first-layer biases U(+-t_scale/2): inside a
    plasma stage the betatron phase advance depends strongly on a particle's
    wake phase, i.e. on t, so the exit transverse coordinates oscillate many
    times across the bunch in t, and hidden units spread over t resolve that
    (with the default initialisation the transverse outputs stay at their
    mean).

    domain: record the box of the training inputs on the surrogate, so that
    in tracking the particles outside it take the plain pusher instead."""
    from synth.bunch import mlp_init
    n = xin.shape[1]
    ntest = int(round(test_frac * n))
    ntrain = n - ntest
    mu_i, sd_i = norm_constants(xin)
    mu_o, sd_o = norm_constants(xout)
    scale = None if t_scale == 1.0 else [1.0, 1.0, 1.0, 1.0, t_scale, 1.0]
    Ws, bs = mlp_init(list(widths), seed if init_seed is None else init_seed,
                      first_layer_scale=scale,
                      first_bias_range=None if t_scale == 1.0 else 0.5 * t_scale)
    sur = bl.Surrogate(Ws, bs, mu_i, sd_i, mu_o, sd_o)
    xin = xin.contiguous()
    xout = xout.contiguous()
    test_in = xin[:, ntrain:].contiguous()
    test_out = xout[:, ntrain:].contiguous()
    gen = torch.Generator(device=xin.device).manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float64, device=xin.device)
    chunk = 1000
    t0 = time.time()
    history = []
    for s0 in range(0, steps, chunk):
        k = min(chunk, steps - s0)
        idx = torch.randint(0, ntrain, (k, batch), device=xin.device, generator=gen)
        for j in range(k):
            s = s0 + j
            # cosine decay from lr to lr_final
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / max(1, steps)))
            bl.bl_surrogate_train_step(sur, xin, xout, idx=idx[j], batch=batch, lr=a)
        if log_every and ((s0 // chunk) % log_every == 0 or s0 + k >= steps):
            bl.bl_surrogate_loss(sur, test_in, test_out, loss)
            torch.cuda.synchronize()
            history.append((s0 + k, loss.item(), time.time() - t0))
    bl.bl_surrogate_loss(sur, test_in, test_out, loss)
    if domain:
        tr = xin[:, :ntrain]
        sur.set_domain(tr.min(dim=1).values.double().cpu().numpy(),
                       tr.max(dim=1).values.double().cpu().numpy())
    torch.cuda.synchronize()
    info = {"steps": steps, "batch": batch, "lr": lr, "lr_final": lr_final,
            "train_pairs": ntrain, "test_pairs": ntest, "test_loss": loss.item(),
            "seconds": time.time() - t0, "history": history}
    return sur, info


def fit_wide_surrogate(xin, xout, widths, steps=2000, batch=4096, lr=1e-3, lr_final=1e-5,
                       seed=0, slope0=0.25, test_frac=0.3, log_every=0):
    """Train one of the paper's wide PReLU networks (widths 6, H, ..., H, 6;
    every slope starts at slope0 and is learned, Sec. 3) on device pairs
    with the library's wide training step; returns (network, info) with the
    held-out loss history and the learned slopes."""
    from synth.bunch import mlp_init
    n = xin.shape[1]
    ntest = int(round(test_frac * n))
    ntrain = n - ntest
    mu_i, sd_i = norm_constants(xin)
    mu_o, sd_o = norm_constants(xout)
    Ws, bs = mlp_init(list(widths), seed)
    net = bl.WideSurrogate(Ws, bs, [slope0] * (len(widths) - 2), mu_i, sd_i, mu_o, sd_o)
    xin = xin.contiguous()
    xout = xout.contiguous()
    test_idx = torch.arange(ntrain, n, device=xin.device)[:65536]
    gen = torch.Generator(device=xin.device).manual_seed(seed)
    loss = torch.zeros(1, device=xin.device)
    scratch = torch.zeros(net.num_params, device=xin.device)
    history = []

    def test_loss():
        bl.bl_wide_mlp_grad(net, xin, xout, scratch, idx=test_idx, loss_out=loss)
        torch.cuda.synchronize()
        return loss.item()

    t0 = time.time()
    history.append((0, test_loss(), 0.0))
    chunk = max(1, steps // 10) if log_every else steps
    for s0 in range(0, steps, chunk):
        k = min(chunk, steps - s0)
        idx = torch.randint(0, ntrain, (k, batch), device=xin.device, generator=gen)
        for j in range(k):
            s = s0 + j
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / max(1, steps)))
            bl.bl_wide_mlp_train_step(net, xin, xout, idx=idx[j], batch=batch, lr=a)
        if log_every:
            history.append((s0 + k, test_loss(), time.time() - t0))
    final = test_loss()
    info = {"steps": steps, "batch": batch, "lr": lr, "train_pairs": ntrain, "test_pairs": ntest,
            "test_loss": final, "seconds": time.time() - t0, "history": history,
            "slopes": net.params()[2].tolist()}
    return net, info


def plasma_wavenumber(n0_cm3=1.0e17):
    """k_p = omega_p / c of a plasma of electron density n0 [cm^-3] (CODATA 2018)."""
    e, eps0, me, c = 1.602176634e-19, 8.8541878128e-12, 9.1093837015e-31, 299792458.0
    return math.sqrt(n0_cm3 * 1e6 * e * e / (eps0 * me)) / c


def train_beamline_surrogates(elements, gamma_ref, pairs_per_stage=1 << 22, steps=120000,
                              batch=8192, lr=2e-3, t_scale=8.0, seed=1000, log_every=0,
                              log=None):
    """One surrogate per plasma stage of `elements` (one network per stage,
    Sec. 4.2), each trained on the (entry, exit) pairs of its stage from the
    plain pusher tracking a randomised population of 65,536-particle bunches
    (emittance, energy spread and injection phase drawn per bunch, the phase
    jitter +-0.2 rad applied as a centroid shift in t) through the whole
    beamline. Returns (surrogates, infos)."""
    from synth.bunch import training_population
    per = 65536
    nb = max(1, pairs_per_stage // per)
    zt, _ = training_population(nb, per, gamma_ref, 0.2 / plasma_wavenumber(), seed=seed)
    pairs = stage_pairs(device_bunch(zt, gamma_ref), elements)
    surs, infos = [], []
    for s in range(len(pairs)):
        xin, xout, _ = pairs[s]
        sur, info = fit_surrogate(xin, xout, steps=steps, batch=batch, lr=lr, seed=100 + s,
                                  t_scale=t_scale, log_every=log_every)
        info["pairs"] = nb * per
        surs.append(sur)
        infos.append(info)
        pairs[s] = None
        if log:
            log("stage %d surrogate: test loss %.3e after %d steps (%.1fs)"
                % (s + 1, info["test_loss"], info["steps"], info["seconds"]))
    torch.cuda.empty_cache()
    return surs, infos


def surrogate_beamline(elements, surrogates):
    """Copy of `elements` whose plasma stages use the given surrogates, in order."""
    out, i = [], 0
    for e in elements:
        e = dict(e)
        if e["kind"] == "plasma":
            e["surrogate"] = surrogates[i]
            i += 1
        out.append(e)
    return out


def plasma_lens_k(gradient_T_per_m, gamma_ref):
    """Focusing strength [1/m^2] of an active plasma lens with azimuthal field
    gradient g = dB/dr [T/m] for the reference momentum: k = e g / p_ref,
    p_ref = (beta gamma)_ref m_e c (CODATA 2018 constants)."""
    e = 1.602176634e-19
    me_c = 9.1093837015e-31 * 299792458.0
    bg = (gamma_ref * gamma_ref - 1.0) ** 0.5
    return e * gradient_T_per_m / (bg * me_c)

