"""Benchmark: particle-stages/s of the BF16 MLP surrogate beamline versus the
FP32 RK4 wake pusher on the same GPU, with the final-moment error between them.

Workload: a 2^24-particle FP32 Gaussian bunch (1 GeV, eps_n 1 um, sigma_x
2 um, 10 fs, 1 % energy spread) tracked through 8 x (0.3 m plasma stage +
17-element matching section with a 4-dipole chicane), moments after every
element. A step = one pass of the whole beamline with the surrogate stages
(8 tcgen05 MLP launches + 8 fused segment-map/moment passes), starting from
the same initial bunch (restored by a device copy inside the timed region).
The 8 surrogates are first trained on the GPU with the library's own kernels
on pairs that the pusher generates from a randomised 4M-particle population.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank tracks its own bunch (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-stages/s: BF16 MLP surrogate vs FP32 wake pusher, same GPU, moment err"
N_PARTICLES = 1 << 24
N_STAGES = 8
STEPS_PER_STAGE = 400
FLOP_PER_PARTICLE_STAGE = 2 * (6 * 128 + 3 * 128 * 128 + 128 * 6)  # 101,376
SEG_BYTES_PER_PARTICLE = 48
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch on
# 8,388,608 particles in one ncu capture of each current kernel, scaled per
# particle to the launch size: mlp_forward_kernel 201.6 MB + 139.7 MB,
# seg_f32_kernel<apply, moments> 201.6 MB + 140.3 MB (the writes still in L2
# when a kernel ends are not counted)
MLP_DRAM_BYTES_PER_PARTICLE = (201.640448e6 + 139.659520e6) / 8388608
SEG_DRAM_BYTES_PER_PARTICLE = (201.502720e6 + 140.391680e6) / 8388608
DRAM_BASIS = "ncu dram bytes of one launch on 2^23 particles, scaled by the particle count"
# algorithmic flop per particle-stage of a whole gradient: the forward
# surrogate pass plus the VJP (forward recomputation and reverse sweep)
ADJOINT_FLOP_PER_PARTICLE_STAGE = 3 * FLOP_PER_PARTICLE_STAGE
KEYS = ("x", "px", "y", "py", "t", "pt")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    """Roofline denominators: the measured copy bandwidth and BF16 GEMM rates
    of this GPU model (MEASURED_PEAKS.json at the repository root), else the
    fallback figures of one earlier GB300 measurement."""
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {"bf16": p.get("bf16_tflops", 1900.0),
                "bf16_sustained": p.get("bf16_tflops_sustained", 1700.0),
                "hbm": p.get("hbm_gbs", 6800.0), "source": "measured"}
    except (OSError, ValueError):
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "fallback"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--particles", type=int, default=N_PARTICLES)
    p.add_argument("--train-steps", type=int, default=120000)
    p.add_argument("--train-batch", type=int, default=8192)
    p.add_argument("--train-lr", type=float, default=2e-3)
    p.add_argument("--train-pairs", type=int, default=1 << 22)
    p.add_argument("--train-t-scale", type=float, default=8.0,
                   help="first-layer init width on the t input (1 = plain U(+-1/sqrt(fan_in)))")
    p.add_argument("--pusher-steps", type=int, default=2)
    p.add_argument("--cpu-sample", type=int, default=1 << 15)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the batched-bunch, adjoint and training side measurements")
    p.add_argument("--paper-networks-only", action="store_true",
                   help="time only the paper-shaped wide PReLU networks and print their JSON")
    p.add_argument("--paper-particles", type=int, default=10_000_000)
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.rows = []
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ reference arm
def host_cpu():
    """Model name and logical CPU count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model, "logical_cpus": os.cpu_count()}


def cpu_oracle_rate(sample, nets=None, seconds_cap=30.0):
    """Oracle (FP64 numpy) surrogate beamline on a bounded sample; returns
    particle-stages/s, the thread count numpy/BLAS may use and a description."""
    from oracle import beamline, mlp as omlp
    from synth import lattice
    from synth.bunch import BunchRecipe, gaussian_bunch, mlp_init
    z, g = gaussian_bunch(BunchRecipe(n=sample, seed=0))
    zz = [z[k] for k in KEYS]
    if nets is None:
        Ws, bs = mlp_init([6, 128, 128, 128, 128, 6], 1)
        Z = np.stack(zz, axis=1)
        mu, sd = Z.mean(axis=0), Z.std(axis=0)
        nets = [omlp.Surrogate(Ws, bs, mu, sd, mu, sd)] * N_STAGES
    els = lattice.staged_beamline(N_STAGES, STEPS_PER_STAGE)
    i = 0
    for e in els:
        if e["kind"] == "plasma":
            e["surrogate"] = nets[i]
            i += 1
    t = time.perf_counter()
    beamline.track(zz, g, els, snapshots=True)
    dt = time.perf_counter() - t
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return sample * N_STAGES / dt, cores, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    W, K = args.warmup, args.steps
    sample = 4096  # particles per step: about a second of host work, so K steps stay short
    for _ in range(W):
        cpu_oracle_rate(sample)
    t0 = time.perf_counter()
    rates = []
    for _ in range(K):
        r, cores, dt = cpu_oracle_rate(sample)
        rates.append(r)
    total = time.perf_counter() - t0
    value = sample * N_STAGES * K / total
    desc = ("FP64 numpy oracle of the same 8-stage surrogate beamline (moments after every "
            "element) on %d particles per step" % sample)
    line = {"metric": METRIC, "value": value, "unit": "particle-stages/s", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * total / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "8-stage surrogate beamline, FP64 CPU oracle sample",
                       "particles_per_step": sample, "stages": N_STAGES},
            "cpu_baseline": {"value": value, "unit": "particle-stages/s", "cores": cores,
                             "kind": "oracle", "sample": desc, "host": host_cpu()},
            "e2e": {"value": value, "unit": "particle-stages/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def plateau_report(infos):
    """Per stage: steps and seconds of the fit until the held-out loss first
    came within 10 % (and within 2x) of its final value (from the fit's loss
    history; the seconds include the held-out evaluations)."""
    out = []
    for info in infos:
        hist = info.get("history") or []
        if not hist:
            out.append(None)
            continue
        final = hist[-1][1]
        rec = {}
        for name, f in (("within_10pct", 1.1), ("within_2x", 2.0)):
            st, _, sec = next((h for h in hist if h[1] <= f * final), hist[-1])
            rec[name] = {"steps": st, "seconds": round(sec, 2)}
        out.append(rec)
    return out


# ------------------------------------------------------------ side measurements
def side_measurements(args, bl, workflow, lattice, surs, infos, z0, g, elements, dev):
    """Throughput of the other paths on the hot-path list, reported beside the
    headline (not part of it): surrogate training, the batched uneven-bunch
    beamline with per-bunch quadrupoles, the adjoint and the paper's own wide
    PReLU network shapes."""
    import torch
    from synth.bunch import random_quad_magnitudes, uneven_counts
    out = {}
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    # training: samples per second of bl_surrogate_train_step (wall clock of
    # the whole fit, held-out loss evaluations included)
    steps = sum(i["steps"] for i in infos)
    secs = sum(i["seconds"] for i in infos)
    out["training"] = {"samples_per_s": steps * args.train_batch / secs, "batch": args.train_batch,
                       "steps": steps, "seconds": secs,
                       "kernels": "mlp_train_tc_kernel + reduce_adam_kernel + mlp_pack_kernel per step"}
    # the paper's minibatch (1200 pairs, 9.4 tiles of 128): steps of a scratch
    # surrogate on 2^20 random pairs, CUDA events around 280 steps
    from synth.bunch import mlp_init
    Wt, bt = mlp_init([6, 128, 128, 128, 128, 6], 1)
    scratch = bl.Surrogate(Wt, bt, np.zeros(6), np.ones(6), np.zeros(6), np.ones(6))
    gen = torch.Generator(device=dev).manual_seed(0)
    pin = torch.randn(6, 1 << 20, device=dev, generator=gen)
    pout = torch.randn(6, 1 << 20, device=dev, generator=gen)
    pidx = torch.randint(0, 1 << 20, (300, 1200), device=dev, generator=gen)
    for j in range(20):
        bl.bl_surrogate_train_step(scratch, pin, pout, idx=pidx[j], batch=1200, lr=1e-4)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for j in range(20, 300):
        bl.bl_surrogate_train_step(scratch, pin, pout, idx=pidx[j], batch=1200, lr=1e-4)
    ev[1].record(stream)
    torch.cuda.synchronize()
    us = ev[0].elapsed_time(ev[1]) * 1e3 / 280
    out["training"]["paper_batch"] = {"batch": 1200, "us_per_step": us,
                                      "samples_per_s": 1200 / (us * 1e-6)}
    del scratch, pin, pout, pidx

    # batched: 256 bunches with log-uniform counts in [1e4, 1e6] and 32 quad
    # strengths each (magnitudes U[20, 80], signs -,+,-,+), stored back to
    # back, through the 8-stage surrogate beamline with per-bunch moments after
    # every element. Bunch b's particles are counts[b] consecutive particles
    # of the 2^24 pool starting at a seeded offset (wrapping), so no new host
    # draw is needed.
    nbunch = 256
    counts = uneven_counts(nbunch, 1.0e4, 1.0e6, seed=0)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    ntot = int(off[-1])
    pool = z0[0].numel()
    rng = np.random.default_rng(0)
    starts = rng.integers(0, pool, size=nbunch)
    idx = np.concatenate([(st + np.arange(c)) % pool for st, c in zip(starts, counts)])
    idx_d = torch.tensor(idx, device=dev)
    zb0 = [c.index_select(0, idx_d) for c in z0]
    del idx_d
    zb = [c.clone() for c in zb0]
    bb = bl.Bunch(zb, g, offsets=off)
    kmag = random_quad_magnitudes(nbunch, 32, 20.0, 80.0, seed=0)
    signs = np.array([-1.0, 1.0, -1.0, 1.0] * 8)
    els = workflow.surrogate_beamline(elements, surs)
    qi = 0
    for e in els:
        if e["kind"] == "quad":
            e["per_bunch_k"] = (signs[qi] * kmag[:, qi]).copy()
            qi += 1
    # the per-bunch strengths (config 4) mismatch most bunches on purpose, so
    # their particles leave the networks' training domains; this is a
    # throughput configuration, so the surrogates map every particle here
    # instead of handing those to the plain pusher (which loses them as
    # non-finite)
    saved = [s_.domain for s_ in surs]
    for s_ in surs:
        s_.set_domain(None, None)
    lat_b = bl.Lattice(els, n_bunch_k=nbunch)
    # the whole pass (24 launches) captured once as a CUDA graph and replayed;
    # each step restores the input and reads the per-bunch moments back
    tg = bl.TrackGraph(bb, lat_b)

    def step_b():
        for w, s0 in zip(zb, zb0):
            w.copy_(s0, non_blocking=True)
        tg.replay()
        return tg.moments()

    step_b()
    torch.cuda.synchronize()
    kb = 3
    ev[0].record(stream)
    for _ in range(kb):
        m_b, nf_b = step_b()
    ev[1].record(stream)
    torch.cuda.synchronize()
    b_ms = ev[0].elapsed_time(ev[1]) / kb
    out["batched"] = {"value": ntot * N_STAGES / (b_ms * 1e-3), "unit": "particle-stages/s",
                      "ms_per_step": b_ms, "particles": ntot, "bunches": nbunch,
                      "snapshots_per_bunch": len(m_b), "nonfinite": int(nf_b), "cuda_graph": True,
                      "fallback": "off (mismatched bunches leave the training domains)",
                      "workload": "256 bunches, counts floor(exp(U[ln 1e4, ln 1e6])), per-bunch "
                                  "quad strengths, 8 surrogate stages, per-bunch moments after "
                                  "every element"}
    del zb, zb0, bb, tg
    for s_, d in zip(surs, saved):
        if d is not None:
            s_.set_domain(*d)
    torch.cuda.empty_cache()

    # adjoint: d eps_n,x / dk for the 32 quads of the 8-stage surrogate
    # beamline on the first 2^22 particles (forward with checkpoints, reverse
    # sweep, FP64 reductions)
    na = min(1 << 22, z0[0].numel())
    za0 = [c[:na].clone() for c in z0]
    za = [c.clone() for c in za0]
    ba = bl.Bunch(za, g)
    lat_a = bl.Lattice(workflow.surrogate_beamline(elements, surs))

    def step_a():
        for w, s0 in zip(za, za0):
            w.copy_(s0, non_blocking=True)
        ba.struct.gamma_ref = g
        return bl.bl_track_grad(ba, lat_a, "eps_n_x")

    step_a()
    torch.cuda.synchronize()
    ka = 3
    ev[0].record(stream)
    for _ in range(ka):
        J, grad = step_a()
    ev[1].record(stream)
    torch.cuda.synchronize()
    a_ms = ev[0].elapsed_time(ev[1]) / ka
    a_tflops = ADJOINT_FLOP_PER_PARTICLE_STAGE * na * N_STAGES / (a_ms * 1e-3) / 1e12
    pk = load_peaks()
    out["adjoint"] = {"value": na * N_STAGES / (a_ms * 1e-3), "unit": "particle-stages/s",
                      "ms_per_gradient": a_ms, "particles": na, "quads": int(grad.shape[1]),
                      "objective": "eps_n_x", "J": float(J[0]),
                      "timing": "CUDA events on the stream around each bl_track_grad call (the "
                                "call synchronises twice to read moments and dJ/dk)",
                      "roofline": {"bound": "tensor", "achieved": a_tflops,
                                   "peak": pk["bf16_sustained"], "unit": "TFLOP/s",
                                   "frac": a_tflops / pk["bf16_sustained"],
                                   "peak_source": pk["source"] + " bf16 sustained",
                                   "flop_per_particle_stage": ADJOINT_FLOP_PER_PARTICLE_STAGE,
                                   "kernels": "8 mlp_forward + 8 mlp_vjp + segment maps and "
                                              "transposes per gradient"}}
    del za, za0, ba
    torch.cuda.empty_cache()

    out["paper_networks"] = paper_networks(bl, args.paper_particles, g, dev)
    torch.cuda.empty_cache()
    return out


def paper_networks(bl, npw, g, dev, train_steps=1000):
    """The paper's own surrogate shapes (Sec. 4.2): PReLU networks with five
    hidden layers of 900 units and three of 700, on npw particles (1e7 in the
    paper's timing, Sec. 4.3): first as random-init networks applied alone,
    then trained on the GPU (Adam on weights, biases and slopes, a short fit
    on one plasma stage's pusher pairs) and timed as the surrogate stage of a
    lattice (bl_track over the stage and its matching section); the paper's
    A100 figures are context only."""
    import torch
    from paper_2402_17248_gb300 import workflow
    from synth import lattice
    from synth.bunch import BunchRecipe, mlp_init, training_population
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    zw = [torch.randn(npw, device=dev, dtype=torch.float32) for _ in range(6)]
    bw = bl.Bunch(zw, g)
    one, zero = np.ones(6), np.zeros(6)
    rows = []
    g0 = BunchRecipe().gamma_ref
    zt, _ = training_population(4, 65536, g0, 0.2 / workflow.plasma_wavenumber(), seed=1001)
    els = lattice.staged_beamline(1, STEPS_PER_STAGE)
    xin, xout, gin = workflow.stage_pairs(workflow.device_bunch(zt, g0), els)[0]
    zs = workflow.device_bunch(zt, g0)
    pool = [c.repeat((npw + c.numel() - 1) // c.numel())[:npw].contiguous() for c in zs.coords]
    work = [c.clone() for c in pool]
    bs_ = bl.Bunch(work, g0)
    for widths, paper_ns in (([6] + [900] * 5 + [6], 112.0), ([6] + [700] * 3 + [6], 49.4)):
        Ws, bs = mlp_init(widths, 1)
        net = bl.WideSurrogate(Ws, bs, [0.25] * (len(widths) - 2), zero, one, zero, one)
        bl.bl_wide_mlp_apply(net, bw)
        torch.cuda.synchronize()
        kw = 3
        ev[0].record(stream)
        for _ in range(kw):
            bl.bl_wide_mlp_apply(net, bw)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / kw
        H, L = widths[1], len(widths) - 2
        flop = 2 * (6 * H + (L - 1) * H * H + H * 6)
        row = {"hidden": [H] * L, "activation": "PReLU (learned slope)", "particles": npw,
               "ms_per_stage": ms, "ns_per_particle_stage": ms * 1e6 / npw,
               "particle_stages_per_s": npw / (ms * 1e-3),
               "tflops_algorithmic": flop * npw / (ms * 1e-3) / 1e12,
               "paper_A100_ns_per_particle_stage": paper_ns}
        del net
        # trained on the stage's pusher pairs, then as the lattice's stage
        t = time.time()
        tnet, info = workflow.fit_wide_surrogate(xin, xout, widths, steps=train_steps,
                                                 batch=4096, lr=1e-3, seed=3)
        torch.cuda.synchronize()
        lat = bl.Lattice([dict(els[0], surrogate=tnet)] + els[1:])
        for w, s0 in zip(work, pool):
            w.copy_(s0)
        bs_.struct.gamma_ref = gin
        bl.bl_track(bs_, lat, moments=False)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(kw):
            for w, s0 in zip(work, pool):
                w.copy_(s0, non_blocking=True)
            bs_.struct.gamma_ref = gin
            bl.bl_track(bs_, lat, moments=False)
        ev[1].record(stream)
        torch.cuda.synchronize()
        lms = ev[0].elapsed_time(ev[1]) / kw
        row["trained_in_lattice"] = {
            "train_steps": train_steps, "batch": 4096, "train_seconds": time.time() - t,
            "held_out_loss": info["test_loss"], "learned_slopes": info["slopes"],
            "ms_per_stage_and_section": lms, "ns_per_particle_stage": lms * 1e6 / npw,
            "particle_stages_per_s": npw / (lms * 1e-3),
            "timing": "bl_track over the stage (trained network) and its 17-element matching "
                      "section, the input restored by a device copy each pass"}
        rows.append(row)
        del tnet, lat
    peak = load_peaks()["bf16"]
    for r in rows:
        r["frac_of_bf16_peak"] = r["tflops_algorithmic"] / peak
    return rows



# ------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_2402_17248_gb300 import bl, build, workflow
    if not os.path.exists(bl.LIB_PATH):
        build.build()
    bl.lib()
    if args.paper_networks_only:
        print(json.dumps({"paper_networks": paper_networks(bl, args.paper_particles, 2000.0, dev)}),
              flush=True)
        return 0
    from synth import lattice
    from synth.bunch import BunchRecipe, gaussian_bunch

    t_setup = time.time()
    n = args.particles
    # ---- training data from the plain pusher over a randomised population,
    # then one network per stage (held-out loss every 5000 steps at the
    # defaults, for the time to the loss plateau)
    g0 = BunchRecipe().gamma_ref
    elements = lattice.staged_beamline(N_STAGES, STEPS_PER_STAGE)
    surs, infos = workflow.train_beamline_surrogates(
        elements, g0, pairs_per_stage=args.train_pairs, steps=args.train_steps,
        batch=args.train_batch, lr=args.train_lr, t_scale=args.train_t_scale, log_every=5,
        log=log)
    nb, per = infos[0]["pairs"] // 65536, 65536
    log("training done (%.1fs)" % (time.time() - t_setup))

    # ---- the tracked bunch: rank r tracks particles [r n, (r+1) n) of one
    # world*n-particle bunch (weak scaling, no exchange in the data path)
    z, g = gaussian_bunch(BunchRecipe(n=n, seed=0, first_index=rank * n))
    z0 = [torch.tensor(z[k], dtype=torch.float32, device=dev) for k in KEYS]
    host_pinned = [torch.tensor(z[k], dtype=torch.float32).pin_memory() for k in KEYS]
    del z
    work = [c.clone() for c in z0]
    bunch = bl.Bunch(work, g)
    lat_sur = bl.Lattice(workflow.surrogate_beamline(elements, surs))
    lat_push = bl.Lattice(elements)
    nel = lat_sur.num_elements
    stream = torch.cuda.current_stream()

    def restore():
        for w, s in zip(work, z0):
            w.copy_(s, non_blocking=True)
        bunch.struct.gamma_ref = g

    def step_surrogate(moments=True):
        restore()
        return bl.bl_track(bunch, lat_sur, moments=moments)

    # ---- warm-up (also builds the lattice plans) and the moment comparison
    for _ in range(args.warmup):
        m_sur, nf = step_surrogate()
    torch.cuda.synchronize()
    restore()
    m_push, nf_push = bl.bl_track(bunch, lat_push)
    torch.cuda.synchronize()
    g_final = bunch.gamma_ref
    if world > 1:  # moments of the whole bunch from the per-rank moments
        from paper_2402_17248_gb300.shard import gather_moments
        m_sur = gather_moments(m_sur)
        m_push = gather_moments(m_push)
    d_sur = bl.bl_beam_quantities(m_sur[-1][0], g_final)
    d_push = bl.bl_beam_quantities(m_push[-1][0], g_final)
    moment_err = {k: abs(d_sur[k] / d_push[k] - 1) for k in d_push}
    log("final moments surrogate vs pusher:", json.dumps(moment_err))

    # ---- timed surrogate steps (max over ranks)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()  # marks the timed region for a profiler; no-op otherwise
    e0.record(stream)
    for _ in range(args.steps):
        step_surrogate()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = t.item()
    value = world * n * N_STAGES / (ms * 1e-3)
    # per stage: MLP, fused segment map + moments, moment finalize, and the
    # list-mode fallback pusher when the surrogate has a training domain
    launches_per_step = sum(3 + (1 if s_.domain is not None else 0) for s_ in surs)

    # ---- the dominant kernel alone: tcgen05 MLP over the full bunch
    restore()
    bl.bl_surrogate_apply(surs[0], bunch)
    torch.cuda.synchronize()
    reps = 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        bl.bl_surrogate_apply(surs[0], bunch)
    ev[1].record(stream)
    torch.cuda.synchronize()
    mlp_ms = ev[0].elapsed_time(ev[1]) / reps
    mlp_tflops = FLOP_PER_PARTICLE_STAGE * n / (mlp_ms * 1e-3) / 1e12
    # the HBM-bound segment pass the step runs: one fused 17-element section
    # map with the moment reduction at its entry (and its finalize), enqueued
    # through bl_track_async on a lattice whose device plan is cached
    lat_seg = bl.Lattice(lattice.matching_section())
    red_seg = torch.zeros(bl.reduced_size(lat_seg, bunch), dtype=torch.float64, device=dev)
    restore()
    bl.bl_track_async(bunch, lat_seg, red_seg)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        bl.bl_track_async(bunch, lat_seg, red_seg)
    ev[1].record(stream)
    torch.cuda.synchronize()
    seg_ms = ev[0].elapsed_time(ev[1]) / reps
    seg_gbs = SEG_BYTES_PER_PARTICLE * n / (seg_ms * 1e-3) / 1e9
    # and the map alone (no moments), for comparison
    restore()
    bl.bl_track(bunch, lat_seg, moments=False)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        bl.bl_track(bunch, lat_seg, moments=False)
    ev[1].record(stream)
    torch.cuda.synchronize()
    map_ms = ev[0].elapsed_time(ev[1]) / reps

    # ---- the plain FP32 pusher beamline on the same bunch
    restore()
    bl.bl_track(bunch, lat_push, moments=False)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.pusher_steps):
        restore()
        bl.bl_track(bunch, lat_push, moments=True)
    ev[1].record(stream)
    torch.cuda.synchronize()
    push_ms = ev[0].elapsed_time(ev[1]) / args.pusher_steps
    push_value = n * N_STAGES / (push_ms * 1e-3)

    # ---- end to end through the C ABI with host buffers (pinned):
    # bl_track_host copies the bunch in 2^21-particle chunks that run the
    # first stage as they arrive, tracks the stages in between once on the
    # device-resident bunch, and copies each chunk back as soon as it has
    # passed the last stage and section
    out_host = [torch.empty_like(h).pin_memory() for h in host_pinned]
    chunk = 1 << 21

    def e2e_step():
        return bl.bl_track_host(host_pinned, out_host, g, lat_sur, chunk=chunk)

    m_e2e, _, _ = e2e_step()
    torch.cuda.synchronize()
    ke = max(2, args.steps // 2)
    ev[0].record(stream)
    for _ in range(ke):
        e2e_step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = ev[0].elapsed_time(ev[1]) / ke
    e2e_value = world * n * N_STAGES / (e2e_ms * 1e-3)
    # the streamed pass's whole-bunch moments against the device pass's
    # (pooled from the chunks in FP64: equal up to rounding order)
    fin_d, fin_e = np.asarray(m_sur)[-1][0], m_e2e[-1][0]
    e2e_mom_diff = (float(np.max(np.abs(fin_e[7:] - fin_d[7:])) / np.abs(fin_d[7:]).max())
                    if world == 1 else None)
    # the host link itself: the whole bunch copied in, then out, alone
    dev_tmp = [torch.empty_like(c) for c in bunch.coords]
    for d_, h_ in zip(dev_tmp, host_pinned):
        d_.copy_(h_, non_blocking=True)
    torch.cuda.synchronize()
    ev3 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev3[0].record(stream)
    for d_, h_ in zip(dev_tmp, host_pinned):
        d_.copy_(h_, non_blocking=True)
    ev3[1].record(stream)
    for h_, d_ in zip(out_host, dev_tmp):
        h_.copy_(d_, non_blocking=True)
    ev3[2].record(stream)
    torch.cuda.synchronize()
    h2d_ms, d2h_ms = ev3[0].elapsed_time(ev3[1]), ev3[1].elapsed_time(ev3[2])
    del dev_tmp
    nchunks = -(-n // chunk)
    n_red = bl.lib().bl_track_num_reductions(lat_sur.handle)
    n_regions = 2 * nchunks + 1 if nchunks > 1 else 1  # head and tail per chunk, middle once
    h2d = 6 * 4 * n
    d2h = 6 * 4 * n + n_regions * (n_red * 28 + 1) * 8

    extras = {}
    if world == 1 and not args.no_extras:
        extras = side_measurements(args, bl, workflow, lattice, surs, infos, z0, g, elements, dev)

    pk = load_peaks()
    bf16_peak, hbm_peak, peak_src = pk["bf16"], pk["hbm"], pk["source"]

    cpu = cpu_push = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import mlp as omlp
        nets = []
        for s in surs:
            Ws, bs = s.params()
            nets.append(omlp.Surrogate([omlp.bf16_round(W.astype(np.float64)) for W in Ws],
                                       [b.astype(np.float64) for b in bs],
                                       s.mu_in, s.sd_in, s.mu_out, s.sd_out))
        rate, cores, dt = cpu_oracle_rate(args.cpu_sample, nets)
        cpu = {"value": rate, "unit": "particle-stages/s", "cores": cores, "kind": "oracle",
               "host": host_cpu(),
               "sample": "FP64 numpy oracle of the trained 8-stage surrogate beamline with "
                         "moments after every element, %d particles (%.1f s)" % (args.cpu_sample, dt)}
        # the plain method on the host: the oracle's FP64 RK4 stage push
        from oracle import beamline as obeam, wake as owake
        zc, gc = gaussian_bunch(BunchRecipe(n=4096, seed=0))
        t = time.perf_counter()
        owake.push_stage([zc[k] for k in KEYS], gc, obeam.stage_of(elements[0]))
        dtp = time.perf_counter() - t
        cpu_push = {"value": 4096 / dtp, "unit": "particle-stages/s", "cores": cores,
                    "kind": "oracle", "sample": "FP64 numpy oracle RK4 push of 4096 particles "
                    "through one 400-step stage (%.1f s)" % dtp}

    line = {
        "metric": METRIC, "value": value, "unit": "particle-stages/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "2^24-particle FP32 bunch through 8 x (BF16 MLP surrogate stage "
                               "6-128x4-6 GELU + 17-element matching section), moments after "
                               "every element; FP32 400-step RK4 pusher beamline timed beside it",
                   "particles_per_gpu": n, "stages": N_STAGES, "l2": "inputs (384 MiB) larger than L2",
                   "train": {"pairs_per_stage": nb * per, "steps": args.train_steps,
                             "batch": args.train_batch, "lr": args.train_lr,
                             "t_init_scale": args.train_t_scale,
                             "test_loss": [i["test_loss"] for i in infos],
                             "seconds": sum(i["seconds"] for i in infos),
                             "plateau": plateau_report(infos)}},
        "pusher": {"value": push_value, "unit": "particle-stages/s", "ms_per_step": push_ms,
                   "dtype": "f32", "rk4_steps_per_stage": STEPS_PER_STAGE},
        "speedup_vs_pusher": value / push_value,
        "moment_rel_err_vs_pusher": moment_err,
        "roofline": {"bound": "tensor", "achieved": mlp_tflops, "peak": bf16_peak,
                     "unit": "TFLOP/s", "frac": mlp_tflops / bf16_peak,
                     "traffic": MLP_DRAM_BYTES_PER_PARTICLE * n, "traffic_basis": DRAM_BASIS,
                     "kernel": "mlp_forward_kernel", "peak_source": peak_src + " bf16 burst",
                     "ms_per_launch": mlp_ms},
        "roofline_segment": {"bound": "hbm", "achieved": seg_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": seg_gbs / hbm_peak,
                             "traffic": SEG_DRAM_BYTES_PER_PARTICLE * n, "traffic_basis": DRAM_BASIS,
                             "kernel": "seg_f32_kernel<apply, moments> + moments_finalize_kernel "
                                       "(the segment pass of every stage of the step)",
                             "bytes_per_particle": SEG_BYTES_PER_PARTICLE,
                             "ms_per_launch": seg_ms, "map_only_ms_per_launch": map_ms,
                             "peak_source": peak_src + " copy bandwidth"},
        "cpu_baseline": cpu,
        "cpu_baseline_pusher": cpu_push,
        "e2e": {"value": e2e_value, "unit": "particle-stages/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "call": "bl_track_host, page-locked host buffers, %d chunks of 2^21 particles: "
                        "copies in overlap the first stage, copies out the last; the bunch "
                        "stays on the device in between" % nchunks,
                "final_second_moments_max_rel_diff_vs_device": e2e_mom_diff,
                "link": {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
                         "h2d_gbs": 6 * 4 * n / (h2d_ms * 1e-3) / 1e9,
                         "d2h_gbs": 6 * 4 * n / (d2h_ms * 1e-3) / 1e9,
                         "timing": "the bunch copied alone, page-locked host <-> device, "
                                   "CUDA events"}},
        "gpu_launches": launches_per_step * args.steps,
        **extras,
        "clocks": clk,
        "nonfinite": nf,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
