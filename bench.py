"""Benchmark: incident rays/s through forward + backward of the ray-wave DOE step.

Headline workload (default --config c5): the batched end-to-end design
workload -- three spherical singlets behind a planar DOE carrying the seeded
Zernike + holographic phase map (2048 x 2048 at 1 um); 31 wavelengths
(400-700 nm) x 16 fields (4 x 4 over +-1.5 deg) = 496 jobs with uneven,
log-uniform ray counts; 96 x 96 patches; sampled emission with 1024
Gumbel-max draws per incident ray; incoherent 512 x 512 PSF per job at 2 um;
FP32.  One step = ray generation (A0) + fused forward (A1..A7) + Eq. 3 loss
(A8) + adjoint with the straight-through Gumbel-softmax (A9) over every
incident ray of all 496 jobs in one persistent launch per kernel.  The
workload's ray counts are 64k..2M per job (2.8e8 rays); the sampled method
costs N x M^2 = 9.4e6 Gumbel scores per incident ray and pass, so the
benchmark divides every job's count range by --c5-scale (stated in config).

Also measured (nested under "also"): the full C2 step (two singlets, planar
DOE, 9 jobs of 1M rays, 64 x 64 patches, exhaustive emission with exact
block culling, taped adjoint over the visibility mask); the C4 forward
(conformal DOE on a sphere behind an even asphere, 4096^2 map, 27 jobs of
4M rays, bilinear 64 x 64 patches) with the FP32 FFT ("c4") and with the
tcgen05 patch transform fused into the forward ("c4tc").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun every rank runs its own copy of the
workload (weak scaling, no data-path collective); value = rays of all ranks
/ max-over-ranks time.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("rays/s fwd+bwd through DOE ray–wave step at PSF err≤1e-4 vs FP64; "
          "% HBM/TC peak")
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16
C5_FULL_LO, C5_FULL_HI = 65536, 2 * 1024 * 1024
# DRAM bytes (read + write) per launch of the C2 step at full size, from one
# ncu capture of the current kernels at n-side 256 scaled by the incident-ray
# count (16x), as the profiles/ summaries record.
C2_TRAFFIC = {"k_bs_scatter": 16 * (1.584282e9 + 0.201948e9),
              "k_bs_trace": 16 * (1.421939e9 + 0.822920e9),
              "k_cull": 16 * 0.023777e9,
              "k_forward": 16 * (0.316977e9 + 1.525885e9)}


# DRAM bytes (read + write) per incident ray of the C5 kernels, from one ncu
# capture of the current kernels on the same workload with its ray counts
# divided by 32768 (9,270 rays; the launch's traffic grows with the rays:
# dL/dPSF reads and PSF atomics per draw): see the profiles/ summaries.
C5_TRAFFIC_PER_RAY = {"k_backward": (913.137408e6 + 274.656512e6) / 9270,
                      "k_forward": (594.386944e6 + 50.164224e6) / 9270}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5", choices=["c5", "c2"])
    ap.add_argument("--c5-scale", type=int, default=4096,
                    help="C5 ray counts per job divided by this (64k..2M -> 16..512 at 4096)")
    ap.add_argument("--n-side", type=int, default=1024, help="C2 rays per field = n_side^2")
    ap.add_argument("--also", default="c2,c4,c4tc,c1",
                    help="comma-separated extra workloads measured after the headline ('' = "
                         "none); c4tc is the C4 forward with the tensor-core patch transform, "
                         "c1 the grating's secondary rays written to HBM (rw_doe_emit)")
    ap.add_argument("--c1-n-side", type=int, default=512,
                    help="C1 rays per incidence angle = n_side^2 (emit line)")
    ap.add_argument("--c4-n-side", type=int, default=2048,
                    help="C4 rays per field = n_side^2 (2048: 4M, the stated workload)")
    ap.add_argument("--also-steps", type=int, default=5)
    ap.add_argument("--also-warmup", type=int, default=3)
    ap.add_argument("--cpu-rays", type=int, default=0,
                    help="incident rays per oracle sample (0: the workload's default)")
    ap.add_argument("--parity-rays", type=int, default=0,
                    help="incident rays of the parity sample (0: the workload's default)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU time the cpu_baseline leg keeps sampling for")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the occupancy-default persistent grids (no rw_autotune)")
    return ap.parse_args()


# ------------------------------------------------------------------ workloads
def workload(name, args):
    import rwinputs as R
    if name == "c5":
        s = max(1, int(args.c5_scale))
        return R.configs.c5(count_lo=max(1, C5_FULL_LO // s), count_hi=max(4, C5_FULL_HI // s))
    if name in ("c4", "c4tc"):
        return R.configs.c4(n_side=args.c4_n_side)
    if name == "c1":
        return R.configs.c1(n_side=args.c1_n_side)
    return R.configs.c2(n_side=args.n_side)


def default_cpu_rays(name):
    # incident rays per oracle sample: the C2 oracle runs ~500 rays/s, the C5
    # one (1024 draws over 96^2 bins per ray, fwd + bwd) a few seconds per ray
    return 576 if name == "c2" else 8


# ------------------------------------------------------------------ algorithmic work
# C2 (exhaustive emission, FP32 tracing): FP32 operations, each add,
# multiply, divide, square root and compare counted once, an FMA twice.
def fft_flops(M):
    """Radix FFT count of one M x M patch transform: 5 N log2 N, N = M^2."""
    return 5.0 * M * M * math.log2(M * M)


def bin_fwd_flops(S):
    """One traced secondary ray: emission 45, each spherical surface 65
    (intersection 20 + 3 sqrt/div, hit 6, normal 15, Snell 20), sensor +
    bilinear splat 20."""
    return 45.0 + 65.0 * S + 20.0


def bin_bwd_flops(S):
    """Re-trace of one visible secondary ray plus its reverse (emission 40,
    each surface 150, sensor 40)."""
    return bin_fwd_flops(S) + 40.0 + 150.0 * S + 40.0


def block_test_flops(S):
    """Affine-arithmetic test of one 8 x 8 block of bins for a group of rays
    (affine forms with four noise terms): direction setup ~200, each sphere
    ~1,290 (21 affine products at 34, 25 sums/scalings at 14, five square
    roots / reciprocals at 45), sensor plane ~200."""
    return 400.0 + 1290.0 * S


def c4_kernel_flops(name, M, n_rays, blocks, kept):
    """Algorithmic FP32 work of one launch of `name` in the C4 forward
    (conformal DOE, bilinear patch gather, no surface behind the DOE)."""
    if name in ("k_forward", "k_forward_tc"):
        # gather: per sample 4 complex taps x 2 FMAs + the weights (~20);
        # every kept bin is emitted and splat (no surface to trace)
        return n_rays * (fft_flops(M) + 20.0 * M * M) + 64.0 * kept * bin_fwd_flops(0)
    if name == "k_cull":
        # conformal DOE: one affine test per (ray, 8 x 8 block of bins)
        return float(blocks) * block_test_flops(0)
    return None


def c2_kernel_flops(name, M, D, S, n_rays, rays_with_items, items, blocks, kept):
    """Algorithmic FP32 work of one launch of `name` in the C2 step."""
    if name == "k_forward":
        traced = 64.0 * kept if blocks else float(n_rays) * M * M
        return n_rays * fft_flops(M) + traced * bin_fwd_flops(S)
    if name == "k_cull":
        # planar DOE: one test per block covers a group of 8 rays of one job
        return blocks / 8.0 * block_test_flops(S)
    if name == "k_bs_spectra":
        return rays_with_items * fft_flops(M) + items * 30.0
    if name == "k_bs_trace":
        return items * bin_bwd_flops(S)
    if name == "k_bs_scatter":
        return rays_with_items * (fft_flops(M) + 8.0 * D * D) + items * 20.0
    return None


# C5 (sampled emission): the work is the (draw, bin) Gumbel score, N x M^2
# per incident ray and pass.  Counted in 32-bit lane operations at
# instruction granularity (an FMA, an integer multiply-wide, a 3-input
# logical op, a compare: one each); multi-function-unit operations (log2,
# reciprocal) are counted separately against their own, eight times
# lower, rate.  Philox4x32-10 takes 10 rounds x (2 multiply-wide + 2
# three-input xor) = 40 ops per block of 4 words: 10 per score.
#   forward: 10 (Philox) + 1 (threshold compare)                 = 11 ALU
#   adjoint pass A: 10 + 13 (-log u: convert, 1 - u, series of 5 FMAs, the
#     log2 branch, select) + 1 (t = p e) + 5 (sums) + 4 (screen test)
#     + 2 (broadcast loads)                                     = 35 ALU, 2 MUFU
#   adjoint pass B: 10 + 13 + 6 (accumulators)                   = 29 ALU, 2 MUFU
C5_FWD_ALU, C5_BWD_ALU, C5_BWD_MUFU = 11.0, 35.0 + 29.0, 4.0


def tc_mma_flops(D):
    """Tensor-core work of one D x D patch transform in the BF16x3 form: two
    stages, each one real (2D x 2D) by (2D x D) product per split term
    (hi hi, hi lo, lo hi), 2 M N K flops apiece."""
    return 2 * 3 * 2.0 * (2 * D) * D * (2 * D)


def c5_kernel_work(name, n_rays, M, N):
    """(ALU lane-ops, MUFU lane-ops) of one launch of `name` in the C5 step."""
    pairs = float(n_rays) * N * M * M
    if name == "k_forward":
        return pairs * C5_FWD_ALU, 0.0
    if name == "k_backward":
        return pairs * C5_BWD_ALU, pairs * C5_BWD_MUFU
    return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample(w, n_rays, seed):
    """Seeded sample of about n_rays incident rays of `w`: contiguous runs of
    ray indices (so that the GPU run on the same runs draws the same sampling
    stream), at least 4 rays per sampled job (a PSF of a single incident ray
    is dominated by the rounding of its few deposits).  Returns per-job index
    lists."""
    import rwinputs as R
    njob = len(w.jobs)
    per = max(1, n_rays // njob)
    starts, subsets = R.ray_blocks(w.jobs, max(per, 4), seed)
    if per < 4:
        rng = np.random.default_rng(seed)
        keep = set(rng.choice(njob, max(1, n_rays // 4), replace=False).tolist())
        subsets = [s if j in keep else s[:0] for j, s in enumerate(subsets)]
    return subsets


def oracle_step(w, subsets):
    """FP64 oracle forward + autograd backward of Eq. 3 on the sample; returns
    (seconds, rays, PSF stack)."""
    import torch
    from oracle import loss as OL
    from oracle import pipeline as OP
    tgt = torch.from_numpy(w.target.astype(np.float64))
    chunk = 32 if w.system.doe.emit == "exhaustive" else 1
    t0 = time.perf_counter()
    prm = OP.params_of(w.system, requires_grad=True)
    phi = torch.from_numpy(w.system.doe.phi.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, params=prm, phi=phi, subsets=subsets, chunk=chunk)
    Lv, _ = OL.eq3_loss(img, tgt)
    Lv.backward()
    return time.perf_counter() - t0, int(sum(len(s) for s in subsets)), img.detach().numpy()


def parity_sample(w, n_rays, seed=4242):
    """The oracle's FP64 PSF (forward only) of a seeded sample of about n_rays
    incident rays, for the GPU's parity on the same rays."""
    import torch
    from oracle import pipeline as OP
    sub = oracle_sample(w, n_rays, seed)
    chunk = 32 if w.system.doe.emit == "exhaustive" else 1
    with torch.no_grad():
        img = OP.psf(w, subsets=sub, chunk=chunk).numpy()
    return sub, img


def default_parity_rays(name):
    # the sampled PSF of a few rays is a few thousand deposits, each carrying
    # its own hit rounding: parity wants enough rays for deposits to overlap
    return 576 if name == "c2" else 64


def cpu_baseline(w, n_rays, budget_s):
    """Oracle throughput on the host: independent seeded samples of n_rays
    incident rays, repeated until budget_s seconds of CPU work were timed.
    Also returns the first sample and its PSF (the parity check)."""
    import torch
    secs, n, k = 0.0, 0, 0
    first = None
    while k == 0 or secs < budget_s:
        sub = oracle_sample(w, n_rays, seed=1000 + k)
        s, m, img = oracle_step(w, sub)
        if first is None:
            first = (sub, img)
        secs += s
        n += m
        k += 1
    return ({"value": n / secs, "unit": "rays/s", "cores": torch.get_num_threads(),
             "kind": "oracle",
             "sample": f"{k} seeded samples of {n // k} incident rays (contiguous runs in "
                       f"seeded jobs) of the same workload, each a float64 forward + "
                       f"autograd backward of Eq. 3, {secs:.1f} s in total"}, first)


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    import torch
    w = workload(args.config, args)
    per_step = args.cpu_rays or default_cpu_rays(args.config)
    for i in range(args.warmup):
        oracle_step(w, oracle_sample(w, per_step, seed=100 + i))
    tot, nr = 0.0, 0
    for i in range(args.steps):
        s, n, _ = oracle_step(w, oracle_sample(w, per_step, seed=i))
        tot += s
        nr += n
    val = nr / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.config, w, args),
            "cpu_baseline": {"value": val, "unit": "rays/s", "cores": torch.get_num_threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} seeded incident rays per step"},
            "e2e": {"value": val, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(name, w, args):
    """The workload description shared by both arms."""
    d = w.system.doe
    c = {"workload": w.name, "incident_rays": w.n_rays, "jobs": len(w.jobs), "D": d.D,
         "emission": d.emit, "sensor": f"{w.system.sensor.nx}x{w.system.sensor.ny}x{len(w.jobs)}",
         "surfaces_after_doe": len(w.system.surfaces) - w.system.doe_index - 1,
         "l2": "flushed between steps (256 MB)"}
    if name == "c5":
        s = max(1, int(args.c5_scale))
        c.update({"n_ssr": d.n_ssr, "ray_count_range": [max(1, C5_FULL_LO // s),
                                                        max(4, C5_FULL_HI // s)],
                  "reduced": f"ray counts per job divided by {s} (full workload: "
                             f"{C5_FULL_LO}..{C5_FULL_HI} per job)"})
    return c


# ------------------------------------------------------------------ ranks
def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over all ranks (the job's time is its slowest rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(rays_per_rank, world, ms_per_step):
    """Whole-job incident rays/s: every rank runs its own replica."""
    return world * rays_per_rank / (ms_per_step / 1e3)


# ------------------------------------------------------------------ our arm
class Step:
    """One fwd + Eq. 3 + bwd step of a workload through the C ABI."""

    def __init__(self, name, w, dev, local, dft="fft32"):
        import torch
        from paper_2605_15418_gb300 import raywave as RW
        self.RW, self.name, self.w = RW, name, w
        self.fwd_only = name in ("c4", "c4tc")  # the C4 workload is a forward study
        if w.target is None:
            w.target = np.zeros((len(w.jobs), w.system.sensor.ny, w.system.sensor.nx),
                                np.float32)
        self.sim = RW.Simulator(w, device=local, dft=dft)
        sim = self.sim
        self.tgt = torch.as_tensor(w.target, device=dev)
        self.gI = torch.empty(sim.psf_shape, dtype=torch.float32, device=dev)
        self.psf = torch.empty(sim.psf_shape, dtype=torch.float32, device=dev)
        self.dphi = torch.zeros_like(sim.phi)
        self.dsurf = torch.zeros(len(w.system.surfaces), 8, dtype=torch.float64, device=dev)
        self.loss = torch.empty(3, dtype=torch.float64, device=dev)
        # C2: one visibility bit per secondary ray, taped split adjoint
        self.vis = RW.alloc_vis(sim.n_rays, w.system.doe.M, dev) if name == "c2" else None

    def __call__(self, ev=None, stream=None):
        RW, sim = self.RW, self.sim
        s, keep = sim.sys_struct()
        if ev: ev[0].record(stream)
        RW.rw_generate_rays(sim.ctx, self.w.z_start, self.w.system.n_object, sim.jobs, sim.rays)
        if ev: ev[1].record(stream)
        if self.vis is not None:
            RW.rw_forward_vis(sim.ctx, s, sim.jobs, sim.rays, self.psf, self.vis)
        else:
            RW.rw_forward(sim.ctx, s, sim.jobs, sim.rays, self.psf)
        if ev: ev[2].record(stream)
        if self.fwd_only:
            if ev: ev[3].record(stream); ev[4].record(stream)
            return
        RW.rw_loss_eq3(sim.ctx, self.psf, self.tgt, self.loss, self.gI)
        self.dphi.zero_()
        self.dsurf.zero_()
        if ev: ev[3].record(stream)
        if self.vis is not None:
            RW.rw_backward_vis(sim.ctx, s, sim.jobs, sim.rays, self.gI, self.vis, self.dphi,
                               None, self.dsurf)
        else:
            RW.rw_backward(sim.ctx, s, sim.jobs, sim.rays, self.gI, self.dphi, None, self.dsurf)
        if ev: ev[4].record(stream)


def time_steps(st, steps, warmup, flush, dev, autotune, dist, local, sample_clocks):
    """Warm-up, then `steps` timed steps with an L2 flush between them;
    per-kernel times from the library's CUDA events around every launch."""
    import torch
    sim = st.sim
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if autotune:
        st()
        tuned = sim.ctx.autotune(sim, st.gI, st.vis)
    for _ in range(warmup):
        st()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    clk = ClockSampler(local) if sample_clocks else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.ctx.launches
    sim.ctx.profile(True)
    if clk:
        clk.start()
    for k in range(steps):
        flush.zero_()
        st(evs[k], stream)
    torch.cuda.synchronize()
    clocks = clk.stop() if clk else None
    prof = sim.ctx.profile_read()
    sim.ctx.profile(False)
    launches = sim.ctx.launches - launches0
    if dist:
        dist.barrier()
    t_step = [evs[k][0].elapsed_time(evs[k][4]) for k in range(steps)]
    t_fwd = [evs[k][1].elapsed_time(evs[k][2]) for k in range(steps)]
    t_bwd = [evs[k][3].elapsed_time(evs[k][4]) for k in range(steps)]
    return {"ms": float(np.sum(t_step)), "fwd_ms": float(np.mean(t_fwd)),
            "bwd_ms": float(np.mean(t_bwd)), "prof": prof, "launches": int(launches),
            "clocks": clocks, "tuned": tuned}


def e2e_rate(st, steps, dev, world):
    """The same step through the public API with host buffers: the DOE map and
    the target come from pinned host memory, and the PSF, dL/dphi, the surface
    gradients and the loss go back, every step, inside the timed region."""
    import torch
    sim = st.sim
    stream = torch.cuda.current_stream(dev)
    phi_h = torch.from_numpy(np.ascontiguousarray(st.w.system.doe.phi)).pin_memory()
    tgt_h = torch.from_numpy(np.ascontiguousarray(st.w.target)).pin_memory()
    psf_h = torch.empty(sim.psf_shape, dtype=torch.float32).pin_memory()
    dphi_h = torch.empty_like(phi_h).pin_memory()
    dsurf_h = torch.empty(len(st.w.system.surfaces), 8, dtype=torch.float64).pin_memory()
    loss_h = torch.empty(3, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        sim.phi.copy_(phi_h, non_blocking=True)
        st.tgt.copy_(tgt_h, non_blocking=True)
        st()
        psf_h.copy_(st.psf, non_blocking=True)
        dphi_h.copy_(st.dphi, non_blocking=True)
        dsurf_h.copy_(st.dsurf, non_blocking=True)
        loss_h.copy_(st.loss, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h2d = phi_h.numel() * 4 + tgt_h.numel() * 4
    d2h = psf_h.numel() * 4 + dphi_h.numel() * 4 + dsurf_h.numel() * 8 + 24
    return {"value": world * sim.n_rays / (ms / 1e3), "unit": "rays/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def gpu_parity(st, subsets, ref):
    """PSF relative L2 of the GPU on the oracle's sample against the oracle's
    FP64 PSF of it (same rays, same launch configuration)."""
    import rwinputs as R
    import torch
    RW, sim, w = st.RW, st.sim, st.w
    off = R.jobs_offsets(w.jobs)
    starts = [int(s[0]) if len(s) else 0 for s in subsets]
    jobs = RW.jobs_struct(w.jobs, offsets=[int(off[j]) + starts[j] for j in range(len(w.jobs))],
                          counts=[len(s) for s in subsets])
    s, keep = sim.sys_struct()
    psf = torch.empty(sim.psf_shape, dtype=torch.float32, device=st.psf.device)
    RW.rw_forward(sim.ctx, s, jobs, sim.rays, psf)
    torch.cuda.synchronize()
    got = psf.cpu().numpy().astype(np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def roofline_c5(tm, st, peaks, n_sms, clocks):
    """ALU (and MUFU) roofline of the dominant kernel of the C5 step."""
    prof = tm["prof"]
    d = st.w.system.doe
    M, N = d.M, d.n_ssr
    kernel_ms = {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}
    work = {k: c5_kernel_work(k, st.sim.n_rays, M, N) for k in kernel_ms}
    name = max((k for k in kernel_ms if work[k] is not None), key=lambda k: prof[k][0])
    t = kernel_ms[name] / 1e3
    alu, mufu = work[name]
    f = 2070e6
    alu_peak = n_sms * FP32_LANES_PER_SM * f / 1e12
    mufu_peak = n_sms * MUFU_LANES_PER_SM * f / 1e12
    a_alu, a_mufu = alu / t / 1e12, mufu / t / 1e12
    fr_alu, fr_mufu = a_alu / alu_peak, a_mufu / mufu_peak
    return kernel_ms, {
        "kernel": name, "bound": "alu", "achieved": a_alu, "peak": alu_peak,
        "unit": "Tops/s (32-bit lane ops)", "frac": fr_alu,
        "traffic": (C5_TRAFFIC_PER_RAY[name] * st.sim.n_rays
                    if name in C5_TRAFFIC_PER_RAY else None),
        "peak_source": f"{n_sms} SMs x 128 lanes x 2070 MHz (one 32-bit op per lane per "
                       "clock; nominal unit counts and the maximum SM clock)",
        "other_bounds": {"mufu": {"achieved": a_mufu, "peak": mufu_peak, "frac": fr_mufu,
                                  "peak_source": f"{n_sms} SMs x 16 MUFU lanes x 2070 MHz"},
                         "hbm": {"frac": (C5_TRAFFIC_PER_RAY.get(name, 0.0) * st.sim.n_rays
                                          / t / 1e9 / peaks["hbm_gbs"])}},
        "work_per_launch": {"pairs": float(st.sim.n_rays) * N * M * M,
                            "alu_ops_per_pair": C5_FWD_ALU if name == "k_forward"
                            else C5_BWD_ALU,
                            "mufu_ops_per_pair": 0.0 if name == "k_forward" else C5_BWD_MUFU}}


# bytes rw_doe_emit writes per secondary ray (dx, dy, dz, a_re, a_im, bin)
# and per incident ray (hit x, y, z, optical path), and reads per incident ray
# (its nine ray fields); the map and the job table stay in L2
EMIT_W_SEC, EMIT_W_RAY, EMIT_R_RAY = 24, 20, 36


def emit_line(w, args, dev, local, flush, peaks, dist=None, world=1):
    """C1: the planar grating's secondary rays written to HBM by rw_doe_emit,
    timed with CUDA events on the launching stream (the output, larger than
    L2, is written every step; the flush buffer is zeroed between steps)."""
    import torch
    from paper_2605_15418_gb300 import raywave as RW
    sim = RW.Simulator(w, device=local)
    M = w.system.doe.M
    out = RW.alloc_emitted(sim.n_rays, M * M, dev)
    s, keep = sim.sys_struct()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.also_warmup):
        RW.rw_doe_emit(sim.ctx, s, sim.jobs, sim.rays, out)
    torch.cuda.synchronize()
    ms = []
    sim.ctx.profile(True)
    for _ in range(args.also_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        RW.rw_doe_emit(sim.ctx, s, sim.jobs, sim.rays, out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = sim.ctx.profile_read()
    sim.ctx.profile(False)
    kernel_ms = {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}
    t = max_over_ranks(float(np.mean(ms)), dist, dev)
    kt = kernel_ms.get("k_forward", t)
    nbytes = sim.n_rays * (M * M * EMIT_W_SEC + EMIT_W_RAY + EMIT_R_RAY)
    gbs = nbytes / (kt / 1e3) / 1e9
    cfg = {"workload": w.name, "incident_rays": sim.n_rays, "jobs": len(w.jobs), "D": M,
           "emission": "exhaustive", "step": "rw_doe_emit: every secondary ray to HBM",
           "bytes_per_launch": nbytes, "kernel_ms": {k: round(v, 4) for k, v in kernel_ms.items()}}
    roof = {"kernel": "k_forward (MODE_EMIT)", "bound": "hbm", "achieved": gbs,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "traffic": None}
    res = {"value": weak_scaling_value(sim.n_rays, world, t), "unit": "rays/s", "ms_per_step": t,
           "steps": args.also_steps, "warmup": args.also_warmup, "config": cfg,
           "roofline": roof}
    del out, sim
    torch.cuda.empty_cache()
    return res


def roofline_c4(tm, st, n_sms, peaks=None):
    """FP32 roofline of the dominant kernel of the C4 forward; with the
    tensor-core transform also its tcgen05 throughput against the measured
    bf16 peak."""
    prof = tm["prof"]
    M = st.w.system.doe.M
    blocks, kept = st.sim.ctx.cull_stats()
    peak = n_sms * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    kernel_ms = {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}
    modelled = {k: c4_kernel_flops(k, M, st.sim.n_rays, blocks, kept) for k in kernel_ms}
    name = max((k for k in kernel_ms if modelled[k] is not None), key=lambda k: prof[k][0])
    achieved = modelled[name] / (kernel_ms[name] / 1e3) / 1e12
    extra = {"traced_secondary_fraction": (64.0 * kept / (st.sim.n_rays * M * M)
                                           if blocks else 1.0)}
    if name == "k_forward_tc" and peaks is not None:
        tens = st.sim.n_rays * tc_mma_flops(M) / (kernel_ms[name] / 1e3) / 1e12
        extra["tensor_core"] = {"achieved": tens, "peak": peaks["bf16_tflops"],
                                "unit": "TFLOP/s", "frac": tens / peaks["bf16_tflops"],
                                "flops_per_ray": tc_mma_flops(M)}
    return kernel_ms, extra, {
        "kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
        "peak_source": f"{n_sms} SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal)"}


def red_peak(sim, dev, win=64, nwin=1 << 18):
    """Float atomic-add (reduction) throughput of this GPU in the adjoint's
    scatter pattern: rw_probe_red onto a 2048 x 2048 map (L2-resident, like
    dL/dphi), CUDA events, best of three after a warm-up; adds per second."""
    import torch
    m = torch.zeros(2048, 2048, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sim.ctx.probe_red(m, win, nwin)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.ctx.probe_red(m, win, nwin)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return float(win) * win * nwin / (best / 1e3)


def roofline_c2(tm, st, n_sms):
    """FP32 roofline of the dominant kernel of the C2 step."""
    import torch
    prof = tm["prof"]
    sysm = st.w.system
    D, M = sysm.doe.D, sysm.doe.M
    n_rays = st.sim.n_rays
    lut = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.int64,
                       device=st.vis.device)
    vrow = st.vis.view(n_rays, M * M // 32)
    items = int(lut[vrow.view(torch.uint8).long()].sum().item())
    rays_with_items = int((vrow != 0).any(1).sum().item())
    blocks, kept = st.sim.ctx.cull_stats()
    n_post = len(sysm.surfaces) - sysm.doe_index - 1
    peak = n_sms * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    kernel_ms = {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}
    modelled = {k: c2_kernel_flops(k, M, D, n_post, n_rays, rays_with_items, items, blocks,
                                   kept) for k in kernel_ms}
    name = max((k for k in kernel_ms if modelled[k] is not None), key=lambda k: prof[k][0])
    achieved = modelled[name] / (kernel_ms[name] / 1e3) / 1e12
    extra = {"visible_secondary_fraction": items / float(n_rays * M * M),
             "traced_secondary_fraction": (64.0 * kept / (n_rays * M * M) if blocks else 1.0)}
    if "k_bs_scatter" in kernel_ms:
        # the scatter's dL/dphi adds (one per patch sample of every ray with
        # visible bins; two with an amplitude map) against the measured
        # reduction throughput in the same pattern
        adds = rays_with_items * D * D * (2 if sysm.doe.amp is not None else 1)
        rate = adds / (kernel_ms["k_bs_scatter"] / 1e3)
        red_pk = red_peak(st.sim, st.vis.device)
        extra["k_bs_scatter_red"] = {"achieved": rate, "peak": red_pk, "unit": "adds/s",
                                     "frac": rate / red_pk,
                                     "peak_source": "rw_probe_red: 64 x 64 windows on a "
                                                    "2048^2 float map, measured here"}
    return kernel_ms, extra, {
        "kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": C2_TRAFFIC.get(name),
        "peak_source": f"{n_sms} SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal)"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, peak_kind = measured_peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    name = args.config
    w = workload(name, args)
    st = Step(name, w, dev, local)
    tm = time_steps(st, args.steps, args.warmup, flush, dev,
                    autotune=(name == "c2" and not args.no_autotune), dist=dist, local=local,
                    sample_clocks=True)
    ms_per_step = max_over_ranks(tm["ms"], dist, dev) / args.steps
    value = weak_scaling_value(st.sim.n_rays, world, ms_per_step)
    e2e = e2e_rate(st, max(1, min(args.steps, 3)), dev, world)
    cfg = config_of(name, w, args)
    cfg.update({"fwd_ms": tm["fwd_ms"], "bwd_ms": tm["bwd_ms"]})
    if name == "c5":
        kernel_ms, roof = roofline_c5(tm, st, peaks, n_sms, tm["clocks"])
    else:
        kernel_ms, extra, roof = roofline_c2(tm, st, n_sms)
        cfg.update(extra)
        cfg["tuned_grids"] = tm["tuned"]
    cfg["kernel_ms"] = {k: round(v, 4) for k, v in kernel_ms.items()}
    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg, "roofline": roof, "e2e": e2e,
            "gpu_launches": tm["launches"], "clocks": tm["clocks"],
            "peak_memory_gb": torch.cuda.max_memory_allocated(dev) / 1e9}

    # ---- the other workloads, fewer steps each
    also = []
    for other in [x for x in args.also.split(",") if x and x != name]:
        wo = workload(other, args)
        if other == "c1":
            also.append(emit_line(wo, args, dev, local, flush, peaks, dist, world))
            continue
        so = Step(other, wo, dev, local, dft="tc" if other == "c4tc" else "fft32")
        to = time_steps(so, args.also_steps, args.also_warmup, flush, dev,
                        autotune=(other == "c2" and not args.no_autotune), dist=dist,
                        local=local, sample_clocks=False)
        mso = max_over_ranks(to["ms"], dist, dev) / args.also_steps
        co = config_of(other, wo, args)
        co.update({"fwd_ms": to["fwd_ms"], "bwd_ms": to["bwd_ms"]})
        if other == "c5":
            kmo, ro = roofline_c5(to, so, peaks, n_sms, None)
        elif other in ("c4", "c4tc"):
            kmo, exo, ro = roofline_c4(to, so, n_sms, peaks)
            co.update(exo)
            co["step"] = "ray generation + forward (the C4 workload is a forward study)"
            co["patch_transform"] = ("tcgen05 BF16x3 F X F^T" if other == "c4tc"
                                     else "FP32 shared-memory FFT")
        else:
            kmo, exo, ro = roofline_c2(to, so, n_sms)
            co.update(exo)
        co["kernel_ms"] = {k: round(v, 4) for k, v in kmo.items()}
        also.append({"value": weak_scaling_value(so.sim.n_rays, world, mso), "unit": "rays/s",
                     "ms_per_step": mso, "steps": args.also_steps,
                     "warmup": args.also_warmup, "config": co, "roofline": ro,
                     "gpu_launches": to["launches"]})
        del so
        torch.cuda.empty_cache()
    if also:
        line["also"] = also

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_cpu = args.cpu_rays or default_cpu_rays(name)
        cb, _ = cpu_baseline(w, n_cpu, args.cpu_seconds)
        line["cpu_baseline"] = cb
        sub, ref = parity_sample(w, args.parity_rays or default_parity_rays(name))
        line["parity"] = {"psf_rel_l2": gpu_parity(st, sub, ref), "bar": 1e-4,
                          "rays": int(sum(len(s) for s in sub)),
                          "sample": "seeded contiguous runs of incident rays, the same rays "
                                    "on both sides, oracle forward in FP64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
