"""Benchmark: incident rays/s through forward + backward of the ray-wave DOE step.

Workload (default): two spherical singlets behind a planar DOE with a seeded
Zernike + holographic phase map (2048 x 2048 at 1 um), 1M collimated rays
per field (1024 x 1024 grid at 2 um), fields {0, 1, 2} deg x wavelengths
{486, 550, 656} nm = 9 jobs, 64 x 64 patches (exhaustive emission: 4096
secondary rays per incident ray), incoherent 512 x 512 PSF per job at 2 um,
FP32.  One step = ray generation (A0) + fused forward (A1..A7) + Eq. 3 loss
(A8) + adjoint (A9) over all 9.4M incident rays.

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
# DRAM bytes (read + write) per launch at the default workload, from one ncu
# capture of the current kernel at n-side 256 scaled by the incident-ray
# count (16x): see the profiles/ summaries.  A kernel missing here has no
# capture of its current code.
TRAFFIC = {"k_bs_scatter": 16 * (1.535592e9 + 0.192266e9),
           "k_bs_trace": 16 * (1.408312e9 + 0.820282e9),
           "k_cull": 16 * 0.023748e9,
           "k_forward": 16 * (0.310524e9 + 1.472937e9)}
NUM_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-side", type=int, default=1024, help="rays per field = n_side^2")
    ap.add_argument("--cpu-rays", type=int, default=576,
                    help="incident rays per oracle sample (cpu_baseline and the reference arm)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="CPU time the cpu_baseline leg keeps sampling for")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the occupancy-default persistent grids (no rw_autotune)")
    return ap.parse_args()


def workload(n_side):
    import rwinputs as R
    return R.configs.c2(n_side=n_side)


# ------------------------------------------------------------------ algorithmic work
# FP32 operations (each add, multiply, divide, square root and compare
# counted once, an FMA twice) of the kernels of one step.
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


def kernel_flops(name, M, D, S, n_rays, rays_with_items, items, blocks, kept):
    """Algorithmic work of one launch of `name` in the benchmark step."""
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


# ------------------------------------------------------------------ oracle (CPU)
def oracle_step_seconds(w, n_rays, seed=0):
    """Time the FP64 oracle forward + backward (autograd) on a seeded sample
    of n_rays incident rays spread over the jobs.  Returns (seconds, rays)."""
    import torch
    from oracle import loss as OL
    from oracle import pipeline as OP
    rng = np.random.default_rng(seed)
    per = max(1, n_rays // len(w.jobs))
    subsets = [np.sort(rng.choice(j.n_rays, per, replace=False)) for j in w.jobs]
    tgt = torch.from_numpy(w.target.astype(np.float64))
    t0 = time.perf_counter()
    prm = OP.params_of(w.system, requires_grad=True)
    phi = torch.from_numpy(w.system.doe.phi.astype(np.float64)).requires_grad_(True)
    img = OP.psf(w, params=prm, phi=phi, subsets=subsets, chunk=32)
    Lv, _ = OL.eq3_loss(img, tgt)
    Lv.backward()
    return time.perf_counter() - t0, per * len(w.jobs)


def cpu_baseline(w, n_rays, budget_s):
    """Oracle throughput on the host: independent seeded samples of n_rays
    incident rays each (the autograd graph of one sample holds ~10 MB per
    ray), repeated until budget_s seconds of CPU work have been timed."""
    import torch
    secs, n, k = 0.0, 0, 0
    while k == 0 or secs < budget_s:
        s, m = oracle_step_seconds(w, n_rays, seed=1000 + k)
        secs += s
        n += m
        k += 1
    return {"value": n / secs, "unit": "rays/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"{k} seeded samples of {n // k} incident rays ({n // k // len(w.jobs)} "
                      f"per job) of the same workload, each a float64 forward + autograd "
                      f"backward of Eq. 3, {secs:.1f} s in total"}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    import torch
    w = workload(args.n_side)
    per_step = max(len(w.jobs), args.cpu_rays)
    for i in range(args.warmup):
        oracle_step_seconds(w, per_step, seed=100 + i)
    tot, nr = 0.0, 0
    for i in range(args.steps):
        s, n = oracle_step_seconds(w, per_step, seed=i)
        tot += s
        nr += n
    val = nr / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "rays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "incident_rays_per_step_sampled": per_step,
                       "jobs": len(w.jobs), "D": w.system.doe.D},
            "cpu_baseline": {"value": val, "unit": "rays/s", "cores": torch.get_num_threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} seeded incident rays per step"},
            "e2e": {"value": val, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    from paper_2605_15418_gb300 import raywave as RW

    w = workload(args.n_side)
    sysm = w.system
    sim = RW.Simulator(w, device=local)
    n_rays = sim.n_rays
    tgt = torch.as_tensor(w.target, device=dev)
    gI = torch.empty(sim.psf_shape, dtype=torch.float32, device=dev)
    psf = torch.empty(sim.psf_shape, dtype=torch.float32, device=dev)
    dphi = torch.zeros_like(sim.phi)
    dsurf = torch.zeros(len(sysm.surfaces), 8, dtype=torch.float64, device=dev)
    loss = torch.empty(3, dtype=torch.float64, device=dev)
    vis = RW.alloc_vis(n_rays, sysm.doe.M, dev)      # 1 bit per secondary ray
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        s, keep = sim.sys_struct()
        if ev: ev[0].record(stream)
        RW.rw_generate_rays(sim.ctx, w.z_start, sysm.n_object, sim.jobs, sim.rays)
        if ev: ev[1].record(stream)
        RW.rw_forward_vis(sim.ctx, s, sim.jobs, sim.rays, psf, vis)
        if ev: ev[2].record(stream)
        RW.rw_loss_eq3(sim.ctx, psf, tgt, loss, gI)
        dphi.zero_()
        dsurf.zero_()
        if ev: ev[3].record(stream)
        RW.rw_backward_vis(sim.ctx, s, sim.jobs, sim.rays, gI, vis, dphi, None, dsurf)
        if ev: ev[4].record(stream)

    tuned = None
    if not args.no_autotune:
        # one step to size every buffer, then the library's launch tuning (A10)
        step()
        tuned = sim.ctx.autotune(sim, gI, vis)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.ctx.launches
    sim.ctx.profile(True)
    clk.start()
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    clocks = clk.stop()
    prof = sim.ctx.profile_read()
    sim.ctx.profile(False)
    launches = sim.ctx.launches - launches0
    if dist:
        dist.barrier()
    t_step = [evs[k][0].elapsed_time(evs[k][4]) for k in range(args.steps)]
    t_fwd = [evs[k][1].elapsed_time(evs[k][2]) for k in range(args.steps)]
    t_bwd = [evs[k][3].elapsed_time(evs[k][4]) for k in range(args.steps)]
    ms = max_over_ranks(float(np.sum(t_step)), dist, dev)
    ms_per_step = ms / args.steps
    value = weak_scaling_value(n_rays, world, ms_per_step)

    # ---- end to end through the public API with host buffers
    phi_h = torch.from_numpy(np.ascontiguousarray(sysm.doe.phi)).pin_memory()
    tgt_h = torch.from_numpy(np.ascontiguousarray(w.target)).pin_memory()
    psf_h = torch.empty(sim.psf_shape, dtype=torch.float32).pin_memory()
    dphi_h = torch.empty_like(phi_h).pin_memory()
    dsurf_h = torch.empty(len(sysm.surfaces), 8, dtype=torch.float64).pin_memory()
    loss_h = torch.empty(3, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        sim.phi.copy_(phi_h, non_blocking=True)
        tgt.copy_(tgt_h, non_blocking=True)
        step()
        psf_h.copy_(psf, non_blocking=True)
        dphi_h.copy_(dphi, non_blocking=True)
        dsurf_h.copy_(dsurf, non_blocking=True)
        loss_h.copy_(loss, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    h2d = phi_h.numel() * 4 + tgt_h.numel() * 4
    d2h = psf_h.numel() * 4 + dphi_h.numel() * 4 + dsurf_h.numel() * 8 + 24

    # ---- roofline of the dominant kernel (FP32 ALU bound), per-launch times
    # from the library's CUDA events around every launch of the timed steps
    D, M = sysm.doe.D, sysm.doe.M
    lut = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.int64, device=dev)
    vrow = vis.view(n_rays, M * M // 32)
    items = int(lut[vrow.view(torch.uint8).long()].sum().item())
    rays_with_items = int((vrow != 0).any(1).sum().item())
    vfrac = items / float(n_rays * M * M)
    blocks, kept = sim.ctx.cull_stats()
    n_post = len(sysm.surfaces) - sysm.doe_index - 1
    fwd_ms = float(np.mean(t_fwd))
    bwd_ms = float(np.mean(t_bwd))
    peak = NUM_SMS * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12      # TFLOP/s at max SM clock
    kernel_ms = {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}
    modelled = {k: kernel_flops(k, M, D, n_post, n_rays, rays_with_items, items, blocks, kept)
                for k in kernel_ms}
    name = max((k for k in kernel_ms if modelled[k] is not None), key=lambda k: prof[k][0])
    tms = kernel_ms[name]
    achieved = modelled[name] / (tms / 1e3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "incident_rays": n_rays, "jobs": len(w.jobs),
                       "D": D, "secondary_rays_per_incident": D * D, "sensor": "512x512x9",
                       "surfaces_after_doe": n_post, "l2": "flushed between steps (256 MB)",
                       "visible_secondary_fraction": vfrac,
                       "traced_secondary_fraction": (64.0 * kept / (n_rays * M * M)
                                                     if blocks else 1.0),
                       "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
                       "kernel_ms": {k: round(v, 4) for k, v in kernel_ms.items()},
                       "tuned_grids": tuned},
            "roofline": {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": TRAFFIC.get(name),
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal)"},
            "e2e": {"value": world * n_rays / (e2e_ms / 1e3), "unit": "rays/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_rays, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
