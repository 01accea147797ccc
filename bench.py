#!/usr/bin/env python
"""Benchmark of the GB300 map-maker on the ground-based workload.

Workload: 512 detectors x 4 stationary intervals x 524,288 samples (1.07e9 samples), a 1024x1024
IQU patch, raster scan with a rotating half-wave plate, 1/f noise (f_knee 1 Hz, alpha 1.5,
per-detector sigma ~ U(0.8, 1.2)), banded inverse-noise weights with lambda = 8192; seeded
synthetic data generated on the device.

One step = one whole pass of the hot path on resident inputs: the right-hand side
b = P^T N^-1 d and a mixed-precision PCG solve to rel. residual 1e-6 (FP32 P, N^-1, P^T in the
iterations; FP64 vectors, dot products, alpha/beta and 3x3 blocks; the right-hand side and the
residual replacements apply the operators in double-float arithmetic, pairs of FP32 numbers with
a 48-bit significand, which runs on the FP32 pipes).  The timed steps run the library as a user
would (iteration groups replayed as CUDA graphs); one extra profiled solve afterwards brackets
every operator launch with CUDA events for the kernel split and the roofline object.  The plan
(pixel compaction, block-Jacobi blocks, pixel windows, spectra) is built once before the timed
region; the e2e number rebuilds it from pinned host buffers in every step and hands the host TOD
to the library.

value  = TOD samples pushed through A per second (N x A-applications per step / step time),
         summed over ranks.  Extra keys give solves/s, PCG iterations/s, the map error of the
         mixed-precision solve against a full FP64-class (double-float) PCG solve of the same
         right-hand side and against the FP64 CPU oracle on a detector cut, and a `secondary`
         object with the other workloads (tiny FP64 PCG, satellite BD vs two-level, batched block
         CG, serving).
--impl reference runs the FP64 CPU oracle (numpy/scipy) on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TOD samples/s through A=PᵀN⁻¹P; PCG solves/s + p50/p99 at map err ≤1e-6"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_FILE = os.path.join(ROOT, "profiles", "ninv32_ground.json")
FP32_LANES_PER_SM = 128


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dets", type=int, default=512, help="detectors (512 = the full workload)")
    p.add_argument("--samples", type=int, default=524288,
                   help="samples per block (524288 = the full workload; fewer: a cut for profiling)")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--cpu-dets", type=int, default=2, help="CPU baseline: detectors per oracle worker")
    p.add_argument("--cut-dets", type=int, default=8, help="oracle map-error cut: detectors")
    p.add_argument("--cut-samp", type=int, default=262144, help="oracle map-error cut: samples per block")
    p.add_argument("--workload", default="ground",
                   choices=["ground", "batched", "satellite", "serving", "ecg", "deflation", "noise",
                            "templates", "tiny", "crossover"])
    p.add_argument("--nrhs", type=int, default=64, help="batched: noise realisations")
    p.add_argument("--widths", default="8,16,32,64", help="batched: block widths")
    p.add_argument("--enlarge", default="1,4,16,64", help="ecg: enlarging factors t")
    p.add_argument("--requests", type=int, default=200, help="serving: requests")
    p.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    p.add_argument("--lams", default="0,16,32,64,96,128", help="crossover: half-bandwidths")
    p.add_argument("--iters", type=int, default=20, help="crossover: PCG iterations per algorithm")
    return p.parse_args()


# ------------------------------------------------------------------------------------------
# roofline helpers
# ------------------------------------------------------------------------------------------

def fft_flops_per_sample(L: int, lam: int) -> float:
    """Algorithmic flops per output sample of the overlap-save Toeplitz product: a real forward
    and inverse FFT of L points (2.5 L log2 L each) plus the pointwise product (3 L), shared by
    the L - 2 lam outputs the tile keeps."""
    return (5.0 * L * math.log2(L) + 3.0 * L) / (L - 2 * lam)


def kernel_source_hash() -> str:
    """Hash of the FP32 N^-1 tile kernel's own source (k_toeplitz.cu, fft_smem.cuh, df64.cuh and
    the TileArgs definition it is compiled against)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2112_03370_gb300", "csrc")
    for f in ("df64.cuh", "fft_smem.cuh", "k_toeplitz.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    internal = open(os.path.join(d, "mm_internal.cuh")).read()
    a = internal.index("struct TileArgs")
    h.update(internal[a:internal.index("\n};", a)].encode())
    return h.hexdigest()[:16]


def measured_traffic(n_samples: int):
    """DRAM bytes per launch of the FP32 N^-1 tile from the committed ncu summary, scaled to this
    launch; None when absent or taken on different kernel source."""
    try:
        prof = json.load(open(PROFILE_FILE))
    except Exception:
        return None
    if prof.get("kernel_source_hash") != kernel_source_hash():
        return None
    return prof["dram_bytes_per_sample"] * n_samples


def peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.rows = []
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:   # no nvidia-smi: report no clocks
            log("clock sampler unavailable:", e)
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        rows = self.rows
        if self.bus_id:
            mine = [r for r in rows if len(r) > 1 and r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 6 + i and r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# CPU oracle baseline: independent oracle instances on the host cores, each on its own
# detectors of the same workload (the oracle itself is single-threaded numpy/scipy)
# ------------------------------------------------------------------------------------------

def _oracle_worker(job):
    """One oracle instance (spawned process): plan, right-hand side, then `n_iter` PCG iterations
    (A-apply + Algorithm 1 vector work) on detectors [d0, d1) x 1 interval; returns the samples of
    one iteration and the seconds of each iteration."""
    d0, d1, n_iter = job
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    import synth
    cfg = synth.ground_config(n_int=1)
    prob = synth.make_ground_problem(cfg, det_range=(d0, d1))
    nb = synth.to_numpy(prob)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], nb["band"], nb["n_pix"])
    b = O.rhs(op, nb["d"])
    x = O.precond_bd(op, b)
    times = []
    for _ in range(n_iter):
        t0 = time.perf_counter()
        y = O.apply_A(op, x)
        den = float(np.vdot(y, x))
        a = float(np.vdot(b, x)) / den if den != 0.0 else 0.0
        x = x + a * O.precond_bd(op, b - y)
        times.append(time.perf_counter() - t0)
    return int(nb["pix"].size), times


def cpu_oracle_rate(dets_per_worker: int, n_iter: int = 2, skip: int = 0, workers: int = 0):
    """Samples/s through A (PCG iterations) of `workers` concurrent oracle instances (default: one
    per host core), each on its own detectors x 1 interval x 524,288 samples of the ground
    workload, over iterations skip..n_iter-1 of each.  Returns (value, cores, description,
    per-iteration values)."""
    import multiprocessing as mpr
    cores = workers or len(os.sched_getaffinity(0))
    jobs = [(dets_per_worker * i % 512, dets_per_worker * i % 512 + dets_per_worker, n_iter)
            for i in range(cores)]
    ctx = mpr.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    n_it = n_iter - skip
    samples = sum(n * n_it for n, _ in res)
    busy = max(sum(ts[skip:]) for _, ts in res)
    per_iter = [sum(n for n, _ in res) / max(ts[i] for _, ts in res) for i in range(skip, n_iter)]
    desc = (f"{cores} concurrent oracle processes (numpy/scipy FP64, one thread each), each on "
            f"{dets_per_worker} detectors x 1 interval x 524288 samples of the ground workload, "
            f"{n_it} timed PCG iterations (A-apply + vector update) each; rate = total samples / the "
            f"slowest worker's time ({busy:.1f} s; {wall:.0f} s with set-up); CPU: {cpu_model()}")
    return samples / busy, cores, desc, per_iter


def ground_config_json(cfg, world: int) -> dict:
    """The bench line's config for the ground workload."""
    return {"workload": f"ground: {cfg.n_det} det x {cfg.n_int} int x {cfg.n_samp} "
                        f"samples, {cfg.side}x{cfg.side} IQU patch, lambda {cfg.lam}",
            "n_samples": cfg.n_total, "lambda": cfg.lam, "tol": cfg.tol,
            "step": "mm_solve_tod: the map from the TOD by mixed-precision PCG (FP32 operators in "
                    "the iterations and for the right-hand side; FP64 CG vectors, dots and scalars; "
                    "every true residual P^T N^-1 G (d - P x) with the double-float operators)",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (window slot 2 B + angle 4 B per sample read twice, "
                  "t and N^-1 t 4 B each written and read: 28 B/sample, 30 GB per A-application)"}


def aggregate(elapsed: float, samples: float, dist_mod=None, device="cpu"):
    """Whole-job timing across ranks: the slowest rank's elapsed time and the samples all ranks
    processed (replicas may run different iteration counts)."""
    if dist_mod is None or not dist_mod.is_initialized() or dist_mod.get_world_size() == 1:
        return elapsed, samples
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    n = torch.tensor([samples], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    dist_mod.all_reduce(n, op=dist_mod.ReduceOp.SUM)
    return float(t), float(n)


# ------------------------------------------------------------------------------------------
# the reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------------

def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    v, cores, desc, per_iter = cpu_oracle_rate(a.cpu_dets, n_iter=a.warmup + a.steps, skip=a.warmup)
    cfg_full = synth.ground_config()
    cfg = ground_config_json(cfg_full, 1)
    cfg["sample_of_workload"] = (f"each step: {cores} x {a.cpu_dets} detectors x 1 interval x "
                                 f"{cfg_full.n_samp} samples of it, one PCG iteration per oracle instance")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": cores * a.cpu_dets * cfg_full.n_samp / v * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg, "per_step_values": per_iter,
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def _safe(name, fn):
    """Run one secondary measurement; a failure is reported in the line instead of ending the run."""
    try:
        t0 = time.perf_counter()
        out = fn()
        log(f"secondary {name}: {time.perf_counter() - t0:.1f}s")
        return out
    except Exception as e:   # reported, not hidden: the key carries the error
        log(f"secondary {name} failed: {e!r}")
        return {"error": repr(e)[:300]}


def oracle_cut_map_error(mm, dev, n_det: int, n_samp: int, tol: float):
    """Map error of the mixed-precision GPU solve against the FP64 oracle's PCG at the same tol,
    on a cut of the ground workload the oracle finishes in seconds: the first n_det detectors, the
    first two intervals (one sweeping in x, one in y) of n_samp samples each."""
    import numpy as np
    import torch
    import oracle as O
    import synth
    cfg = synth.ground_config(n_det=n_det, n_int=2, n_samp=n_samp)
    prob = synth.make_ground_problem(cfg, device=dev)
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    mm.mm_rhs(plan, prob.d, b)
    x = torch.empty_like(b)
    inf = mm.mm_pcg_solve(plan, b, x, tol=tol, max_iter=5000, precision=mm.MM_FP32, raise_on_error=False)[0]
    nb = synth.to_numpy(prob)
    t0 = time.perf_counter()
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], nb["band"], nb["n_pix"])
    ref = O.pcg(op, O.rhs(op, nb["d"]), tol=tol, max_iter=5000)
    t_or = time.perf_counter() - t0
    xg = x.cpu().numpy()
    return {"map_err": float(np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)),
            "cut": f"ground: first {n_det} det x 2 intervals (x and y sweeps) x {n_samp} samples, "
                   f"{cfg.side}^2 patch, lambda {cfg.lam}",
            "n_samples": int(nb["pix"].size), "n_obs": int(op.n_obs), "tol": tol,
            "gpu_iters": inf.iters, "gpu_status": inf.status, "oracle_iters": int(ref.iters),
            "oracle_s": t_or, "metric": "||m_gpu - m_oracle|| / ||m_oracle|| over kept IQU, both at tol"}


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_2112_03370_gb300.mm as mm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    n_sm = props.multi_processor_count

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # replicas: each rank solves its own problem (independent seeds per rank)
    cfg = synth.ground_config(n_det=a.dets, n_samp=a.samples)
    t_gen = time.perf_counter()
    prob = synth.make_ground_problem(cfg, device=dev, real_offset=1000 * rank)
    torch.cuda.synchronize()
    log(f"[rank {rank}] generated {prob.n_total:.3e} samples in {time.perf_counter() - t_gen:.1f}s")
    band_d = prob.band.to(dev)
    t_plan = time.perf_counter()
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix,
                      prob.psi, prob.lam, band_d, precision=mm.MM_FP32_DF64)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    N = plan.n_samples
    log(f"[rank {rank}] plan: n_obs={plan.n_obs} N={N} bytes={plan.bytes / 1e9:.2f} GB "
        f"in {t_plan:.2f}s")
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)

    def step(profile=False):
        # the map from the TOD: FP32 right-hand side, mixed-precision PCG, every true residual
        # P^T N^-1 G (d - P x) in double-float (one FP64-class pass per solve)
        return mm.mm_solve_tod(plan, prob.d, x, tol=cfg.tol, max_iter=5000, precision=mm.MM_FP32,
                               profile=profile, raise_on_error=False)[0]

    for i in range(a.warmup):
        inf = step()
        log(f"[rank {rank}] warmup {i}: iters={inf.iters} status={inf.status} "
            f"true_rel_res={inf.true_rel_res:.2e} t={inf.t_ms:.0f}ms")
    barrier()
    clocks = ClockSampler(bus).start() if rank == 0 else None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    step_ms = []
    ev0.record()
    for i in range(a.steps):
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record()
        infos.append(step())
        e_b.record()
        e_b.synchronize()
        step_ms.append(e_a.elapsed_time(e_b))
    ev1.record()
    barrier()
    clk = clocks.stop() if clocks else None
    elapsed = ev0.elapsed_time(ev1) / 1e3
    applies = sum(i.n_apply32 + i.n_apply64 for i in infos)
    iters = sum(i.iters for i in infos)
    elapsed, samples = aggregate(elapsed, float(N * applies), dist if world > 1 else None, dev)
    _, iters_all = aggregate(elapsed, float(iters), dist if world > 1 else None, dev)
    value = samples / elapsed
    launches = sum(i.n_kernels for i in infos) + 2 * a.steps   # + rhs split and tile per step
    x_mixed = x.clone()

    # kernel split of the FP32 A-application from one profiled solve after the timed region:
    # P over the pixel windows, the FP32 N^-1 tiles (overlap-save FFT, the dominant kernel,
    # FP32-ALU bound at lambda = 8192), P^T over the windows
    pinf = step(profile=True)
    n32 = max(pinf.n_apply32, 1)
    t_up = pinf.t_unpoint32_ms / n32 / 1e3
    t_pt = pinf.t_point32_ms / n32 / 1e3
    t_tile = (pinf.t_apply32_ms - pinf.t_unpoint32_ms - pinf.t_point32_ms) / n32 / 1e3
    t_apply = pinf.t_apply32_ms / n32 / 1e3
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    fp32_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12      # TFLOP/s
    L = 32768
    flops_launch = N * fft_flops_per_sample(L, cfg.lam)
    achieved = flops_launch / t_tile / 1e12
    n_obs = plan.n_obs
    tile_bytes = 8.0 * N                      # t in, N^-1 t out (float32)
    win_bytes = 10.0 * N                      # slot (2) + angle (4) + t or N^-1 t (4)
    apply_alg_bytes = 8.0 * N + 6.0 * n_obs * 4   # the fused floor of the A-application (8 B/sample)
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": measured_traffic(N),
            "kernel": "k_tile<float,1,MODE_NINV_T> (overlap-save FFT N^-1, L = 32768: "
                      f"{fft_flops_per_sample(L, cfg.lam):.0f} flops per output sample)",
            "peak_kind": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                         f"{sm_max:.0f} MHz ({pk_kind} sm_max_mhz)",
            "ms_per_launch": t_tile * 1e3,
            "hbm_achieved_gbs": tile_bytes / t_tile / 1e9,
            "hbm_frac": tile_bytes / t_tile / 1e9 / hbm_peak,
            "hbm_peak_kind": pk_kind,
            "unpoint_kernel": {"name": "k_unpoint_win32 (t = P x over pixel windows)",
                               "ms_per_launch": t_up * 1e3, "achieved_gbs": win_bytes / t_up / 1e9,
                               "hbm_frac": win_bytes / t_up / 1e9 / hbm_peak, "bound": "hbm"},
            "point_kernel": {"name": "k_point_win32 (y += P^T u over pixel windows)",
                             "ms_per_launch": t_pt * 1e3, "achieved_gbs": win_bytes / t_pt / 1e9,
                             "hbm_frac": win_bytes / t_pt / 1e9 / hbm_peak, "bound": "hbm"},
            "a_apply_ms": t_apply * 1e3,
            "a_apply_hbm_frac_fused_floor": apply_alg_bytes / t_apply / 1e9 / hbm_peak,
            "a_apply_alu_frac": flops_launch / t_apply / 1e12 / fp32_peak}

    out = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": elapsed / a.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64",
           "data": "synthetic (seeded, generated on the device)",
           "config": ground_config_json(cfg, world), "n_obs": n_obs,
           "solves_per_s": a.steps * world / elapsed,
           "pcg_iters_per_s": iters_all / elapsed,
           "iters_per_solve": iters / a.steps,
           "a_applies_per_solve": applies / a.steps,
           "true_rel_res": max(i.true_rel_res for i in infos),
           "status": [i.status for i in infos],
           "step_ms_p50": float(np.percentile(step_ms, 50)),
           "step_ms_p99": float(np.percentile(step_ms, 99)),
           "timing_mode": "production: iteration groups replayed as CUDA graphs; the kernel split "
                          "comes from one profiled solve after the timed region",
           "df64_apply_ms": (pinf.t_apply64_ms / pinf.n_apply64) if pinf.n_apply64 else None,
           "plan_s": t_plan,
           "roofline": roof, "gpu_launches": int(launches), "clocks": clk}

    if rank == 0:
        # the FP64-class solve of the same problem: the double-float right-hand side, then plain
        # PCG with the double-float operator in every iteration, to the same tolerance; the mixed
        # map's error against it
        mm.mm_rhs(plan, prob.d, b)
        x64 = torch.empty_like(b)
        mm.mm_pcg_solve(plan, b, x64, tol=cfg.tol, max_iter=5000, precision=mm.MM_FP64, raise_on_error=False)
        inf64, t64 = _timed(lambda: mm.mm_pcg_solve(plan, b, x64, tol=cfg.tol, max_iter=5000,
                                                    precision=mm.MM_FP64, raise_on_error=False)[0])
        out["df64_pcg"] = {"iters": inf64.iters, "status": inf64.status, "s": t64,
                           "solves_per_s": 1.0 / t64, "ms_per_iter": t64 * 1e3 / max(inf64.iters, 1),
                           "true_rel_res": inf64.true_rel_res,
                           "samples_per_s_through_A": N * (inf64.n_apply64 + inf64.n_apply32) / t64,
                           "arithmetic": "double-float (FP64-class) operators in every iteration, "
                                         "FP64 vectors and scalars"}
        out["map_err_vs_fp64class"] = float(torch.linalg.norm(x_mixed - x64) / torch.linalg.norm(x64))
        out["map_err_vs_fp64class_note"] = ("||m_mixed - m_df64|| / ||m_df64|| over kept IQU, both "
                                            f"certified to tol {cfg.tol} on the same TOD; stated bound 1e-5")
        out["speedup_vs_df64_pcg"] = out["solves_per_s"] / out["df64_pcg"]["solves_per_s"]

    # end to end through the public API from pinned host buffers: plan, TOD handed over in host
    # memory (the library copies it), rhs, solve, map back
    if not a.no_e2e:
        pix_h = prob.pix.cpu().pin_memory()
        psi_h = prob.psi.cpu().pin_memory()
        band_h = prob.band.cpu().contiguous()
        d_h = prob.d.cpu().pin_memory()
        h2d = pix_h.numel() * 4 + psi_h.numel() * 4 + band_h.numel() * 8 + d_h.numel() * 8

        def e2e_step():
            tm = [time.perf_counter()]
            p2 = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, pix_h,
                            psi_h, prob.lam, band_h, precision=mm.MM_FP32_DF64)
            tm.append(time.perf_counter())
            x2 = torch.empty(p2.n_obs, 3, dtype=torch.float64, device=dev)
            inf = mm.mm_solve_tod(p2, d_h, x2, tol=cfg.tol, max_iter=5000, precision=mm.MM_FP32,
                                  raise_on_error=False)[0]
            tm.append(time.perf_counter())
            m_host = x2.cpu()
            p2.destroy()
            tm.append(time.perf_counter())
            return inf, m_host, [tm[i + 1] - tm[i] for i in range(3)]

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        e_app = 0
        parts = [0.0, 0.0, 0.0]
        for _ in range(a.e2e_steps):
            inf, m_host, tp = e2e_step()
            e_app += inf.n_apply32 + inf.n_apply64
            parts = [p + q for p, q in zip(parts, tp)]
        barrier()
        te = time.perf_counter() - t0
        te, e_samples = aggregate(te, float(N * e_app), dist if world > 1 else None, dev)
        out["e2e"] = {"value": e_samples / te, "unit": "samples/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(m_host.numel() * 8),
                      "steps": a.e2e_steps, "ms_per_step": te / a.e2e_steps * 1e3,
                      "includes": "mm_plan from pinned host pix/psi/band, mm_solve_tod from the pinned "
                                  "host TOD (copied by the library), D2H of the map, plan destroy",
                      "ms_plan": parts[0] / a.e2e_steps * 1e3, "ms_solve_incl_h2d_of_d": parts[1] / a.e2e_steps * 1e3,
                      "ms_d2h_and_destroy": parts[2] / a.e2e_steps * 1e3}
    del prob

    if rank == 0 and world == 1 and not a.no_cpu:
        out["map_err_vs_oracle_cut"] = _safe("oracle cut", lambda: oracle_cut_map_error(
            mm, dev, a.cut_dets, a.cut_samp, cfg.tol))
        r, cores, desc, _ = cpu_oracle_rate(a.cpu_dets, n_iter=3, skip=1)
        out["cpu_baseline"] = {"value": r, "unit": "samples/s", "cores": cores, "kind": "oracle",
                               "sample": desc}
    if rank == 0 and world == 1 and not a.no_secondary:
        del plan
        torch.cuda.empty_cache()
        sec = {}
        sec["tiny"] = _safe("tiny", lambda: run_tiny(a))
        sec["satellite"] = _safe("satellite", lambda: run_satellite(a))
        sec["batched"] = _safe("batched", lambda: run_batched(a, widths=(64,), nrhs=64))
        sec["serving"] = _safe("serving", lambda: run_serving(a, n_requests=a.requests, compare_fp64=40))
        out["secondary"] = sec
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# other workloads (each returns a dict; run alone with --workload it is printed as one line)
# ------------------------------------------------------------------------------------------

def run_tiny(a):
    """Config 0: 4 det x 65,536 samples, 128^2 patch, lambda 1024, plain FP64 PCG to 1e-8 (IEEE
    FP64 operators), latency-bound: iterations/s, solve latency, and the map error against the
    FP64 oracle's PCG at the same tolerance."""
    import numpy as np
    import torch
    import oracle as O
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg, device=dev)
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP64)
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    mm.mm_rhs(plan, prob.d, b)
    mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP64)
    lat = []
    inf = None
    for _ in range(5):
        inf, dt = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP64)[0])
        lat.append(dt)
    nb = synth.to_numpy(prob)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], nb["band"], nb["n_pix"])
    t0 = time.perf_counter()
    ref = O.pcg(op, O.rhs(op, nb["d"]), tol=cfg.tol, max_iter=5000)
    t_or = time.perf_counter() - t0
    err = float(np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x))
    med = statistics.median(lat)
    return {"workload": "tiny: 4 det x 65536 samples, 128^2 IQU, lambda 1024, tol 1e-8, plain FP64 PCG",
            "iters": inf.iters, "oracle_iters": int(ref.iters), "solve_ms_p50": med * 1e3,
            "pcg_iters_per_s": inf.iters / med, "solves_per_s": 1.0 / med, "status": inf.status,
            "true_rel_res": inf.true_rel_res, "map_err_vs_oracle": err,
            "cpu_baseline": {"value": 1.0 / t_or, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": "the whole tiny solve"}}


def run_batched(a, widths=None, nrhs=None):
    """Ground geometry cut to 128 dets x 1 interval x 524,288 samples, nrhs noise realisations:
    block CG (widths given) vs independent FP64-class (double-float) PCG and independent mixed
    FP32 PCG (rates from two right-hand sides)."""
    import torch
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    nrhs = nrhs or a.nrhs
    widths = widths or [int(v) for v in a.widths.split(",")]
    cfg = synth.batched_config()
    prob = synth.make_ground_problem(cfg, device=dev, n_real=nrhs)
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    N = plan.n_samples
    B = torch.empty(nrhs, plan.n_obs, 3, dtype=torch.float64, device=dev)
    mm.mm_rhs(plan, prob.d, B)
    del prob
    X = torch.empty_like(B)
    res = {}
    for w in widths:
        mm.mm_block_cg_solve(plan, B[:w].contiguous(), X[:w].contiguous(), block_width=w, tol=cfg.tol,
                             max_iter=3, raise_on_error=False)   # warm-up: buffers and kernels
        infos, dt = _timed(lambda: mm.mm_block_cg_solve(plan, B, X, block_width=w, tol=cfg.tol,
                                                        raise_on_error=False))
        # the block A X of w columns alone (FP32 operator; FP64 in and out as the solver sees it)
        Xw, Yw = B[:w].contiguous(), torch.empty_like(B[:w])
        mm.mm_apply_A(plan, Xw, Yw)
        _, dta = _timed(lambda: [mm.mm_apply_A(plan, Xw, Yw) for _ in range(3)])
        dta /= 3
        n_blk_it = infos[0].n_apply32
        res[str(w)] = {"solves_per_s": nrhs / dt, "s": dt,
                       "iters_max": max(i.iters for i in infos),
                       "true_rel_res_max": max(i.true_rel_res for i in infos),
                       "status": sorted(set(i.status for i in infos)),
                       "block_applies_first_group": n_blk_it,
                       "block_ax_ms": dta * 1e3,
                       "block_ax_samples_per_s_per_column": w * N / dta,
                       "block_ax_share_of_iteration": (dta * n_blk_it * (nrhs // w)) / dt}
        del Xw, Yw
    x1 = torch.empty(2, plan.n_obs, 3, dtype=torch.float64, device=dev)
    infos, dt64 = _timed(lambda: mm.mm_pcg_solve(plan, B[:2].contiguous(), x1, tol=cfg.tol,
                                                 precision=mm.MM_FP64, raise_on_error=False))
    infos32, dt32 = _timed(lambda: mm.mm_pcg_solve(plan, B[:2].contiguous(), x1, tol=cfg.tol,
                                                   precision=mm.MM_FP32, raise_on_error=False))
    best_w, best = max(res.items(), key=lambda kv: kv[1]["solves_per_s"])
    return {"workload": f"batched: ground cut {plan.n_samples // cfg.n_samp} det x {cfg.n_samp} samples, "
                        f"{cfg.side}^2 IQU, lambda {cfg.lam}, {nrhs} noise realisations, tol {cfg.tol}",
            "metric": "solves/s", "value": best["solves_per_s"], "best_width": int(best_w),
            "n_samples": N, "n_obs": plan.n_obs, "block_cg": res,
            "df64_pcg": {"solves_per_s": 2 / dt64, "iters": [i.iters for i in infos]},
            "fp32_pcg_independent": {"solves_per_s": 2 / dt32, "iters": [i.iters for i in infos32]},
            "vs_df64_pcg": best["solves_per_s"] / (2 / dt64),
            "vs_fp32_pcg": best["solves_per_s"] / (2 / dt32)}


def run_ecg(a):
    """Enlarged CG (Orthomin and Orthodir) for one right-hand side of the 128-detector ground cut,
    against the mixed-precision PCG on the same plan: iterations, A column-applications and
    time to solution per enlarging factor t."""
    import torch
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    cfg = synth.batched_config()
    prob = synth.make_ground_problem(cfg, device=dev, n_real=1)
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    N = plan.n_samples
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    mm.mm_rhs(plan, prob.d, b)
    x = torch.empty_like(b)
    mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32)
    ipcg, tpcg = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32)[0])
    res = {}
    for variant, vname in ((mm.MM_ECG_ORTHOMIN, "orthomin"), (mm.MM_ECG_ORTHODIR, "orthodir")):
        for t in [int(v) for v in a.enlarge.split(",")]:
            mm.mm_ecg_solve(plan, b, x, t, variant=variant, tol=cfg.tol, raise_on_error=False)
            inf, dt = _timed(lambda: mm.mm_ecg_solve(plan, b, x, t, variant=variant, tol=cfg.tol,
                                                     raise_on_error=False))
            res[f"{vname}_t{t}"] = {"iters": inf.iters, "status": inf.status, "s": dt,
                                    "true_rel_res": inf.true_rel_res, "restarts": inf.n_true_res - 1,
                                    "column_applies": inf.iters * t,
                                    "samples_per_s_through_A": N * t * inf.iters / dt,
                                    "s_per_iter": dt / max(inf.iters, 1),
                                    "vs_pcg_time": tpcg / dt}
    return {
        "workload": "ecg", "metric": "time to solution, one right-hand side (ECG vs PCG)",
        "value": min(r["s"] for r in res.values()), "unit": "s", "higher_is_better": False,
        "config": {"workload": f"ground cut: {prob.n_det} det x {cfg.n_samp} samples, "
                               f"{cfg.side}^2 IQU, lambda {cfg.lam}, one realisation",
                   "n_samples": N, "n_obs": plan.n_obs, "tol": cfg.tol,
                   "precision": "FP32 search blocks and operator, FP64 X/R and t x t, df64 true residual"},
        "pcg": {"iters": ipcg.iters, "s": tpcg, "s_per_iter": tpcg / max(ipcg.iters, 1),
                "samples_per_s_through_A": N * ipcg.iters / tpcg},
        "ecg": res,
        "orthomin_t1_s_per_iter_vs_pcg": (res["orthomin_t1"]["s_per_iter"] / (tpcg / max(ipcg.iters, 1))
                                          if "orthomin_t1" in res else None)}


def run_noise(a):
    """Noise weights estimated from the data of the ground workload (2048 blocks of 524,288
    samples): periodogram, PSD fit and inverse band on the GPU, against the true PSD parameters of
    the generator, with the oracle's estimate on one block as the CPU baseline.  The TOD is the
    noise alone, the estimator's stated assumption (Sect. 2.2); with the sky signal in, its power
    adds to the fitted white level."""
    import numpy as np
    import torch
    import oracle as O
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    cfg = synth.ground_config(n_det=a.dets)
    prob = synth.make_ground_problem(cfg, device=dev, with_signal=False)
    bl = prob.block_len.tolist()
    mm.mm_estimate_bands(prob.n_det, prob.n_int, bl, prob.pix, prob.d, cfg.lam)
    (bands, par), t = _timed(lambda: mm.mm_estimate_bands(prob.n_det, prob.n_int, bl, prob.pix, prob.d, cfg.lam))
    sig = prob.sigmas.cpu().numpy() if prob.sigmas is not None else None
    fk_true = cfg.f_knee / cfg.fs
    err = {"log_f_knee_median_abs": float(np.median(np.abs(par[:, 1] - math.log(fk_true)))),
           "alpha_median_abs": float(np.median(np.abs(par[:, 2] - cfg.alpha)))}
    if sig is not None:
        per_blk = np.repeat(sig, prob.n_int) if sig.size == prob.n_det else sig
        err["sigma2_median_rel"] = float(np.median(np.abs(np.exp(par[:, 0]) / per_blk ** 2 - 1)))
    n0 = int(bl[0])
    t0 = time.perf_counter()
    O.estimate_bands(prob.d[:n0].cpu().numpy(), prob.pix[:n0].cpu().numpy(), [n0], cfg.lam)
    t_cpu = time.perf_counter() - t0
    pk, pk_kind = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    nbytes = 12.0 * prob.n_total   # the periodogram reads the pixel index (4 B) and d (8 B) once
    return {
        "workload": "noise", "metric": "TOD samples/s through the noise-weight estimation",
        "value": prob.n_total / t, "unit": "samples/s", "higher_is_better": True,
        "config": {"workload": f"ground: {prob.n_det} det x {prob.n_int} int x {cfg.n_samp} samples, "
                               f"lambda {cfg.lam}, 32768-sample segments, noise-only TOD",
                   "blocks": len(bl), "n_samples": prob.n_total},
        "s": t, "vs_true_parameters": err,
        "roofline": {"bound": "hbm", "achieved": nbytes / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": nbytes / t / 1e9 / hbm_peak, "traffic": None,
                     "kernel": "k_periodogram + k_psd_fit + k_band_from_fit (whole estimation; the "
                               "periodogram reads 12 B/sample)", "peak_kind": pk_kind},
        "cpu_baseline": {"value": n0 / t_cpu, "unit": "samples/s", "cores": 1, "kind": "oracle",
                         "sample": f"one block of {n0} samples, numpy/scipy"}}


def run_templates(a):
    """Template map-making with diagonal weights (lambda = 0) on the ground geometry (512 det x 4
    intervals x 524,288 samples): Legendre trends (3 orders), 30 azimuth bins and 6 HWP harmonics per
    block, the template classes of the validation in Sect. 4 with one interval per block; ground
    pickup and an HWP-synchronous signal are injected on top of sky + 1/f noise.  Times the setup
    (bins, T^T W T, pseudo-inverse), the RHS and a mixed-precision solve; the oracle's template
    operator on one block is the CPU baseline."""
    import numpy as np
    import torch
    import oracle as O
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    cfg = synth.ground_config(n_det=a.dets, lam=0)
    prob = synth.make_ground_problem(cfg, device=dev)
    az, hwp = synth.ground_template_streams(cfg, device=dev)
    prob.d += synth.template_systematics(cfg, az, hwp, seed=synth.seed_for(cfg.config_id, 11))
    torch.cuda.synchronize()
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    N = plan.n_samples
    tm = dict(n_poly=3, n_az=30, n_hwp=6)
    mm.mm_templates_set(plan, **tm, az=az, hwp=hwp)
    _, t_setup = _timed(lambda: mm.mm_templates_set(plan, **tm, az=az, hwp=hwp))
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    mm.mm_rhs(plan, prob.d, b)
    _, t_rhs = _timed(lambda: mm.mm_rhs(plan, prob.d, b))
    x = torch.empty_like(b)
    tol = cfg.tol
    mm.mm_pcg_solve(plan, b, x, tol=tol, precision=mm.MM_FP32, raise_on_error=False)
    infos, t_solve = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=tol, precision=mm.MM_FP32,
                                                    raise_on_error=False))
    inf = infos[0]
    pinf = mm.mm_pcg_solve(plan, b, x, tol=tol, precision=mm.MM_FP32, profile=True, raise_on_error=False)[0]
    ms32 = pinf.t_apply32_ms / max(1, pinf.n_apply32)
    ms64 = pinf.t_apply64_ms / max(1, pinf.n_apply64)
    # template removal at full size: the same sky and injected systematics without noise, solved with
    # the templates and with a plain binned plan (no templates); Q, U against the input sky (I carries
    # an offset degenerate with the constant templates)
    ms = prob.m_sky.to(dev)[plan.obs_to_global.long()]
    seed_sys = synth.seed_for(cfg.config_id, 11)
    prob.d = None
    dc = synth.make_ground_problem(cfg, device=dev, with_noise=False).d
    dc += synth.template_systematics(cfg, az, hwp, seed=seed_sys)

    def qu_err(xm):
        return float(torch.sqrt(((xm[:, 1:] - ms[:, 1:]) ** 2).mean()) / torch.sqrt((ms[:, 1:] ** 2).mean()))
    mm.mm_rhs(plan, dc, b)
    ic = mm.mm_pcg_solve(plan, b, x, tol=1e-8, precision=mm.MM_FP32, raise_on_error=False)[0]
    err_t = qu_err(x)
    plan0 = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                       prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    mm.mm_rhs(plan0, dc, b)
    mm.mm_pcg_solve(plan0, b, x, tol=1e-8, precision=mm.MM_FP32, raise_on_error=False)
    err_b = qu_err(x)
    del plan0, dc
    # CPU baseline: the oracle's template operator on one block
    n0 = int(prob.block_len[0])
    nb0 = {"pix": prob.pix[:n0].cpu().numpy(), "psi": prob.psi[:n0].cpu().numpy()}
    op0 = O.make_plan(nb0["pix"], nb0["psi"], [n0], prob.band[:1].numpy(), prob.n_pix)
    tmo = O.Templates(**tm)
    x0 = np.random.default_rng(0).standard_normal((op0.n_obs, 3))
    t0 = time.perf_counter()
    O.apply_A_templates(op0, prob.band[:1, 0].numpy(), tmo, az[:n0].cpu().numpy(), hwp[:n0].cpu().numpy(), x0)
    t_cpu = time.perf_counter() - t0
    # algorithmic DRAM bytes per sample of the fused FP32 operator: two passes over lpix (4), the
    # pointing weights (8), cos/sin of the HWP angle (8) and the azimuth bin (1); the map gathers and
    # the per-pixel M x stay in L2
    tmpl_b = 2 * (4 + 8 + 8 + 1)
    pk, pk_kind = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    return {
        "workload": "templates", "metric": "TOD samples/s per PCG iteration, template map-making",
        "value": N * inf.iters / t_solve, "unit": "samples/s", "higher_is_better": True,
        "config": {"workload": f"ground: {prob.n_det} det x {prob.n_int} int x {cfg.n_samp} samples, "
                               f"{cfg.side}^2 IQU, lambda 0 (diagonal weights), templates "
                               f"n_poly {tm['n_poly']}, n_az {tm['n_az']}, n_hwp {tm['n_hwp']} "
                               f"(K = {tmo.k} per block), ground pickup + HWPSS injected",
                   "n_samples": N, "n_obs": plan.n_obs, "blocks": prob.n_det * prob.n_int, "tol": tol},
        "setup_s": t_setup, "rhs_s": t_rhs, "solve_s": t_solve, "iters": inf.iters, "status": inf.status,
        "true_rel_res": inf.true_rel_res,
        "noiseless_check": {"qu_rel_err_templates": err_t, "qu_rel_err_binned": err_b, "iters": ic.iters,
                            "status": ic.status, "tol": 1e-8,
                            "data": "sky + ground pickup + HWPSS, no noise"},
        "fp32_apply_ms": ms32, "fp64_class_apply_ms": ms64,
        "roofline": {"bound": "hbm", "achieved": N * tmpl_b / (ms32 * 1e-3) / 1e9, "peak": hbm_peak,
                     "unit": "GB/s", "frac": N * tmpl_b / (ms32 * 1e-3) / 1e9 / hbm_peak, "traffic": None,
                     "kernel": "k_tmpl_apply32 (42 B/sample over two passes) + k_tmpl_mx32",
                     "peak_kind": pk_kind},
        "cpu_baseline": {"value": n0 / t_cpu, "unit": "samples/s through the template operator",
                         "cores": 1, "kind": "oracle",
                         "sample": f"one block of {n0} samples, numpy (dense T)"}}


def run_satellite(a):
    """Satellite-like full sky: BD vs two-level (16 Ritz vectors) mixed-precision solves."""
    import torch
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    cfg = synth.satellite_config(n_det=a.dets if a.dets != 512 else 64)
    prob, tg = _timed(lambda: synth.make_satellite_problem(cfg, device=dev))
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    N = plan.n_samples
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    mm.mm_rhs(plan, prob.d, b)
    del prob
    x = torch.empty_like(b)
    mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32, raise_on_error=False)
    i_bd, t_bd = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32,
                                               raise_on_error=False)[0])
    _, t_build = _timed(lambda: mm.mm_deflation_build(plan, b, 16, precision=mm.MM_FP32))
    i_2l, t_2l = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32,
                                               precond=mm.MM_PREC_2LVL_POST, raise_on_error=False)[0])
    return {
        "workload": f"satellite: {cfg.n_det} det x {cfg.n_samp} samples at 20 Hz, "
                    f"{cfg.n_rings}x{cfg.n_phi} equal-area pixels, lambda {cfg.lam}, tol {cfg.tol}",
        "metric": "PCG solves/s (BD vs 2lvl a posteriori, 16 Ritz vectors)",
        "value": 1.0 / t_2l, "unit": "solves/s", "n_samples": N, "n_obs": plan.n_obs, "gen_s": tg,
        "bd": {"iters": i_bd.iters, "s": t_bd, "solves_per_s": 1.0 / t_bd, "status": i_bd.status,
               "true_rel_res": i_bd.true_rel_res,
               "samples_per_s_through_A": N * (i_bd.n_apply32 + i_bd.n_apply64) / t_bd},
        "two_level": {"iters": i_2l.iters, "s": t_2l, "solves_per_s": 1.0 / t_2l, "build_s": t_build,
                      "status": i_2l.status, "true_rel_res": i_2l.true_rel_res},
        "two_level_apriori": _apriori(mm, plan, b, x, cfg.tol),
        "speedup_per_solve": t_bd / t_2l,
        "solves_to_amortise_build": t_build / max(t_bd - t_2l, 1e-9)}


def _apriori(mm, plan, b, x, tol):
    """Mixed-precision PCG with the a-priori two-level space (one column per interval)."""
    _, t_build = _timed(lambda: mm.mm_deflation_build_apriori(plan, precision=mm.MM_FP32))
    mm.mm_pcg_solve(plan, b, x, tol=tol, precision=mm.MM_FP32, precond=mm.MM_PREC_2LVL_POST,
                    raise_on_error=False)
    inf, t = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=tol, precision=mm.MM_FP32,
                                            precond=mm.MM_PREC_2LVL_POST, raise_on_error=False)[0])
    return {"columns": mm.mm_deflation_get(plan)[0], "iters": inf.iters, "s": t, "build_s": t_build,
            "status": inf.status, "true_rel_res": inf.true_rel_res}


def run_deflation(a):
    """Ground workload (4 stationary intervals): block-Jacobi PCG against the two-level
    preconditioner with the a-priori space (4 columns) and the a-posteriori one (16 Ritz vectors),
    all mixed precision, same right-hand side."""
    import torch
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    cfg = synth.ground_config(n_det=a.dets)
    prob = synth.make_ground_problem(cfg, device=dev)
    plan = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                      prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64)
    b = torch.empty(plan.n_obs, 3, dtype=torch.float64, device=dev)
    mm.mm_rhs(plan, prob.d, b)
    x = torch.empty_like(b)
    mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32, raise_on_error=False)
    i_bd, t_bd = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32,
                                               raise_on_error=False)[0])
    apri = _apriori(mm, plan, b, x, cfg.tol)
    _, t_build = _timed(lambda: mm.mm_deflation_build(plan, b, 16, precision=mm.MM_FP32))
    i_2l, t_2l = _timed(lambda: mm.mm_pcg_solve(plan, b, x, tol=cfg.tol, precision=mm.MM_FP32,
                                               precond=mm.MM_PREC_2LVL_POST, raise_on_error=False)[0])
    return {
        "workload": "deflation", "metric": "PCG time to solution (BD, 2lvl a priori, 2lvl a posteriori)",
        "value": min(t_bd, apri["s"], t_2l), "unit": "s", "higher_is_better": False,
        "config": {"workload": f"ground: {prob.n_det} det x {prob.n_int} int x {cfg.n_samp} samples, "
                               f"{cfg.side}^2 IQU, lambda {cfg.lam}",
                   "n_samples": plan.n_samples, "n_obs": plan.n_obs, "tol": cfg.tol},
        "bd": {"iters": i_bd.iters, "s": t_bd, "status": i_bd.status, "true_rel_res": i_bd.true_rel_res},
        "two_level_apriori": apri,
        "two_level_aposteriori": {"columns": 16, "iters": i_2l.iters, "s": t_2l, "build_s": t_build,
                                  "status": i_2l.status, "true_rel_res": i_2l.true_rel_res}}


def _serve(mm, pool, order, gaps, fp64: bool):
    """Submit pool[order[i]] at the arrival times t0 + gaps[0] + ... + gaps[i] (Poisson arrivals,
    on an absolute schedule, so the time a submission takes does not thin the stream); returns
    per-request latencies (ms, submit to completion), infos, the wall time from the first
    arrival and the host time of the submissions (ms: mean, max)."""
    srv = mm.Server(max_slots=16)
    kw = dict(precision=mm.MM_FP64, plan_precision=mm.MM_DF64) if fp64 else {}
    p = pool[0]
    srv.wait(srv.submit(p["n_det"], p["n_int"], p["block_len"].tolist(), p["n_pix"], p["pix"], p["psi"],
                        p["lam"], p["band"], p["d"], tol=1e-6, **kw))   # warm-up
    t0 = time.perf_counter()
    t_arr = t0
    ids, t_sub = [], []
    for k, gap in zip(order, gaps):
        t_arr += gap
        wait = t_arr - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        p = pool[k]
        ts = time.perf_counter()
        ids.append(srv.submit(p["n_det"], p["n_int"], p["block_len"].tolist(), p["n_pix"], p["pix"],
                              p["psi"], p["lam"], p["band"], p["d"], tol=1e-6, **kw))
        t_sub.append(1e3 * (time.perf_counter() - ts))
    infos = [srv.wait(i, raise_on_error=False)[1] for i in ids]
    dt = time.perf_counter() - t0
    srv.close()
    lat = [i.t_queue_ms + i.t_ms for i in infos]
    return lat, infos, dt, (sum(t_sub) / len(t_sub), max(t_sub))


def run_serving(a, n_requests=None, compare_fp64=0):
    """Poisson stream (mean `rate`/s) of map-making solves with seeded random shapes from the
    serving recipe: detectors {8..256}, samples/detector {2^16..2^20}, patch side {64..512},
    lambda {512..8192}; raster + HWP scan and 1/f noise as in the tiny recipe; tol 1e-6.  A pool
    of 24 distinct seeded requests is drawn from the recipe and the stream cycles through it in a
    seeded random order.  With compare_fp64 > 0 the first compare_fp64 requests of the same stream
    are also served as FP64-class requests (double-float operators in every iteration)."""
    import numpy as np
    import torch
    import synth
    import paper_2112_03370_gb300.mm as mm
    n_requests = n_requests or a.requests
    rng = np.random.default_rng(synth.seed_for(4, 0))
    pool = []
    for i in range(24):
        ndet = int(rng.choice([8, 16, 32, 64, 128, 256]))
        nsamp = int(rng.choice([1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20]))
        side = int(rng.choice([64, 128, 256, 512]))
        lam = int(rng.choice([512, 1024, 2048, 4096, 8192]))
        cfg = synth.tiny_config(config_id=400 + i, n_det=ndet, n_samp=nsamp, side=side, lam=lam,
                                speed=0.25 * side / 128, det_layout="grid23", tol=1e-6)
        pool.append(synth.to_numpy(synth.make_ground_problem(cfg, device="cuda")))
        torch.cuda.empty_cache()
    order = rng.integers(0, len(pool), size=n_requests)
    gaps = rng.exponential(1.0 / a.rate, size=n_requests)
    lat, infos, dt, sub = _serve(mm, pool, order, gaps, fp64=False)
    samples = sum(int(pool[k]["pix"].size) for k in order)
    out = {
        "workload": f"serving: {n_requests} requests at mean {a.rate}/s (pool of {len(pool)} seeded shapes: "
                    f"dets 8-256, samples/det 2^16-2^20, side 64-512, lambda 512-8192), tol 1e-6",
        "metric": "solves/s + p50/p99 latency (Poisson arrivals)", "value": n_requests / dt,
        "unit": "solves/s", "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "offered_per_s": a.rate, "offered_realised_per_s": n_requests / float(np.sum(gaps)),
        "total_samples": samples,
        "status": sorted(set(i.status for i in infos)), "max_batch": max(i.batch for i in infos),
        "iters_mean": float(np.mean([i.iters for i in infos])),
        "arrivals": "absolute Poisson schedule", "submit_ms_mean": sub[0], "submit_ms_max": sub[1],
        "mode": "FP32 iterations batched per launch across requests (P, N^-1 and P^T over pixel windows "
                "and segments, three launches per step), double-float rhs and replacement"}
    if compare_fp64:
        k = min(compare_fp64, n_requests)
        lat64, inf64, dt64, _ = _serve(mm, pool, order[:k], gaps[:k], fp64=True)
        lat32 = lat[:k]
        out["fp64_class_requests"] = {
            "requests": k, "solves_per_s": k / dt64, "p50_ms": float(np.percentile(lat64, 50)),
            "p99_ms": float(np.percentile(lat64, 99)), "status": sorted(set(i.status for i in inf64)),
            "mode": "plain PCG with the double-float FP64-class operator in every iteration, one launch "
                    "per request per step",
            "mixed_first_k_p50_ms": float(np.percentile(lat32, 50))}
        out["served_vs_fp64_class_solves_per_s"] = (n_requests / dt) / (k / dt64)
    return out


def run_crossover(a):
    """N^-1 on the tensor cores (MM_TPLZ_GEMM: banded Toeplitz-block GEMMs, tcgen05, 3xTF32)
    against the overlap-save FFT tiles (MM_TPLZ_FFT), per half-bandwidth, on the ground geometry
    cut to --dets detectors: a profiled FP32 PCG of --iters iterations per algorithm, and the
    N^-1 time per A-application from its per-launch events.  MM_TPLZ_AUTO takes the GEMM up to
    the largest lambda it wins here.  Also the two maps after the same iterations (the algorithms
    differ only by FP32 rounding)."""
    import numpy as np
    import torch
    import synth
    import paper_2112_03370_gb300.mm as mm
    dev = torch.device("cuda")
    pk, pk_kind = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    tf32_peak = float(pk.get("bf16_tflops", 1900.0)) * 1.1 / 2.25   # nominal TF32:BF16 dense ratio
    rows = []
    for lam in [int(v) for v in a.lams.split(",")]:
        cfg = synth.ground_config(n_det=a.dets, n_samp=a.samples, lam=lam)
        prob = synth.make_ground_problem(cfg, device=dev, with_noise=False)
        res, maps = {}, {}
        for algo, name in ((mm.MM_TPLZ_FFT, "fft"), (mm.MM_TPLZ_GEMM, "gemm")):
            p = mm.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix, prob.psi,
                           prob.lam, prob.band.to(dev), precision=mm.MM_FP32_DF64, toeplitz_algo=algo)
            b = torch.empty(p.n_obs, 3, dtype=torch.float64, device=dev)
            x = torch.empty_like(b)
            mm.mm_rhs(p, prob.d, b)
            info = mm.mm_pcg_solve(p, b, x, tol=1e-12, max_iter=a.iters, precision=mm.MM_FP32,
                                   profile=True, raise_on_error=False)[0]
            n = max(info.n_apply32, 1)
            res[name] = (info.t_apply32_ms - info.t_unpoint32_ms - info.t_point32_ms) / n
            maps[name] = x.cpu().numpy()
            p.destroy()
        j0 = (lam + 31) // 32
        tc_flops = 2.0 * 32 * (2 * j0 + 1) * 3 * prob.n_total
        rows.append({"lambda": lam, "fft_ms": res["fft"], "gemm_ms": res["gemm"],
                     "gemm_faster": res["gemm"] < res["fft"],
                     "gemm_tensor_tflops": tc_flops / (res["gemm"] * 1e-3) / 1e12,
                     "gemm_tensor_frac": tc_flops / (res["gemm"] * 1e-3) / 1e12 / tf32_peak,
                     "gemm_hbm_frac": 8.0 * prob.n_total / (res["gemm"] * 1e-3) / 1e9 / hbm_peak,
                     "fft_hbm_frac": 8.0 * prob.n_total / (res["fft"] * 1e-3) / 1e9 / hbm_peak,
                     "map_rel_diff": float(np.linalg.norm(maps["gemm"] - maps["fft"]) /
                                           np.linalg.norm(maps["fft"]))})
        log(f"lambda {lam}: N^-1 per apply fft {res['fft']:.3f} ms  gemm {res['gemm']:.3f} ms")
        n_total = prob.n_total
        del prob
        torch.cuda.empty_cache()
    wins = [r["lambda"] for r in rows if r["gemm_faster"]]
    best = min(rows, key=lambda r: r["gemm_ms"] / r["fft_ms"])
    return {
        "workload": "crossover", "metric": "N^-1 time per A-application, tensor cores vs FFT tiles",
        "value": best["fft_ms"] / best["gemm_ms"], "unit": "x (FFT time / GEMM time, best lambda)",
        "higher_is_better": True,
        "config": {"workload": f"ground geometry: {a.dets} det x 4 int x 524288 samples, FP32 operators, "
                               f"{a.iters} PCG iterations per algorithm", "n_samples": n_total},
        "rows": rows, "gemm_wins_up_to_lambda": max(wins) if wins else None,
        "auto_rule": "MM_TPLZ_AUTO takes the GEMM for lambda <= 64 on FP32 operators",
        "roofline": {"bound": "tensor", "kernel": "k_tplz_tc", "lambda": best["lambda"],
                     "achieved": best["gemm_tensor_tflops"], "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": best["gemm_tensor_frac"], "traffic": None,
                     "peak_kind": f"{pk_kind} bf16 x 1.1/2.25 (TF32)"}}


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload == "ground":
        run_ours(a)
        return
    fn = {"batched": run_batched, "satellite": run_satellite, "serving": run_serving, "ecg": run_ecg,
          "deflation": run_deflation, "noise": run_noise, "templates": run_templates, "tiny": run_tiny,
          "crossover": run_crossover}
    print(json.dumps(fn[a.workload](a)), flush=True)


if __name__ == "__main__":
    main()
