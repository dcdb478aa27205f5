"""Benchmark: primal-dual voxel-iterations/s on the 256 x 256 x 64-slice volume.

One step = one complete solve of the hot path on one batch: zero start and
500 fused primal-dual iterations (forward dipole convolution, dual data and
TV proxes, adjoint convolution, primal step, over-relaxation) for all 64
slices of the synthetic 256 x 256 volume (six seeds/needles in smooth tissue,
elliptical mask, lambda = 5e-4), inputs resident in HBM.  The L2 cache is
flushed (a 256 MiB device write) between timed steps; within a step the
iteration's working set stays wherever the hardware keeps it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.

Multi-GPU (torchrun, one rank per GPU): slices are independent, so every rank
solves its own volume with no data-path collective (weak scaling); the
barrier and the max-over-ranks timing reduction are the only collectives.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 256
SLICES = 64
N_ITER = 500
LAM = 5e-4
WORKLOAD = "256x256x64 slices, 500 PD iterations, lambda=5e-4 (seeds/needles phantom, elliptical mask)"
ALG_BYTES_PER_VOXEL_ITER = 37  # read+write chi, p, qx, qy (4 x 8 B) + read dB (4 B) + mask (1 B)
ALG_FLOPS_PER_VOXEL_ITER = 10 * 16 + 30  # 2 real 2-D FFT round trips (10 log2(HW)) + pointwise/stencil
L2_FLUSH_BYTES = 256 << 20
# What ncu shows limiting the fused iteration kernel (profiles/pd_cluster_kernel_256x256x64.txt): the
# slices in flight stay in L2, DRAM is nearly idle, and the row phases wait on L2 and distributed
# shared-memory round trips; the HBM figure below is the useful-bytes roofline of the target.
LIMITER_2D = "latency of L2 and DSMEM round trips (L2-resident working set; DRAM ~3% busy)"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pd_cluster_kernel_256x256x64.txt")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kernel_source_hash():
    """Hash of the iteration kernel's device code (the FFT engine and the fused kernel), ignoring
    // comments and blank lines (a comment edit does not change the kernel the ncu counters were
    taken from); the variant table and launch glue are host code."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2006_09808_gb300", "csrc")
    for name in ("fft_core.cuh", "pd_cluster.cuh"):  # the iteration kernel's device code
        for line in open(os.path.join(csrc, name), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it matches this kernel source."""
    try:
        vals = {}
        for line in open(PROFILE_SUMMARY):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_source_hash") != kernel_source_hash():
            return None
        return float(vals["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(pb, tau, sigma, n_slices, n_iter):
    """FP64 oracle on n_slices of the workload; returns (voxel-iter/s, seconds)."""
    import numpy as np

    from oracle import pd_oracle as O

    f = pb.field[:n_slices].astype(np.float64)
    m = pb.mask[:n_slices]
    t0 = time.perf_counter()
    for s in range(n_slices):  # the paper's CPU method: one slice after another
        O.pd_solve(f[s], m[s], pb.lam, tau, sigma, n_iter)
    dt = time.perf_counter() - t0
    return n_slices * f.shape[-2] * f.shape[-1] * n_iter / dt, dt


def _oracle_slice(args):
    """One oracle slice solve (a worker of the all-cores CPU baseline); returns its seconds."""
    import numpy as np

    from oracle import pd_oracle as O

    f, m, lam, tau, sigma, n_iter = args
    t0 = time.perf_counter()
    O.pd_solve(np.asarray(f, np.float64), m, lam, tau, sigma, n_iter)
    return time.perf_counter() - t0


def host_description():
    """Host CPU model and core count (the CPU baseline's hardware)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        import platform

        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": os.cpu_count()}


def cpu_oracle_all_cores(fields, masks, lam, tau, sigma, n_iter, pool):
    """The oracle over independent slices on every host core (a spawn process pool, one slice per
    task, one numpy thread per process); returns (voxel-iter/s, wall seconds, processes)."""
    tasks = [(fields[k], masks[k], lam, tau, sigma, n_iter) for k in range(len(fields))]
    t0 = time.perf_counter()
    list(pool.imap_unordered(_oracle_slice, tasks))
    dt = time.perf_counter() - t0
    vox = sum(int(f.size) for f in fields)
    return vox * n_iter / dt, dt, pool._processes


def make_oracle_pool():
    """Process pool for the all-cores CPU baseline: spawned (never forked from a process holding a
    CUDA context), one single-threaded numpy per process, created before the first GPU call."""
    import multiprocessing as mp

    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    n = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(n)
    pool.map(_oracle_slice, [(np_zeros8(), np_ones8(), 1.0, 0.3, 0.3, 1)] * n)  # workers imported and warm
    return pool


def np_zeros8():
    import numpy as np

    return np.zeros((8, 8))


def np_ones8():
    import numpy as np

    return np.ones((8, 8), np.uint8)


PAPER_SPEEDUP = "4~15x whole-volume CPU -> GPU (Sec. III; the paper names no CPU or GPU model)"


def cufft_comparison(field, mask, lam, tau, sigma, n_iter, stream, chi_fused):
    """Comparison points on the same volume, in plain PyTorch on the GPU (cuFFT for the transforms):
    (1) the FFT passes alone -- per iteration two forward and two inverse real 2-D FFTs of the
    volume; (2) the whole iteration unfused, one library call per step (the structure of the
    paper's GPU method: transforms by a library, every pointwise step its own kernel).  Not the
    product path; (2)'s chi is checked against the fused kernel's."""
    import torch

    S, H, W = field.shape
    dev = field.device
    ky = torch.fft.fftfreq(H, device=dev, dtype=torch.float64)[:, None]
    kx = torch.fft.rfftfreq(W, device=dev, dtype=torch.float64)[None, :]
    k2 = kx * kx + ky * ky
    D = torch.where(k2 > 0, 1.0 / 3.0 - ky * ky / torch.where(k2 > 0, k2, 1.0), torch.zeros_like(k2)).float()
    x = torch.zeros_like(field)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(2):  # warm the plans
            x = torch.fft.irfft2(D * torch.fft.rfft2(x), s=(H, W))
        e0.record(stream)
        for _ in range(n_iter):
            x = torch.fft.irfft2(D * torch.fft.rfft2(x), s=(H, W))
            x = torch.fft.irfft2(D * torch.fft.rfft2(x), s=(H, W))
        e1.record(stream)
    torch.cuda.synchronize()
    ms_fft = e0.elapsed_time(e1)

    def Dop(a):
        return torch.fft.irfft2(D * torch.fft.rfft2(a), s=(H, W))

    w = mask.float()
    b = w * field
    chi = torch.zeros_like(field)
    cb = torch.zeros_like(field)
    p = torch.zeros_like(field)
    qx = torch.zeros_like(field)
    qy = torch.zeros_like(field)
    inv = 1.0 / (1.0 + sigma / lam)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(n_iter):
            p = (p + sigma * (w * Dop(cb) - b)) * inv
            gx = torch.zeros_like(cb)
            gy = torch.zeros_like(cb)
            gx[:, :, :-1] = cb[:, :, 1:] - cb[:, :, :-1]
            gy[:, :-1, :] = cb[:, 1:, :] - cb[:, :-1, :]
            qx = torch.clamp(qx + sigma * w * gx, -1.0, 1.0)
            qy = torch.clamp(qy + sigma * w * gy, -1.0, 1.0)
            d = torch.zeros_like(cb)
            d[:, :, 1:] += qx[:, :, :-1]
            d[:, :, :-1] -= qx[:, :, :-1]
            d[:, 1:, :] += qy[:, :-1, :]
            d[:, :-1, :] -= qy[:, :-1, :]
            new = chi - tau * Dop(w * p) - tau * d
            cb = 2.0 * new - chi
            chi = new
        e1.record(stream)
    torch.cuda.synchronize()
    ms_unfused = e0.elapsed_time(e1)
    rel = float(torch.linalg.norm((chi - chi_fused).double()) / torch.linalg.norm(chi_fused.double()))
    work = S * H * W * n_iter
    return {
        "cufft_fft_passes_only": {"ms": ms_fft, "voxel_iter_per_s": work / (ms_fft * 1e-3),
                                  "note": "2 rfft2 + 2 irfft2 of the volume per iteration (torch.fft = cuFFT)"},
        "unfused_library_loop": {"ms": ms_unfused, "voxel_iter_per_s": work / (ms_unfused * 1e-3),
                                 "rel_l2_vs_fused_chi": rel,
                                 "note": "the same iteration as cuFFT transforms plus one elementwise kernel per "
                                         "step, launched from the host (plain PyTorch)"},
    }


def run_reference(args):
    """The oracle (this method's reference implementation) timed on every host core: each step
    solves one slice per core of the workload, 100 iterations each, in a spawn process pool."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import phantoms
    from oracle import pd_oracle as O

    pool = make_oracle_pool()
    pb = phantoms.config2(SLICES)
    L, tau, sigma = O.step_sizes(H, W)
    n_sl = min(pool._processes, SLICES)
    n_it = 100  # bounded sample per step
    for _ in range(args.warmup):
        cpu_oracle_all_cores(pb.field[:n_sl], pb.mask[:n_sl], pb.lam, tau, sigma, 10, pool)
    times = []
    for _ in range(args.steps):
        _, dt, nproc = cpu_oracle_all_cores(pb.field[:n_sl], pb.mask[:n_sl], pb.lam, tau, sigma, n_it, pool)
        times.append(dt)
    pool.close()
    value = n_sl * H * W * n_it * len(times) / sum(times)
    line = {
        "impl": "reference",
        "metric": "PD voxel-iterations/s",
        "value": value,
        "unit": "voxel-iter/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "slices": SLICES, "n_iter": N_ITER},
        "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": nproc, "kind": "oracle",
                         "sample": f"{n_sl} slices x {n_it} iterations per step of the 256x256x64 workload, "
                                   "one slice per process", **host_description()},
        "e2e": {"value": value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import numpy as np
    import torch

    import paper_2006_09808_gb300 as pcs
    import phantoms
    from paper_2006_09808_gb300.sharding import max_over_ranks

    ws, rank, local = dist_env()
    pool = make_oracle_pool() if (rank == 0 and not args.no_cpu_baseline) else None  # before any GPU call
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pcs.load_library()

    # every rank solves its own volume (different phantom seed): weak scaling
    pb = phantoms.volume(H, W, SLICES, seed=rank, lam=LAM, n_iter=N_ITER, name="bench")
    field = torch.from_numpy(pb.field).to(dev)
    mask = torch.from_numpy(pb.mask).to(dev)
    chi = torch.empty_like(field)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)  # a real stream: the solve is replayed as a captured CUDA graph
    torch.cuda.set_stream(stream)
    ctx = pcs.pcs_create(H, W, SLICES, cluster_size=args.cluster_size, max_clusters=args.max_clusters,
                         kernel=args.kernel, threads=args.threads, use_graph=not args.no_graph, stream=stream)
    ones = torch.ones((1, H, W), dtype=torch.uint8, device=dev)
    L = pcs.pcs_opnorm(ctx, ones, 300)[0]  # step sizes of the pseudocode: tau = sigma = 1/L
    tau = sigma = 1.0 / L

    def step():
        pcs.pcs_solve_slices(ctx, field, mask, LAM, tau, sigma, N_ITER, chi)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    pcs.pcs_check(ctx)  # a balanced-schedule wait that gave up would raise PCS_ETIMEOUT here
    chi_warm = chi.clone()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between steps (not timed)
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    dev_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    pcs.pcs_check(ctx)  # every timed solve completed its schedule (else PCS_ETIMEOUT: the run fails)
    assert torch.equal(chi, chi_warm), "a timed solve differs from the warm-up solve"
    ms_step = sum(dev_ms) / len(dev_ms)
    ms_step = max_over_ranks(ms_step, device=dev)  # slowest rank sets the job time
    work = SLICES * H * W * N_ITER  # voxel-iterations per rank per step
    value = ws * work / (ms_step * 1e-3)

    # ---- end to end through the host-buffer C entry point (pinned host memory)
    hf = torch.from_numpy(pb.field).pin_memory().numpy()
    hm = torch.from_numpy(pb.mask).pin_memory().numpy()
    hc = torch.empty(pb.field.shape, dtype=torch.float32).pin_memory().numpy()
    pcs.pcs_solve_slices_host(ctx, hf, hm, LAM, tau, sigma, N_ITER, hc)  # warm the staging buffers
    e2e_t = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pcs.pcs_solve_slices_host(ctx, hf, hm, LAM, tau, sigma, N_ITER, hc)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_t) / len(e2e_t)
    e2e_s = max_over_ranks(e2e_s, device=dev)  # (pcs_solve_slices_host checks the schedule itself)
    dev_chi = chi.cpu().numpy()
    assert np.array_equal(dev_chi, hc), "host-buffer path differs from the device path"

    # ---- the plain per-slice GPU loop (one launch per slice, one slice after another)
    plain = None
    if args.plain_loop:
        ctx1 = pcs.pcs_create(H, W, 1, stream=stream)
        chi1 = torch.empty_like(chi)
        pcs.pcs_solve_slices(ctx1, field[:1], mask[:1], LAM, tau, sigma, N_ITER, chi1[:1])  # warm
        flush.fill_(0.5)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s_ in range(SLICES):
            pcs.pcs_solve_slices(ctx1, field[s_:s_ + 1], mask[s_:s_ + 1], LAM, tau, sigma, N_ITER, chi1[s_:s_ + 1])
        t1.record(stream)
        torch.cuda.synchronize()
        ms_plain = t0.elapsed_time(t1)
        assert np.array_equal(chi1.cpu().numpy(), dev_chi), "per-slice loop differs from the batched solve"
        plain = {"value": work / (ms_plain * 1e-3), "unit": "voxel-iter/s", "ms_per_volume": ms_plain,
                 "launches": SLICES, "note": "64 sequential single-slice solves, same kernel"}
        pcs.pcs_destroy(ctx1)
    pcs.pcs_destroy(ctx)
    cufft = None
    if args.cufft and rank == 0:
        cufft = cufft_comparison(field, mask, LAM, tau, sigma, N_ITER, stream, chi)
        assert cufft["unfused_library_loop"]["rel_l2_vs_fused_chi"] <= 1e-4, cufft

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        hbm_peak = float(peaks["hbm_gbs"])
        achieved = ALG_BYTES_PER_VOXEL_ITER * work / (ms_step * 1e-3) / 1e9
        clocks = clk.summary()
        fp32_peak = 152 * 128 * 2 * 2.070e9 / 1e12  # TFLOP/s at the maximum SM clock
        alu_achieved = ALG_FLOPS_PER_VOXEL_ITER * work / (ms_step * 1e-3) / 1e12
        traffic = profiled_traffic()
        line = {
            "metric": "PD voxel-iterations/s",
            "value": value,
            "unit": "voxel-iter/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": WORKLOAD, "H": H, "W": W, "slices": SLICES, "n_iter": N_ITER, "lambda": LAM,
                "parallelism": f"slices-dp{ws}", "l2": "flushed between steps (256 MiB device write)",
                "cluster_size": args.cluster_size or "default",
                "max_clusters": args.max_clusters or "all resident",
                "kernel": {0: "default", 1: "streaming", 2: "resident"}[args.kernel],
                "threads": args.threads or "default",
            },
            "roofline": {
                "bound": "latency (L2/DSMEM)", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "frac_of": "the measured HBM copy peak, in useful bytes (37 B per voxel-iteration)",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "alg_bytes_per_voxel_iter": ALG_BYTES_PER_VOXEL_ITER,
                "limiter": LIMITER_2D,
                "fp32_alu": {"achieved_tflops": alu_achieved, "peak_tflops": fp32_peak,
                             "frac": alu_achieved / fp32_peak,
                             "alg_flops_per_voxel_iter": ALG_FLOPS_PER_VOXEL_ITER},
            },
            "e2e": {"value": ws * work / e2e_s, "unit": "voxel-iter/s",
                    "h2d_bytes_per_step": int(pb.field.nbytes + pb.mask.nbytes),
                    "d2h_bytes_per_step": int(pb.field.nbytes)},
            "gpu_launches": args.steps,
            "batched_vs_plain": None if plain is None else {"plain_per_slice_loop": plain,
                                                             "speedup": plain["ms_per_volume"] / ms_step},
            "clocks": clocks,
            "wall_s_timed_region": t_wall,
            "L": L,
        }
        if cufft is not None:
            cufft["fused_vs_unfused"] = cufft["unfused_library_loop"]["ms"] / ms_step
            cufft["fused_vs_fft_passes_only"] = cufft["cufft_fft_passes_only"]["ms"] / ms_step
            line["vs_cufft"] = cufft
        if pool is not None:
            cv, dt = cpu_oracle_sample(pb, tau, sigma, 4, N_ITER)
            n_all = pool._processes
            av, adt, nproc = cpu_oracle_all_cores(pb.field[:n_all], pb.mask[:n_all], pb.lam, tau, sigma, N_ITER, pool)
            host = host_description()
            line["cpu_baseline"] = {"value": cv, "unit": "voxel-iter/s", "cores": 1, "kind": "oracle",
                                    "sample": f"4 slices x {N_ITER} iterations of this workload ({dt:.1f} s), "
                                              "one core (the paper's sequential CPU method)",
                                    "all_cores": {"value": av, "unit": "voxel-iter/s", "cores": nproc,
                                                  "sample": f"{n_all} slices x {N_ITER} iterations, one slice per "
                                                            f"process ({adt:.1f} s wall)"},
                                    **host}
            line["speedup_vs_cpu"] = {"one_core": value / cv, "all_cores": value / av, "paper": PAPER_SPEEDUP}
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# 3-D variant (the whole volume one unknown): state and inputs 45 B (read+write chi, p, qx, qy,
# qz; read dB, mask) plus the half spectrum through global memory, 4 passes of (W/2+1)/W x 8 B per
# dipole convolution (slice kernel writes, z pass reads and writes, slice kernel reads), 2 per iteration
ALG_BYTES_3D = 45 + 2 * 4 * 8 * (W // 2 + 1) / W
STEP_3D = 1.0 / (4.0 / 9.0 + 12.0) ** 0.5  # tau = sigma: ||K|| <= sqrt(||D||^2 + ||G||^2) for any 0/1 mask


def run_volume3d(args):
    """3-D variant on the same 256 x 256 x 64 volume: one pcs_solve_volume_3d call per step."""
    import numpy as np
    import torch

    import paper_2006_09808_gb300 as pcs
    import phantoms

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pcs.load_library()
    pb = phantoms.volume(H, W, SLICES, seed=rank, lam=LAM, n_iter=N_ITER, name="bench3d")
    field = torch.from_numpy(pb.field).to(dev)
    mask = torch.from_numpy(pb.mask).to(dev)
    chi = torch.empty_like(field)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        pcs.pcs_solve_volume_3d(field, mask, LAM, STEP_3D, STEP_3D, N_ITER, chi, stream=stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    ms_step = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    work = SLICES * H * W * N_ITER
    # end to end: pinned host field and mask in, chi out, around the same call
    hf = torch.from_numpy(pb.field).pin_memory()
    hm = torch.from_numpy(pb.mask).pin_memory()
    hc = torch.empty(pb.field.shape, dtype=torch.float32).pin_memory()
    e2e = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        field.copy_(hf, non_blocking=True)
        mask.copy_(hm, non_blocking=True)
        step()
        hc.copy_(chi, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    assert torch.equal(hc, chi.cpu())
    if rank == 0:
        peaks, peak_kind = measured_peaks()
        hbm_peak = float(peaks["hbm_gbs"])
        achieved = ALG_BYTES_3D * work / (ms_step * 1e-3) / 1e9
        line = {
            "metric": "PD voxel-iterations/s (3-D variant)",
            "value": work / (ms_step * 1e-3),
            "unit": "voxel-iter/s",
            "n_gpus": 1,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "3-D: the 256x256x64 volume as one unknown (3-D G and D, B0 along z), "
                                   "500 PD iterations, lambda=5e-4", "H": H, "W": W, "slices": SLICES,
                       "n_iter": N_ITER, "tau_sigma": STEP_3D, "l2": "flushed between steps (256 MiB device write)"},
            "roofline": {"bound": "latency (HBM round trips of the row kernel; the plane kernel issue- and "
                                   "shared-pipe-bound)", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "frac_of": "the measured HBM copy peak, in useful bytes (state, inputs and the half "
                                    "spectrum's four passes per convolution)",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "alg_bytes_per_voxel_iter": ALG_BYTES_3D},
            "e2e": {"value": work / (sum(e2e) / len(e2e)), "unit": "voxel-iter/s",
                    "h2d_bytes_per_step": int(pb.field.nbytes + pb.mask.nbytes),
                    "d2h_bytes_per_step": int(pb.field.nbytes)},
            "gpu_launches": args.steps * (4 * N_ITER - 1),
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            from oracle import pd_oracle_3d as O3  # cpu_baseline leg only

            n_it = 3
            t0 = time.perf_counter()
            O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, LAM, STEP_3D, STEP_3D, n_it)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": work / N_ITER * n_it / dt, "unit": "voxel-iter/s", "cores": 1,
                                    "kind": "oracle",
                                    "sample": f"the whole volume x {n_it} iterations ({dt:.1f} s)"}
        print(json.dumps(line), flush=True)
    return 0


NATIVE_H, NATIVE_W, NATIVE_S = 256, 258, 25
STEP_2D_SAFE = 1.0 / (4.0 / 9.0 + 8.0) ** 0.5  # ||K|| <= sqrt(4/9 + 8) for every 0/1 mask


def run_native_shape(args):
    """Any-size path on the stent acquisition's slice shape, 256 x 258 x 25: one
    pcs_solve_slices_generic call per step (500 iterations)."""
    import numpy as np
    import torch

    import paper_2006_09808_gb300 as pcs
    import phantoms

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pcs.load_library()
    pb = phantoms.volume(NATIVE_H, NATIVE_W, NATIVE_S, seed=rank, lam=LAM, n_iter=N_ITER, name="bench258")
    field = torch.from_numpy(pb.field).to(dev)
    mask = torch.from_numpy(pb.mask).to(dev)
    chi = torch.empty_like(field)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        pcs.pcs_solve_slices_generic(field, mask, LAM, STEP_2D_SAFE, STEP_2D_SAFE, N_ITER, chi, stream=stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    ms_step = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    work = NATIVE_S * NATIVE_H * NATIVE_W * N_ITER
    hf = torch.from_numpy(pb.field).pin_memory()
    hm = torch.from_numpy(pb.mask).pin_memory()
    hc = torch.empty(pb.field.shape, dtype=torch.float32).pin_memory()
    e2e = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        field.copy_(hf, non_blocking=True)
        mask.copy_(hm, non_blocking=True)
        step()
        hc.copy_(chi, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    assert torch.equal(hc, chi.cpu())
    if rank == 0:
        peaks, peak_kind = measured_peaks()
        hbm_peak = float(peaks["hbm_gbs"])
        achieved = ALG_BYTES_PER_VOXEL_ITER * work / (ms_step * 1e-3) / 1e9
        line = {
            "metric": "PD voxel-iterations/s (256x258 slices)",
            "value": work / (ms_step * 1e-3),
            "unit": "voxel-iter/s",
            "n_gpus": 1,
            "steps": args.steps,
            "warmup": max(args.warmup, 3),
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "the stent acquisition's shape: 25 slices of 256x258 (row FFT length 258 = "
                                   "2*3*43), 500 PD iterations, lambda=5e-4", "H": NATIVE_H, "W": NATIVE_W,
                       "slices": NATIVE_S, "n_iter": N_ITER, "tau_sigma": STEP_2D_SAFE,
                       "l2": "flushed between steps (256 MiB device write)"},
            "roofline": {"bound": "latency (L2)", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "frac_of": "the measured HBM copy peak, in useful bytes (37 B per voxel-iteration)",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "alg_bytes_per_voxel_iter": ALG_BYTES_PER_VOXEL_ITER},
            "e2e": {"value": work / (sum(e2e) / len(e2e)), "unit": "voxel-iter/s",
                    "h2d_bytes_per_step": int(pb.field.nbytes + pb.mask.nbytes),
                    "d2h_bytes_per_step": int(pb.field.nbytes)},
            "gpu_launches": args.steps * (4 * N_ITER - 1),
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            from oracle import pd_oracle as O  # cpu_baseline leg only

            n_it = 20
            t0 = time.perf_counter()
            O.pd_solve(pb.field.astype(np.float64), pb.mask, LAM, STEP_2D_SAFE, STEP_2D_SAFE, n_it)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": work / N_ITER * n_it / dt, "unit": "voxel-iter/s", "cores": 1,
                                    "kind": "oracle",
                                    "sample": f"all 25 slices x {n_it} iterations ({dt:.1f} s)"}
        print(json.dumps(line), flush=True)
    return 0


def run_fieldmap(args):
    """Field-map preprocessing (pcs_field_map) of the 256 x 256 x 64 volume's two acquisitions."""
    import torch

    import paper_2006_09808_gb300 as pcs
    import phantoms

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pcs.load_library()
    pb = phantoms.volume(H, W, SLICES, seed=rank, lam=LAM, n_iter=N_ITER, name="benchfm")
    s0h, s1h = phantoms.echo_pair(pb.field, pb.mask, seed=rank + 100)
    s0 = torch.from_numpy(s0h).to(dev)
    s1 = torch.from_numpy(s1h).to(dev)
    f = torch.empty(s0.shape, dtype=torch.float32, device=dev)
    wt = torch.empty_like(f)
    m = torch.empty(s0.shape, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        pcs.pcs_field_map(s0, s1, 0.6e-3, 3.0, 0.25, f, wt, m, stream=stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    n = SLICES * H * W
    alg = 25  # read two complex64 acquisitions (16 B), write field, weight (8 B) and mask (1 B)
    if rank == 0:
        peaks, peak_kind = measured_peaks()
        hbm_peak = float(peaks["hbm_gbs"])
        achieved = alg * n / (ms * 1e-3) / 1e9
        line = {
            "metric": "field-map voxels/s", "value": n / (ms * 1e-3), "unit": "voxel/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "field map, mask and weighting from two 256x256x64 complex acquisitions "
                                   "(T_shift 0.6 ms, 3 T)", "l2": "flushed between steps (256 MiB device write)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "alg_bytes_per_voxel": alg, "note": "the kernels read the first acquisition twice "
                                                             "(maximum pass): 33 B/voxel moved"},
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    return 0


def _gen_volume(sp):
    """One volume of the uneven-batch recipe (a worker of the generation pool)."""
    import phantoms

    pb = phantoms.volume(sp["size"], sp["size"], sp["slices"], seed=sp["seed"], lam=sp["lam"], n_iter=sp["n_iter"])
    return pb.field, pb.mask


def run_uneven(args):
    """Uneven batch: 48 volumes of 128^2..512^2 slices (16-96 slices each, lambda in {2e-4, 5e-4,
    1e-3}), 400 iterations, solved by one pcs_batch_solve call per step (one persistent launch
    per slice size, autotuned variants).  Compared with a per-volume loop (one pcs_solve_slices
    per volume, one after another) and a per-slice loop (one launch per slice, timed on a
    stratified subset and extrapolated by voxel-iterations per size)."""
    import numpy as np
    import torch

    import paper_2006_09808_gb300 as pcs
    import phantoms

    ws, rank, local = dist_env()
    pool = make_oracle_pool() if (rank == 0 and not args.no_cpu_baseline) else None  # before any GPU call
    specs = phantoms.config4_volumes()
    n_iter = specs[0]["n_iter"]
    if pool is not None:
        data = pool.map(_gen_volume, specs)
    else:
        data = [_gen_volume(sp) for sp in specs]
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pcs.load_library()
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    fields = [torch.from_numpy(f).to(dev) for f, _ in data]
    masks = [torch.from_numpy(m).to(dev) for _, m in data]
    chis = [torch.empty_like(f) for f in fields]
    vols = [(fields[k], masks[k], specs[k]["lam"], chis[k]) for k in range(len(specs))]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sizes = sorted({sp["size"] for sp in specs})
    vi_size = {n: sum(sp["slices"] * n * n * n_iter for sp in specs if sp["size"] == n) for n in sizes}
    work = sum(vi_size.values())

    batch = pcs.pcs_batch_create(autotune=True, stream=stream)
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1.0)
        pcs.pcs_batch_solve(batch, vols, n_iter)
    torch.cuda.synchronize()
    pcs.pcs_batch_check(batch)
    warm = [c.clone() for c in chis]
    tun = {n: pcs.pcs_batch_tuning(batch, n, n) for n in sizes}
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            pcs.pcs_batch_solve(batch, vols, n_iter)
            ends[k].record(stream)
        torch.cuda.synchronize()
    pcs.pcs_batch_check(batch)
    assert all(torch.equal(a, b) for a, b in zip(chis, warm)), "a timed batch differs from the warm-up batch"
    ms_step = sum(s_.elapsed_time(e) for s_, e in zip(starts, ends)) / args.steps

    # end to end: pinned host inputs in, chi out, around the same call
    hf = [torch.from_numpy(f).pin_memory() for f, _ in data]
    hm = [torch.from_numpy(m).pin_memory() for _, m in data]
    hc = [torch.empty(f.shape, dtype=torch.float32).pin_memory() for f, _ in data]
    e2e = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in zip(fields, hf):
            a.copy_(b, non_blocking=True)
        for a, b in zip(masks, hm):
            a.copy_(b, non_blocking=True)
        pcs.pcs_batch_solve(batch, vols, n_iter)
        for a, b in zip(hc, chis):
            a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    pcs.pcs_batch_check(batch)
    assert all(torch.equal(a, b.cpu()) for a, b in zip(hc, warm))

    # per-volume loop: one pcs_solve_slices per volume (the batch's variant of its size), in turn
    def tuned_ctx(n, S):  # the variant the batch's autotuner chose for this size
        t = tun[n]
        return pcs.pcs_create(n, n, S, cluster_size=t["cluster_size"], kernel=t["kernel"], threads=t["threads"],
                              tile=t["tile"],
                              stream=stream)

    ctxs = {n: tuned_ctx(n, max(sp["slices"] for sp in specs if sp["size"] == n)) for n in sizes}
    flush.fill_(0.5)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    outs = [torch.empty_like(f) for f in fields]
    for k, sp in enumerate(specs):
        L = tun[sp["size"]]["L"]
        pcs.pcs_solve_slices(ctxs[sp["size"]], fields[k], masks[k], sp["lam"], 1 / L, 1 / L, n_iter, outs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    for c in ctxs.values():
        pcs.pcs_check(c)
    ms_volumes = t0.elapsed_time(t1)
    assert all(torch.equal(a, b) for a, b in zip(outs, warm)), "per-volume solves differ from the batch"
    # per-slice loop: one launch per slice, two slices of the first volume of each size
    per_slice_ms = 0.0
    sub = {}
    for n in sizes:
        k = next(i for i, sp in enumerate(specs) if sp["size"] == n)
        c1 = tuned_ctx(n, 1)
        L = tun[n]["L"]
        o1 = torch.empty_like(fields[k][:1])
        pcs.pcs_solve_slices(c1, fields[k][:1], masks[k][:1], specs[k]["lam"], 1 / L, 1 / L, n_iter, o1)  # warm
        torch.cuda.synchronize()
        t0.record(stream)
        for s_ in range(2):
            pcs.pcs_solve_slices(c1, fields[k][s_:s_ + 1], masks[k][s_:s_ + 1], specs[k]["lam"], 1 / L, 1 / L,
                                 n_iter, o1)
        t1.record(stream)
        torch.cuda.synchronize()
        pcs.pcs_destroy(c1)
        rate = 2 * n * n * n_iter / (t0.elapsed_time(t1) * 1e-3)
        sub[n] = rate
        per_slice_ms += vi_size[n] / rate * 1e3
    for c in ctxs.values():
        pcs.pcs_destroy(c)
    pcs.pcs_batch_destroy(batch)

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        hbm_peak = float(peaks["hbm_gbs"])
        value = work / (ms_step * 1e-3)
        achieved = ALG_BYTES_PER_VOXEL_ITER * work / (ms_step * 1e-3) / 1e9
        line = {
            "metric": "PD voxel-iterations/s (uneven batch)",
            "value": value, "unit": "voxel-iter/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "uneven batch: 48 volumes, slices 128^2..512^2, 16-96 slices each, lambda in "
                                   "{2e-4, 5e-4, 1e-3}, 400 PD iterations, one pcs_batch_solve per step",
                       "voxels": work // n_iter, "n_iter": n_iter,
                       "l2": "flushed between steps (256 MiB device write); inputs 1.3 GB > L2"},
            "roofline": {"bound": "latency (L2/DSMEM)", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None,
                         "frac_of": "the measured HBM copy peak, in useful bytes (37 B per voxel-iteration)",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "alg_bytes_per_voxel_iter": ALG_BYTES_PER_VOXEL_ITER},
            "e2e": {"value": work / (sum(e2e) / len(e2e)), "unit": "voxel-iter/s",
                    "h2d_bytes_per_step": int(sum(f.nbytes + m.nbytes for f, m in data)),
                    "d2h_bytes_per_step": int(sum(f.nbytes for f, _ in data))},
            "gpu_launches": args.steps * len(sizes),
            "batched_vs_plain": {
                "per_volume_loop": {"value": work / (ms_volumes * 1e-3), "unit": "voxel-iter/s",
                                    "ms": ms_volumes, "note": "48 pcs_solve_slices calls, one after another"},
                "per_slice_loop": {"value": work / (per_slice_ms * 1e-3), "unit": "voxel-iter/s",
                                   "ms_extrapolated": per_slice_ms,
                                   "note": "one launch per slice, timed on 2 slices per size, extrapolated"},
                "speedup_vs_per_volume": ms_volumes / ms_step,
                "speedup_vs_per_slice": per_slice_ms / ms_step,
            },
            "tuning": {str(n): {k: tun[n][k] for k in ("cluster_size", "kernel", "threads", "tile", "L")} for n in sizes},
            "clocks": clk.summary(),
        }
        if pool is not None:
            from oracle import pd_oracle as O  # noqa: F401  (cpu_baseline leg only)

            one_t, all_t, nproc = 0.0, 0.0, pool._processes
            n_cpu = 40
            for n in sizes:
                k = next(i for i, sp in enumerate(specs) if sp["size"] == n)
                f, m = data[k]
                L = tun[n]["L"]
                t_a = time.perf_counter()
                _oracle_slice((f[0], m[0], specs[k]["lam"], 1 / L, 1 / L, n_cpu))
                one_t += vi_size[n] / (n * n * n_cpu / (time.perf_counter() - t_a))
                reps = [f[s_ % f.shape[0]] for s_ in range(nproc)]
                repm = [m[s_ % m.shape[0]] for s_ in range(nproc)]
                av, _, _ = cpu_oracle_all_cores(reps, repm, specs[k]["lam"], 1 / L, 1 / L, n_cpu, pool)
                all_t += vi_size[n] / av
            line["cpu_baseline"] = {"value": work / one_t, "unit": "voxel-iter/s", "cores": 1, "kind": "oracle",
                                    "sample": f"one slice per size x {n_cpu} iterations, extrapolated by "
                                              "voxel-iterations per size",
                                    "all_cores": {"value": work / all_t, "unit": "voxel-iter/s", "cores": nproc,
                                                  "sample": f"{nproc} slices per size x {n_cpu} iterations, one "
                                                            "slice per process, extrapolated"},
                                    **host_description()}
            line["speedup_vs_cpu"] = {"one_core": value / (work / one_t), "all_cores": value / (work / all_t),
                                      "paper": PAPER_SPEEDUP}
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.close()
    return 0


def run_serve(args):
    """Serving leg: Poisson arrivals of uneven-batch-style volumes, streamed slice by slice."""
    import heapq

    import numpy as np
    import torch

    import paper_2006_09808_gb300 as pcs
    import phantoms

    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    pcs.load_library()
    n_iter = 400
    reqs = phantoms.config5_arrivals(args.requests, rate_hz=args.rate, seed=0)
    sizes = sorted({r["size"] for r in reqs})
    # one pinned pool volume per size (96 slices); a request takes its first S slices
    pool = {}
    for k, H in enumerate(sizes):
        pb = phantoms.volume(H, H, 96, seed=5000 + k, lam=5e-4, n_iter=n_iter)
        pool[H] = (torch.from_numpy(pb.field).pin_memory().numpy(), torch.from_numpy(pb.mask).pin_memory().numpy())
    sv = pcs.pcs_serve_start(hbm_budget_bytes=120 << 30, slots=args.slots, n_iter=n_iter, autotune=True)
    tun = {H: pcs.pcs_serve_prepare_size(sv, H, H) for H in sizes}
    outs = {}
    events = []  # (time, seq, kind, request index, s0, n)
    for i, r in enumerate(reqs):
        heapq.heappush(events, (r["t"], 2 * i, "open", i, 0, 0))
        S = r["slices"]
        n_chunks = 4
        for c in range(n_chunks):  # slices released uniformly over 100 ms after arrival
            s0, s1 = c * S // n_chunks, (c + 1) * S // n_chunks
            if s1 > s0:
                heapq.heappush(events, (r["t"] + 0.1 * (c + 1) / n_chunks, 2 * i + 1, "push", i, s0, s1 - s0))
    ids, done = {}, {}
    rid_to_i = {}
    check_every = 50  # these requests' chi is kept and compared with the per-request solves
    t0 = time.perf_counter()
    while events or len(done) < len(reqs):
        now = time.perf_counter() - t0
        while events and events[0][0] <= now:
            _, _, kind, i, s0, n = heapq.heappop(events)
            r = reqs[i]
            H, S = r["size"], r["slices"]
            if kind == "open":
                outs[i] = torch.empty((S, H, H), dtype=torch.float32).pin_memory().numpy()
                ids[i] = pcs.pcs_serve_open(sv, H, H, S, r["lam"], outs[i])
                rid_to_i[ids[i]] = i
            else:
                f, m = pool[H]
                pcs.pcs_serve_push(sv, ids[i], s0, f[s0:s0 + n], m[s0:s0 + n])
        for rid, lat, st_ in pcs.pcs_serve_poll(sv):
            if st_ != pcs.PCS_OK:
                raise RuntimeError(f"request {rid} failed with status {st_}")
            done[rid] = lat
            if rid_to_i[rid] % check_every:
                outs.pop(rid_to_i[rid])  # release the pinned output (only sampled requests are kept)
        time.sleep(0.0005)
    st = pcs.pcs_serve_stats(sv)
    pcs.pcs_serve_stop(sv)
    vox_iters = sum(r["slices"] * r["size"] ** 2 * n_iter for r in reqs)
    window = reqs[-1]["t"] - reqs[0]["t"]
    # baseline: the same requests solved one after another with plain per-request calls
    base_reqs = reqs[: args.baseline_requests] if args.baseline_requests > 0 else reqs
    if args.no_baseline:
        base_reqs = []
    ctxs = {}
    t_base, vi_base = 0.0, 0.0
    for r in base_reqs:
        H, S = r["size"], r["slices"]
        if H not in ctxs:
            t = tun[H]
            ctxs[H] = pcs.pcs_create(H, H, 96, cluster_size=t["cluster_size"], kernel=t["kernel"],
                                     threads=t["threads"], tile=t["tile"])
        f, m = pool[H]
        out = np.empty((S, H, H), np.float32)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        pcs.pcs_solve_slices_host(ctxs[H], f[:S], m[:S], r["lam"], 1 / tun[H]["L"], 1 / tun[H]["L"], n_iter, out)
        t_base += time.perf_counter() - ta
        vi_base += S * H * H * n_iter
        if r["idx"] in outs:  # served == per-request solve, bit for bit (same kernel variant and step)
            assert np.array_equal(outs[r["idx"]], out), f"served request {r['idx']} differs from its plain solve"
    for c in ctxs.values():
        pcs.pcs_destroy(c)
    line = {
        "metric": "PD voxel-iterations/s (served)",
        "value": st["voxel_iters"] / st["span_s"],
        "unit": "voxel-iter/s",
        "n_gpus": 1,
        "higher_is_better": True,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} Poisson arrivals at {args.rate:g} volumes/s of uneven-batch-"
                               "style volumes (128..512^2, 16-96 slices, 400 iterations), slices released over "
                               "100 ms, 120 GB budget", "slots": args.slots, "rate_hz": args.rate},
        "latency_s": {"p50": st["p50_s"], "p99": st["p99_s"], "max": st["max_s"]},
        "offered_voxel_iter_per_s": vox_iters / max(window, 1e-9),
        "served": st,
        "per_request_plain_loop": None if not base_reqs else {
            "value": vi_base / t_base, "unit": "voxel-iter/s", "requests": len(base_reqs),
            "note": "pcs_solve_slices_host, one after another"},
        "tuning": {H: {k: tun[H][k] for k in ("cluster_size", "kernel", "threads", "tile", "L")} for H in sizes},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cluster-size", type=int, default=0)
    ap.add_argument("--max-clusters", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0, help="0 default, 1 streaming, 2 resident")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="direct launches instead of CUDA-graph replay")
    ap.add_argument("--cufft", action=argparse.BooleanOptionalAction, default=True,
                    help="also time cuFFT doing the FFT passes alone and the unfused library loop (comparison)")
    ap.add_argument("--plain-loop", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the plain per-slice GPU loop (one timed volume)")
    ap.add_argument("--workload", choices=["volume", "serve", "volume3d", "fieldmap", "native", "uneven"],
                    default="volume",
                    help="volume: the 256x256x64 solve (default); serve: the serving loop; "
                         "volume3d: the 3-D variant on the same volume; fieldmap: the preprocessing step; "
                         "native: the any-size path on 25 slices of 256x258; uneven: the 48-volume uneven batch")
    ap.add_argument("--requests", type=int, default=400, help="serving: number of requests (the 400-request window)")
    ap.add_argument("--slots", type=int, default=8, help="serving: requests in flight")
    ap.add_argument("--rate", type=float, default=40.0, help="serving: mean arrivals per second (Poisson)")
    ap.add_argument("--no-baseline", action="store_true", help="serving: skip the per-request baseline")
    ap.add_argument("--baseline-requests", type=int, default=0,
                    help="serving: requests in the per-request baseline (0: all of them)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "volume3d":
        return run_volume3d(args)
    if args.workload == "fieldmap":
        return run_fieldmap(args)
    if args.workload == "native":
        return run_native_shape(args)
    if args.workload == "uneven":
        return run_uneven(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
