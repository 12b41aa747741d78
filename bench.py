#!/usr/bin/env python
"""ADMM throughput of t-SVT tensor completion / tensor RPCA on one GB300.

One step = one complete ADMM solve of a seeded synthetic workload with its inputs already
resident on the GPU; `value` is ADMM iterations per second over the whole job (for the
batched workload an iteration advances all 64 tensors).  Workloads (`--workload`):

  batch    64 tensors of uneven shapes (n1, n2 in [48, 256], n3 in [8, 64]), half completion
           and half RPCA, 100 iterations, one batched call                 [default]
  video    grayscale video completion 144x176x100 (translating texture + N(0, 0.01^2)
           noise), 20% of entries observed, 150 iterations
  rpca     tensor RPCA, L = tubal-rank-10 t-product of N(0,1) factors 240x320x60,
           10% entrywise corruption U[-5, 5], lambda = 1/sqrt(320*60), 200 iterations
  color    colour video completion 288x352x3x60 (per-channel textures), 15% observed,
           150 iterations, FFT along modes 3 and 4
  multiview  5-way multi-view colour video completion 144x176x3x2x40 (a texture per channel
           and view), 20% observed, 150 iterations, FFT along modes 3, 4 and 5
  lowrank  tubal-rank-3 32x32x16, 50% observed, 100 iterations
  batch    64 tensors of uneven shapes (n1, n2 in [48, 256], n3 in [8, 64]), half completion
           and half RPCA, 100 iterations, one batched call

`--precision` picks the slice SVT of the headline line: fp32 (plain one-sided Jacobi) or a
mixed form (tf32, bf16, 3xtf32: tensor-core products; rand_fp32: CUDA-core products).  For
the plain headline, `--mixed` (default 3xtf32) also times that mixed form on the same
workload and steps and reports it, with its final recovery error and whether it meets the
equal-error rule (e_mixed <= e_plain + 0.01 e_plain + 1e-5: no worse than the plain form's
recovery error beyond 1%), under the key "mixed"; for the batch the rule is applied to every
tensor and the verdict lists the tensors that miss it.  With the default batch workload the
line also carries, under "color", the plain and mixed forms of the 288x352x3x60 colour video
(the largest single tensor) timed the same way (`--no-color` skips it).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                        [--workload NAME] [--precision P] [--mixed P|none]
For N > 1 run under torchrun (one rank per GPU); every rank solves its own replica of a
single-tensor workload, and the 64 tensors of the batch are split over the ranks by cost
(longest processing time first): weak scaling, no collective on the data path; the slowest
rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "t-SVT ADMM iters/s & HBM/TC roofline %, mixed/batched vs plain FP32 at equal err"
FLUSH_BYTES = 256 << 20      # > 129 MB L2
FP32_LANES_PER_SM = 128
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rates
PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2, "3xtf32": 3, "rand_fp32": 4}
# executed tensor-core flops per algorithmic flop of a complex product (3M: 6 of 8; 3XTF32
# issues three products per real product)
EXECUTED_PER_ALG = {"tf32": 0.75, "bf16": 0.75, "3xtf32": 2.25, "rand_fp32": 0.0}

WORKLOADS = {
    "video": dict(kind="complete", iters=150, cpu_iters=10,
                  desc="grayscale video completion 144x176x100, 20% observed"),
    "rpca": dict(kind="rpca", iters=200, cpu_iters=2,
                 desc="tensor RPCA 240x320x60, tubal rank 10, 10% entrywise corruption"),
    "rpca_tube": dict(kind="rpca", iters=200, cpu_iters=2,
                      desc="tube-sparse tensor RPCA (eq. sparse2) on a 144x256x80 panning "
                           "video, 10% of pixel tubes corrupted in 10-frame blocks"),
    "color": dict(kind="complete", iters=150, cpu_iters=1,
                  desc="colour video completion 288x352x3x60, 15% observed"),
    "multiview": dict(kind="complete", iters=150, cpu_iters=1,
                      desc="5-way multi-view colour video completion 144x176x3x2x40, 20% "
                           "observed, DFT along modes 3-5"),
    "lowrank": dict(kind="complete", iters=100, cpu_iters=100,
                    desc="low-tubal-rank completion 32x32x16, rank 3, 50% observed"),
    "factor": dict(kind="factor", iters=1, cpu_iters=1,
                   desc="economy t-SVD (Algorithm 1) of the 144x176x100 video, all "
                        "min(n1, n2) singular tubes"),
    "compress": dict(kind="compress", iters=1, cpu_iters=1,
                     desc="t-SVD compression (Sec. 3, Methods 1 and 2) of the 144x176x100 "
                          "video: RSE against the compression ratio"),
    "batch": dict(kind="batch", iters=100, cpu_iters=10,
                  desc="64 uneven tensors (n1, n2 in [48, 256], n3 in [8, 64]), half "
                       "completion / half RPCA, one batched call"),
}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one tube-pass launch from an
# ncu capture of the colour-video workload, valid only for the kernel sources it was taken on
# (profiles/tube_tile_kernel_color_288x352x3x60.md); the slice SVT's traffic has no capture on
# the current source, so its roofline reports none.
TUBE_TRAFFIC = {"workload": "color",
                "sources": {"paper_1407_1785_gb300/csrc/tube_tile.cuh":
                            "0200a606ff6e438f8f86a5486581e4bdb0c500caa8365b9a944d2c87be1e8b8b",
                            "paper_1407_1785_gb300/csrc/tube_pass.cu":
                            "c8db9e21a8ca9b2ac2529373ff872fb62320ae3fa533fc2a30f6ed4348e14291"},
                "bytes_per_launch": 219881472 + 106778624}


def tube_traffic(workload):
    """The captured tube-pass traffic per launch when it applies to this workload and source."""
    if workload != TUBE_TRAFFIC["workload"]:
        return None
    for path, sha in TUBE_TRAFFIC["sources"].items():
        if file_sha256(os.path.join(ROOT, path)) != sha:
            return None
    return TUBE_TRAFFIC["bytes_per_launch"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batch")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32")
    ap.add_argument("--mixed", choices=sorted(PRECISIONS) + ["none"], default="3xtf32")
    ap.add_argument("--iters", type=int, default=0, help="ADMM iterations per step (0 = the "
                    "workload's count)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-iters", type=int, default=0)
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel directly instead of replaying captured CUDA "
                         "graphs (for kernel-by-kernel profilers)")
    ap.add_argument("--no-color", action="store_true",
                    help="batch workload: skip the colour-video lines reported alongside")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """The maximum of a per-rank scalar over all ranks (the rank itself when not distributed);
    works with the gloo (CPU) and NCCL (GPU) backends."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tensor_cost(dims):
    """Estimated slice-SVD work of one ADMM iteration of a tensor: m n^2 per distinct Fourier
    slice (n = min(n1, n2))."""
    m, n = max(dims[0], dims[1]), min(dims[0], dims[1])
    return float(m) * n * n * half_slices(dims)


def lpt_shard(costs, world):
    """Longest-processing-time split of independent tensors over `world` ranks: tensors in
    decreasing cost, each to the least loaded rank.  Returns one sorted index list per rank."""
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        if not shutil.which("nvidia-smi"):
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(
            ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        # the timed region starts once nvidia-smi writes samples: its start-up queries to the
        # driver would otherwise overlap (and slow) the first part of the region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def file_sha256(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def half_slices(dims):
    """Distinct Fourier slices the t-SVT computes: the half spectrum of the last mode, and on
    its self-conjugate columns (index 0 and n/2) one of each conjugate pair of indices of
    modes 3..N-1."""
    nf = int(np.prod(dims[2:-1])) if len(dims) > 3 else 1
    nh = dims[-1]
    self_cols = 1 + (1 if nh % 2 == 0 else 0)
    self_f = int(np.prod([1 + (1 if n % 2 == 0 else 0) for n in dims[2:-1]]))
    return nf * (nh // 2 + 1) - self_cols * ((nf - self_f) // 2)


def jacobi_gvl_flops(n1, n2, nslices):
    """Golub-Van Loan operation count of a complex SVD returning Sigma and V of an m x n
    matrix (m >= n): 4 (4 m n^2 + 8 n^3) real flops, per distinct Fourier slice."""
    m, n = max(n1, n2), min(n1, n2)
    return 4.0 * (4.0 * m * n * n + 8.0 * n ** 3) * nslices


def tube_bytes(dims):
    """Tube pass per iteration: read the complex half spectrum, write the next one, and read /
    write the real state tensors (completion: read Yn and V, write V; RPCA: read M and W,
    write W)."""
    N = int(np.prod(dims))
    n12 = dims[0] * dims[1]
    stored = int(np.prod(dims[2:-1])) * (dims[-1] // 2 + 1)
    sc = 8.0 * n12 * stored
    return 2 * sc + 3 * 4.0 * N


# ------------------------------------------------------------------------------- workloads

def build_workload(name, seed):
    """Host inputs of one workload: dict with kind, dims, M, omega / lam, truth; for the batch
    a list of such dicts under "items"."""
    from paper_1407_1785_gb300 import synth
    if name in ("video", "color", "multiview", "lowrank"):
        gen = {"video": synth.workload_video_completion, "color": synth.workload_color_video,
               "multiview": synth.workload_multiview_video,
               "lowrank": synth.workload_lowrank_completion}[name]
        X, om = gen(seed=seed)
        return dict(kind="complete", dims=X.shape, M=(X * om).astype(np.float32), omega=om,
                    truth=X)
    if name == "rpca":
        M, L0, S0, sup, lam = synth.workload_rpca(seed=seed)
        return dict(kind="rpca", dims=M.shape, M=M.astype(np.float32), lam=lam, truth=L0)
    if name == "rpca_tube":
        M, L0, S0, sup, lam = synth.workload_rpca_tube(seed=seed)
        return dict(kind="rpca", dims=M.shape, M=M.astype(np.float32), lam=lam, truth=L0,
                    tube=True)
    if name == "batch":
        items = synth.workload_batch(seed=seed)
        return dict(kind="batch", items=items)
    raise ValueError(name)


NO_GRAPHS = False


def ctx_options(wl):
    """Context options a workload needs besides precision (the tube-wise sparse term), and
    graphs off under --no-graphs."""
    from paper_1407_1785_gb300 import libtsvd
    opts = {"sparse_mode": libtsvd.SPARSE_TUBE} if wl.get("tube") else {}
    if NO_GRAPHS:
        opts["use_graphs"] = 0
    return opts


def to_device(wl):
    import torch
    from paper_1407_1785_gb300 import synth

    def one(it):
        d = dict(it)
        d["m"] = torch.from_numpy(synth.to_colmajor(it["M"])).cuda()
        if it["kind"] == "complete":
            d["o"] = torch.from_numpy(synth.to_colmajor(it["omega"], np.uint8)).cuda()
        d["out0"] = torch.empty_like(d["m"])
        d["out1"] = torch.empty_like(d["m"])
        return d
    if wl["kind"] == "batch":
        return dict(kind="batch", items=[one(it) for it in wl["items"]])
    return one(wl)


def solver(ctx, dw, iters):
    """A callable running one full solve through the C ABI (device buffers); returns stats."""
    if dw["kind"] == "complete":
        return lambda: ctx.tnn_complete(dw["m"], dw["o"], dw["dims"], iters, dw["out0"],
                                        stats=True)
    if dw["kind"] == "rpca":
        return lambda: ctx.trpca(dw["m"], dw["dims"], dw["lam"], iters, dw["out0"], dw["out1"],
                                 stats=True)
    probs = []
    for it in dw["items"]:
        q = dict(kind=it["kind"], dims=it["dims"], M=it["m"], out0=it["out0"], out1=it["out1"])
        if it["kind"] == "complete":
            q["omega"] = it["o"]
        else:
            q["lam"] = it["lam"]
        probs.append(q)
    return lambda: ctx.solve_batched(probs, iters, stats=True)


def recovery_errors(dw):
    """Relative Frobenius recovery error of each tensor against its ground truth."""
    from paper_1407_1785_gb300 import synth
    items = dw["items"] if dw["kind"] == "batch" else [dw]
    out = []
    for it in items:
        R = synth.from_colmajor(it["out0"].cpu().numpy(), it["dims"])
        out.append(float(np.linalg.norm(R - it["truth"]) / np.linalg.norm(it["truth"])))
    return out


def n_voxels(wl):
    items = wl["items"] if wl["kind"] == "batch" else [wl]
    return sum(int(np.prod(it["dims"])) for it in items)


# ------------------------------------------------------------------------------- oracle timing

def oracle_sample(wl, iters_sample):
    """Times the FP64 oracle on a bounded sample of the workload; returns (iters/s of the whole
    workload, seconds, description of the sample)."""
    import oracle
    oracle.build()
    items = wl["items"] if wl["kind"] == "batch" else [wl]
    take = items[:4] if wl["kind"] == "batch" else items
    t0 = time.perf_counter()
    for it in take:
        M = it["M"].astype(np.float64)
        if it["kind"] == "complete":
            oracle.tnn_complete(M, it["omega"], iters_sample)
        else:
            oracle.trpca(M, it["lam"], iters_sample,
                         sparse_mode=oracle.SPARSE_TUBE if it.get("tube") else oracle.SPARSE_ENTRY)
    dt = time.perf_counter() - t0
    frac = sum(int(np.prod(it["dims"])) for it in take) / n_voxels(wl)
    what = (f"first {iters_sample} ADMM iterations of the same workload" if wl["kind"] != "batch"
            else f"first {iters_sample} ADMM iterations of the first {len(take)} of the 64 "
                 f"tensors, scaled by their share of the voxels ({frac:.3f})")
    return iters_sample * frac / dt, dt, what + " (FP64 C oracle, OpenMP over slices)"


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    wl = build_workload(args.workload, 1)
    spec = WORKLOADS[args.workload]
    sample = args.cpu_sample_iters or max(1, min(spec["cpu_iters"], 2))
    for _ in range(args.warmup):
        oracle_sample(wl, sample)
    tot, what = 0.0, ""
    vals = []
    for _ in range(args.steps):
        v, dt, what = oracle_sample(wl, sample)
        tot += dt
        vals.append(v)
    value = len(vals) / sum(1.0 / v for v in vals)      # whole-run rate
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot * 1000.0 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "admm_iters_per_step": sample,
                   "seed": 1},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": what},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------- GPU runs

def timed_solves(solve, steps, flush, stream, barrier):
    """K timed solves (L2 flushed before each); returns (ms of the whole region, stats list).
    One untimed flush and solve run right before the region: the flush kernel's first launch
    (lazy module loading) and a GPU left idle while the clock sampler started stay outside."""
    import torch
    flush.zero_()
    solve()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(steps):
        flush.zero_()
        stats.append(solve())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return ev0.elapsed_time(ev1), stats


def sum_stats(stats, key):
    return sum(s[key] for s in stats)


def add_fp32_peak(peaks, device):
    """Measures the device's FP32 CUDA-core throughput (tsvd_measure_fp32_peak: the best of a
    scalar and a packed FP32x2 FMA loop) into peaks["fp32_tflops"]; falls back to the count
    SMs x 128 lanes x 2 flop x max SM clock, with the SM count from the device, if the
    measurement fails."""
    from paper_1407_1785_gb300 import libtsvd
    try:
        fma, fma2 = libtsvd.measure_fp32_peak(device)
        peaks["fp32_tflops"] = max(fma, fma2)
        peaks["fp32_fma_tflops"], peaks["fp32_fma2_tflops"] = fma, fma2
        peaks["fp32_source"] = ("measured: FP32 FMA loop (tsvd_measure_fp32_peak, best of "
                                "scalar and packed FP32x2)")
    except Exception as e:      # noqa: BLE001 -- report the derived figure instead
        import torch
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        peaks["fp32_tflops"] = sms * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e-6
        peaks["fp32_source"] = (f"derived ({e}): {sms} SMs x 128 FP32 lanes x 2 flop/FMA x "
                                "max SM clock")
    return peaks


def alu_peak(peaks):
    return peaks["fp32_tflops"]


def mixed_rooflines(stats, prec_name, peaks):
    g_gf, g_ms = sum_stats(stats, "rsvt_gemm_gflop"), sum_stats(stats, "rsvt_gemm_ms")
    s_gf, s_ms = sum_stats(stats, "rsvt_svd_gflop"), sum_stats(stats, "rsvt_svd_ms")
    peak = alu_peak(peaks)
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * TF32_PER_BF16
    svd_tf = s_gf / max(s_ms, 1e-9)      # GFLOP / ms = TFLOP/s
    gemm_tf = g_gf / max(g_ms, 1e-9)
    roof_svd = {"bound": "alu", "kernel": "jacobi_svt_kernel (n x k projections)",
                "achieved": svd_tf, "peak": peak, "unit": "TFLOP/s", "frac": svd_tf / peak,
                "traffic": None,
                "peak_source": peaks["fp32_source"],
                "alg": "Golub-Van Loan 4 (4 n k^2 + 8 k^3) per n x k projection",
                "ms": s_ms}
    if prec_name == "rand_fp32":
        roof_gemm = {"bound": "alu", "kernel": "cgemm_fp32_kernel", "achieved": gemm_tf,
                     "peak": peak, "unit": "TFLOP/s", "frac": gemm_tf / peak, "traffic": None,
                     "peak_source": peaks["fp32_source"],
                     "alg": "8 m n k per complex product", "ms": g_ms}
    else:
        roof_gemm = {"bound": "tensor", "kernel": f"cgemm_tc_kernel ({prec_name})",
                     "achieved": gemm_tf, "peak": tf32_peak, "unit": "TFLOP/s",
                     "frac": gemm_tf / tf32_peak, "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 1.1/2.25",
                     "alg": "8 m n k per complex product; executed tensor flops per algorithmic "
                            f"flop {EXECUTED_PER_ALG.get(prec_name, 0)}",
                     "ms": g_ms}
    return roof_svd, roof_gemm


def instrumented_pass(dw, iters, prec_name, stream, flush, barrier, steps, cache):
    """The same solves in a context that brackets every slice-SVT, tube-pass and mixed-form
    stage launch with CUDA events (the per-kernel device times); the events cost the GPU a
    short drain per record, so the throughput figures come from an uninstrumented region."""
    from paper_1407_1785_gb300 import libtsvd
    ctx = libtsvd.Context(device=stream.device.index, stream=stream.cuda_stream, timing=1,
                          precision=PRECISIONS[prec_name], autotune_cache=cache, **ctx_options(dw))
    solve = solver(ctx, dw, iters)
    solve()                                                # warm-up (plan from the cache)
    t_ms, stats = timed_solves(solve, steps, flush, stream, barrier)
    ctx.close()
    return t_ms, stats


FP32_RSE_FLOOR = 1e-4   # recovery error an FP32 solve keeps where the exact answer is recovered


def equal_error_verdict(e_mixed, e_plain):
    """The equal-error rule per tensor: e_mixed <= e_plain + 0.01 e_plain + 1e-5, or both at or
    below the FP32 floor of an exact recovery (1e-4; there both errors are FP32 rounding of a
    solution the FP64 oracle recovers to ~1e-15, and which of the two rounds lower is noise)."""
    ok = [em <= ep + 0.01 * ep + 1e-5 or max(em, ep) <= FP32_RSE_FLOOR
          for em, ep in zip(e_mixed, e_plain)]
    worst = max(range(len(ok)), key=lambda i: e_mixed[i] / max(e_plain[i], 1e-300))
    return {"equal_error": all(ok), "tensors_meeting": int(sum(ok)), "tensors": len(ok),
            "missing": [i for i, v in enumerate(ok) if not v],
            "worst_ratio": e_mixed[worst] / max(e_plain[worst], 1e-300), "worst_tensor": worst}


def mixed_form(args, dw, iters, prec_name, e_plain, stream, flush, barrier, peaks, t_plain_ms,
               cache, steps=None):
    """Times the mixed form on the same workload; returns the "mixed" object.  e_plain: the
    plain form's recovery error of every tensor."""
    from paper_1407_1785_gb300 import libtsvd
    steps = steps or args.steps
    ctx = libtsvd.Context(device=stream.device.index, stream=stream.cuda_stream,
                          precision=PRECISIONS[prec_name], autotune_cache=cache, **ctx_options(dw))
    solve = solver(ctx, dw, iters)
    for _ in range(max(args.warmup, 1)):
        solve()
    t_ms, tstats = timed_solves(solve, steps, flush, stream, barrier)
    ctx.close()
    errs = recovery_errors(dw)
    verdict = equal_error_verdict(errs, e_plain)
    out = {
        "precision": prec_name, "value": iters * steps / (t_ms / 1000.0),
        "unit": "iters/s", "ms_per_step": t_ms / steps, "steps": steps,
        "speedup_vs_plain": t_plain_ms / t_ms,
        "final_rse_db": 20 * math.log10(statistics.mean(errs)),
        "plain_rse_db": 20 * math.log10(statistics.mean(e_plain)),
        # equal error: not worse than the plain form's recovery error beyond 1% (+1e-5), or
        # both at the FP32 floor of an exact recovery, for every tensor
        **verdict,
        "sketch_width_last": tstats[-1]["rsvt_k_last"],
        "saturated_slice_svts": tstats[-1]["rsvt_saturated"],
        "gpu_launches": sum_stats(tstats, "launches"),
    }
    if dw["kind"] == "batch":
        out["final_rse_db_per_tensor"] = [round(20 * math.log10(max(e, 1e-300)), 3) for e in errs]
        # the batched form records no per-stage events: the algorithmic work of the products
        # and of the small SVDs (from the device-chosen widths) over the wall time of a whole
        # solve, i.e. lower bounds of each stage's own rate
        solve_ms = t_ms / steps
        g_tf = tstats[-1]["rsvt_gemm_gflop"] / solve_ms      # GFLOP / ms = TFLOP/s
        s_tf = tstats[-1]["rsvt_svd_gflop"] / solve_ms
        tf32_peak = peaks.get("bf16_tflops", 1900.0) * TF32_PER_BF16
        out["roofline_products_wall"] = {
            "bound": "tensor", "kernel": f"cgemm_tc_kernel ({prec_name})", "achieved": g_tf,
            "peak": tf32_peak, "unit": "TFLOP/s", "frac": g_tf / tf32_peak, "traffic": None,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 1.1/2.25",
            "alg": "8 m n k per complex product, 3 products per slice and iteration",
            "gflop_per_solve": tstats[-1]["rsvt_gemm_gflop"],
            "times_from": "wall time of whole solves (all stages): a lower bound"}
        out["roofline_small_svd_wall"] = {
            "bound": "alu", "kernel": "eig_svt_kernel (k x k Grams)", "achieved": s_tf,
            "peak": alu_peak(peaks), "unit": "TFLOP/s", "frac": s_tf / alu_peak(peaks),
            "traffic": None, "peak_source": peaks["fp32_source"],
            "alg": "Golub-Van Loan 4 (4 n k^2 + 8 k^3) per n x k projection",
            "gflop_per_solve": tstats[-1]["rsvt_svd_gflop"],
            "times_from": "wall time of whole solves (all stages): a lower bound"}
        return out
    tp_ms, stats = instrumented_pass(dw, iters, prec_name, stream, flush, barrier, steps, cache)
    n_it = iters * steps
    parts = {"small_svd": sum_stats(stats, "rsvt_svd_ms"),
             "slice_products": sum_stats(stats, "rsvt_gemm_ms"),
             "cholqr2": sum_stats(stats, "rsvt_orth_ms"),
             "tube_pass": sum_stats(stats, "tube_ms")}
    parts["other"] = max(tp_ms - sum(parts.values()), 0.0)
    roof_svd, roof_gemm = mixed_rooflines(stats, prec_name, peaks)
    out.update({
        "ms_per_iter": {k: v / n_it for k, v in parts.items()},
        "dominant": max(("small_svd", "slice_products", "cholqr2", "tube_pass"), key=parts.get),
        "roofline_small_svd": roof_svd,
        "roofline_slice_products": roof_gemm,
        "stage_times_from": "instrumented pass of the same solves (CUDA events per stage)",
    })
    return out


def side_workload(args, name, stream, flush, barrier, peaks, cache, steps):
    """Plain and mixed form of another workload on the same GPU, timed like the headline
    (inputs resident, L2 flushed between solves); returns its summary object."""
    from paper_1407_1785_gb300 import libtsvd
    spec = WORKLOADS[name]
    iters = spec["iters"]
    wl = build_workload(name, 1)
    dw = to_device(wl)
    ctx = libtsvd.Context(device=stream.device.index, stream=stream.cuda_stream,
                          precision=PRECISIONS["fp32"], autotune_cache=cache, **ctx_options(wl))
    solve = solver(ctx, dw, iters)
    for _ in range(max(args.warmup, 1)):
        solve()
    t_ms, stats = timed_solves(solve, steps, flush, stream, barrier)
    ctx.close()
    errs = recovery_errors(dw)
    out = {"workload": spec["desc"], "admm_iters_per_step": iters, "steps": steps,
           "plain": {"value": iters * steps / (t_ms / 1000.0), "unit": "iters/s",
                     "ms_per_step": t_ms / steps, "final_rse_db": 20 * math.log10(errs[0]),
                     "jacobi_sweeps_per_slice_svd": (sum_stats(stats, "total_sweeps") /
                                                     max(sum_stats(stats, "slice_svds"), 1))}}
    if args.mixed not in ("none", "fp32"):
        out["mixed"] = mixed_form(args, dw, iters, args.mixed, errs, stream, flush, barrier,
                                  peaks, t_ms, cache, steps=steps)
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1407_1785_gb300 import libtsvd, synth

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    spec = WORKLOADS[args.workload]
    iters = args.iters or spec["iters"]
    batch = spec["kind"] == "batch"
    # single tensors: every rank solves its own replica (seed 1 + rank); the batch: one batch,
    # its tensors split over the ranks (no collective on the data path)
    wl = build_workload(args.workload, 1 if batch else 1 + rank)
    n_per_iter = n_voxels(wl)      # voxels of one iteration: one replica, or the whole batch
    if batch and world > 1:
        mine = lpt_shard([tensor_cost(it["dims"]) for it in wl["items"]], world)[rank]
        wl = dict(kind="batch", items=[wl["items"][i] for i in mine])
    items = wl["items"] if batch else [wl]
    N = n_voxels(wl)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        v, dt, what = oracle_sample(wl, args.cpu_sample_iters or spec["cpu_iters"])
        cpu = {"value": v, "unit": "iters/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": what, "seconds": dt}

    stream = torch.cuda.current_stream()
    dw = to_device(wl)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    prec = args.precision
    # the timed context and the instrumented one share the autotuned plans
    cache = os.path.join(tempfile.mkdtemp(prefix="tsvd_tune_"), "plans.txt").encode()
    ctx = libtsvd.Context(device=local, stream=stream.cuda_stream,
                          precision=PRECISIONS[prec], autotune_cache=cache, **ctx_options(wl))
    solve = solver(ctx, dw, iters)
    for _ in range(max(args.warmup, 0)):
        solve()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    t_ms, stats = timed_solves(solve, args.steps, flush, stream, barrier)
    clocks = sampler.stop()
    t_ms = max_over_ranks(t_ms)
    # replicas: the ranks' iterations add up; the sharded batch: one batch iteration spans them
    units = 1 if batch else world
    value = units * iters * args.steps / (t_ms / 1000.0)
    errs = recovery_errors(dw)
    launches = sum_stats(stats, "launches")
    # per-kernel device times from an instrumented pass of the same solves (fewer steps: the
    # per-launch events only split the time, the throughput comes from the region above)
    isteps = min(args.steps, 5)
    tp_ms, pstats = instrumented_pass(dw, iters, prec, stream, flush, barrier, isteps, cache)
    slice_ms, tube_ms = sum_stats(pstats, "slice_ms"), sum_stats(pstats, "tube_ms")
    slice_launches = sum_stats(pstats, "slice_launches")

    # end to end through the public API from pinned host buffers, copies inside the region
    ctx_e2e = None
    if batch:
        hin = [(torch.from_numpy(synth.to_colmajor(it["M"])).pin_memory(),
                torch.from_numpy(synth.to_colmajor(it["omega"], np.uint8)).pin_memory()
                if it["kind"] == "complete" else None) for it in items]
        hout = [torch.empty(it["m"].numel(), dtype=torch.float32).pin_memory()
                for it in dw["items"]]

        def e2e_step():
            for (mh, oh), it in zip(hin, dw["items"]):
                it["m"].copy_(mh, non_blocking=True)
                if oh is not None:
                    it["o"].copy_(oh, non_blocking=True)
            solve()
            for xh, it in zip(hout, dw["items"]):
                xh.copy_(it["out0"], non_blocking=True)
            torch.cuda.synchronize()
        h2d = sum(mh.numel() * 4 + (oh.numel() if oh is not None else 0) for mh, oh in hin)
        d2h = sum(xh.numel() * 4 for xh in hout)
    else:
        mh = torch.from_numpy(synth.to_colmajor(wl["M"])).pin_memory()
        xh = torch.empty(N, dtype=torch.float32).pin_memory()
        ctx_e2e = libtsvd.Context(device=local, stream=stream.cuda_stream,
                                  precision=PRECISIONS[prec], **ctx_options(wl))
        dims = wl["dims"]
        if wl["kind"] == "complete":
            oh = torch.from_numpy(synth.to_colmajor(wl["omega"], np.uint8)).pin_memory()

            def e2e_step():
                ctx_e2e.tnn_complete(mh, oh, dims, iters, xh)   # returns after the D2H copy
            h2d, d2h = mh.numel() * 4 + oh.numel(), xh.numel() * 4
        else:
            sh = torch.empty(N, dtype=torch.float32).pin_memory()

            def e2e_step():
                ctx_e2e.trpca(mh, dims, wl["lam"], iters, xh, sh)
            h2d, d2h = mh.numel() * 4, 2 * xh.numel() * 4
    e2e_step()                                             # warm-up (workspace)
    barrier()
    esteps = min(args.steps, 5)
    t0 = time.perf_counter()
    for _ in range(esteps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": units * iters * esteps / e2e_s, "unit": "iters/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": esteps}

    peaks = add_fp32_peak(measured_peaks(), local)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    n_it = iters * isteps
    if prec == "fp32" and batch:
        # the tensors' chains overlap on stream branches, so per-launch events do not add up
        # to device time: the achieved rate is the algorithmic flops of all slice SVDs of one
        # batch iteration over the wall time of one batch iteration of the timed region (tube
        # passes and warm-start products included, so a lower bound on the kernel's)
        flops = sum(jacobi_gvl_flops(it["dims"][0], it["dims"][1], half_slices(it["dims"]))
                    for it in items)
        it_s = t_ms / 1000.0 / (iters * args.steps)
        achieved = flops / it_s / 1e12
        roofline = {"bound": "alu", "kernel": "batched plain solve (jacobi_svt_kernel, tube "
                    "passes, warm-start products)", "achieved": achieved,
                    "peak": alu_peak(peaks), "unit": "TFLOP/s",
                    "frac": achieved / alu_peak(peaks), "traffic": None,
                    "peak_source": peaks["fp32_source"],
                    "alg_flops_per_iteration": flops, "ms_per_batch_iteration": it_s * 1e3,
                    "times_from": "wall time of the timed region (CUDA events on the stream)"}
    elif prec == "fp32":
        # algorithmic flops of one iteration (all tensors), per-iteration slice time
        flops = sum(jacobi_gvl_flops(it["dims"][0], it["dims"][1], half_slices(it["dims"]))
                    for it in items)
        achieved = flops / (slice_ms / 1000.0 / n_it) / 1e12
        roofline = {"bound": "alu", "kernel": "jacobi_svt_kernel", "achieved": achieved,
                    "peak": alu_peak(peaks), "unit": "TFLOP/s",
                    "frac": achieved / alu_peak(peaks), "traffic": None,
                    "peak_source": peaks["fp32_source"],
                    "alg_flops_per_iteration": flops,
                    "avg_launch_ms": slice_ms / max(slice_launches, 1),
                    "share_of_step": slice_ms / tp_ms,
                    "times_from": "instrumented pass of the same solves (CUDA events per launch)"}
    else:
        roof_svd, roof_gemm = mixed_rooflines(pstats, prec, peaks)
        roofline = roof_svd if roof_svd["ms"] >= roof_gemm["ms"] else roof_gemm
    t_bytes = sum(tube_bytes(it["dims"]) for it in items)
    roofline_tube = None
    if tube_ms > 0 and not batch:
        gbs = t_bytes * n_it / (tube_ms / 1000.0) / 1e9
        roofline_tube = {"bound": "hbm", "kernel": "tube_pass_kernel", "achieved": gbs,
                         "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                         "peak_source": ("MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks
                                         else "fallback"),
                         "alg_bytes_per_iteration": t_bytes, "ms_per_iteration": tube_ms / n_it,
                         "traffic": tube_traffic(args.workload)}

    mixed = None
    if prec == "fp32" and args.mixed not in ("none", "fp32"):
        mixed = mixed_form(args, dw, iters, args.mixed, errs, stream, flush, barrier, peaks,
                           t_ms, cache)
    color = None
    if batch and world == 1 and not args.no_color:
        # the largest single tensor (288x352x3x60 colour video), plain and mixed, alongside
        color = side_workload(args, "color", stream, flush, barrier, peaks, cache,
                              steps=min(args.steps, 3))

    e_db = [20 * math.log10(max(e, 1e-300)) for e in errs]
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": spec["desc"], "admm_iters_per_step": iters, "seed": 1,
                   "precision": prec, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "voxels_per_s": value * n_per_iter,
        "final_rse_db": e_db[0] if not batch else statistics.mean(e_db),
        "roofline": roofline,
        "roofline_tube": roofline_tube,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if batch:
        line["final_rse_db_max"] = max(e_db)
        line["final_rse_db_per_tensor"] = [round(v, 3) for v in e_db]
    if prec == "fp32":
        line["jacobi_sweeps_per_slice_svd"] = (sum_stats(stats, "total_sweeps") /
                                               max(sum_stats(stats, "slice_svds"), 1))
        line["jacobi_nonconverged"] = sum_stats(stats, "nonconverged")
        line["slice_plan"] = {"ctas_per_slice": stats[-1]["slice_ctas"],
                              "lanes_per_pair": stats[-1]["slice_lanes"],
                              "pairs_in_flight": stats[-1]["slice_pairs_in_flight"]}
    else:
        line["sketch_width_last"] = stats[-1]["rsvt_k_last"]
        line["ms_per_iter"] = {"small_svd": sum_stats(pstats, "rsvt_svd_ms") / n_it,
                               "slice_products": sum_stats(pstats, "rsvt_gemm_ms") / n_it,
                               "cholqr2": sum_stats(pstats, "rsvt_orth_ms") / n_it,
                               "tube_pass": tube_ms / n_it}
    if mixed is not None:
        line["mixed"] = mixed
    if color is not None:
        line["color"] = color
    ctx.close()
    if ctx_e2e is not None:
        ctx_e2e.close()
    shutil.rmtree(os.path.dirname(cache.decode()), ignore_errors=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def factor_input(seed):
    from paper_1407_1785_gb300 import synth
    X, _ = synth.workload_video_completion(seed=seed)
    return X.astype(np.float32)


def run_factor(args, reference=False):
    """The t-SVD export: one step = one economy t-SVD (tsvd_factor, k = min(n1, n2)) of the
    144x176x100 video; value = factorisations per second.  The reference arm times the FP64
    oracle's full t-SVD of the same tensor."""
    import torch
    import torch.distributed as dist
    from paper_1407_1785_gb300 import libtsvd, synth
    rank, world, local = dist_info()
    spec = WORKLOADS["factor"]
    if reference:
        spec = WORKLOADS[args.workload]
        unit = "factorizations/s" if args.workload == "factor" else "compressions/s"
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        Y = factor_input(1).astype(np.float64)
        for _ in range(args.warmup):
            oracle.tsvd(Y)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.tsvd(Y)
        dt = time.perf_counter() - t0
        v = args.steps / dt
        cpu = {"value": v, "unit": unit, "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "full t-SVD of the same tensor per step (FP64 C oracle)"}
        print(json.dumps({"metric": METRIC, "impl": "reference", "value": v,
                          "unit": unit, "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": spec["desc"]}, "cpu_baseline": cpu,
                          "e2e": {"value": v, "unit": unit,
                                  "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return 0
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    Y = factor_input(1 + rank)
    dims = Y.shape
    n1, n2, n3 = dims
    k = min(n1, n2)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.tsvd(Y.astype(np.float64))
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "factorizations/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "one full t-SVD of the same tensor (FP64 C oracle)",
               "seconds": dt}
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    y = torch.from_numpy(synth.to_colmajor(Y)).cuda()
    U = torch.empty(n1 * k * n3, device="cuda")
    S = torch.empty(k * k * n3, device="cuda")
    V = torch.empty(n2 * k * n3, device="cuda")
    ctx = libtsvd.Context(device=local, stream=stream.cuda_stream)
    for _ in range(max(args.warmup, 1)):
        ctx.factor(y, dims, 0, U, S, V)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t_ms, _ = timed_solves(lambda: ctx.factor(y, dims, 0, U, S, V), args.steps, flush, stream,
                           barrier)
    clocks = sampler.stop()
    t_ms = max_over_ranks(t_ms)
    value = world * args.steps / (t_ms / 1000.0)
    # reconstruction U * S * V^T through the Fourier domain (numpy), relative to Y
    Uh = np.fft.fft(synth.from_colmajor(U.cpu().numpy(), (n1, k, n3)).astype(np.float64), axis=2)
    Sh = np.fft.fft(synth.from_colmajor(S.cpu().numpy(), (k, k, n3)).astype(np.float64), axis=2)
    Vh = np.fft.fft(synth.from_colmajor(V.cpu().numpy(), (n2, k, n3)).astype(np.float64), axis=2)
    Rh = np.moveaxis(Uh, 2, 0) @ np.moveaxis(Sh, 2, 0) @ np.conj(np.moveaxis(Vh, 2, 0)).transpose(0, 2, 1)
    R = np.real(np.fft.ifft(np.moveaxis(Rh, 0, 2), axis=2))
    rec = float(np.linalg.norm(R - Y) / np.linalg.norm(Y))
    # end to end from pinned host buffers (the library stages them)
    yh = torch.from_numpy(synth.to_colmajor(Y)).pin_memory()
    uh, sh, vh = (torch.empty(x.numel()).pin_memory() for x in (U, S, V))
    ctx.factor(yh, dims, 0, uh, sh, vh)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.factor(yh, dims, 0, uh, sh, vh)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    ctx.close()
    peaks = add_fp32_peak(measured_peaks(), local)
    flops = jacobi_gvl_flops(n1, n2, half_slices(dims))
    achieved = flops / (t_ms / 1000.0 / args.steps) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "factorizations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": spec["desc"], "seed": 1, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "reconstruction_rel_err": rec,
        "roofline": {"bound": "alu", "kernel": "jacobi_svt_kernel", "achieved": achieved,
                     "peak": alu_peak(peaks), "unit": "TFLOP/s", "frac": achieved / alu_peak(peaks),
                     "traffic": None,
                     "peak_source": peaks["fp32_source"],
                     "alg_flops_per_call": flops,
                     "times_from": "whole call (forward pass, slice SVDs in the V form, factor "
                                   "assembly, three inverse passes), CUDA events"},
        "cpu_baseline": cpu,
        "e2e": {"value": world * args.steps / e2e_s, "unit": "factorizations/s",
                "h2d_bytes_per_step": int(yh.numel() * 4),
                "d2h_bytes_per_step": int((uh.numel() + sh.numel() + vh.numel()) * 4)},
        "gpu_launches": 6 * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_compress(args):
    """t-SVD compression of the video: one step = one Method 1 compression at k2 = 10 n3 (ratio
    ~9); the line also carries the RSE-against-ratio curve of both methods (k3 tubes for
    Method 2, k2 = k3 n3 entries for Method 1: the same ratio)."""
    import torch
    import torch.distributed as dist
    from paper_1407_1785_gb300 import libtsvd, synth
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    spec = WORKLOADS["compress"]
    Y = factor_input(1 + rank)
    n1, n2, n3 = Y.shape
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.tsvd(Y.astype(np.float64))
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "compressions/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "the full t-SVD both methods truncate, same tensor "
                                           "(FP64 C oracle)", "seconds": dt}
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    y = torch.from_numpy(synth.to_colmajor(Y)).cuda()
    z = torch.empty_like(y)
    ctx = libtsvd.Context(device=local, stream=stream.cuda_stream)
    nrm = float(np.linalg.norm(Y))
    curve = []
    for k3 in (1, 2, 5, 10, 20, 40):
        for method, k, name in ((libtsvd.COMPRESS_TUBAL, k3, "t-SVD-tubal (Method 2)"),
                                (libtsvd.COMPRESS_GLOBAL, k3 * n3, "t-SVD (Method 1)")):
            kept, ratio = ctx.compress(y, Y.shape, method, k, z)
            R = synth.from_colmajor(z.cpu().numpy(), Y.shape)
            rse = float(np.linalg.norm(R - Y) / nrm)
            curve.append({"method": name, "k": int(k), "kept": int(kept), "ratio": ratio,
                          "rse_db": 20 * math.log10(max(rse, 1e-300))})
    k2 = 10 * n3

    def step():
        ctx.compress(y, Y.shape, libtsvd.COMPRESS_GLOBAL, k2, z)
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t_ms, _ = timed_solves(step, args.steps, flush, stream, barrier)
    clocks = sampler.stop()
    t_ms = max_over_ranks(t_ms)
    yh = torch.from_numpy(synth.to_colmajor(Y)).pin_memory()
    zh = torch.empty(yh.numel()).pin_memory()
    ctx.compress(yh, Y.shape, libtsvd.COMPRESS_GLOBAL, k2, zh)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.compress(yh, Y.shape, libtsvd.COMPRESS_GLOBAL, k2, zh)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    ctx.close()
    peaks = add_fp32_peak(measured_peaks(), local)
    flops = jacobi_gvl_flops(n1, n2, half_slices(Y.shape))
    achieved = flops / (t_ms / 1000.0 / args.steps) / 1e12
    line = {
        "metric": METRIC, "value": world * args.steps / (t_ms / 1000.0), "unit": "compressions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": spec["desc"], "seed": 1, "method_timed": "Method 1, k2 = 10 n3",
                   "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "curve": curve,
        "roofline": {"bound": "alu", "kernel": "jacobi_svt_kernel", "achieved": achieved,
                     "peak": alu_peak(peaks), "unit": "TFLOP/s", "frac": achieved / alu_peak(peaks),
                     "traffic": None,
                     "peak_source": peaks["fp32_source"],
                     "alg_flops_per_call": flops,
                     "times_from": "whole call (forward pass, slice SVDs, singular values to the "
                                   "host, rebuild, inverse pass), CUDA events"},
        "cpu_baseline": cpu,
        "e2e": {"value": world * args.steps / e2e_s, "unit": "compressions/s",
                "h2d_bytes_per_step": int(yh.numel() * 4), "d2h_bytes_per_step": int(zh.numel() * 4)},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    global NO_GRAPHS
    args = parse_args()
    NO_GRAPHS = args.no_graphs
    if args.workload == "compress" and args.impl != "reference":
        return run_compress(args)
    if args.workload in ("factor", "compress"):
        return run_factor(args, reference=args.impl == "reference")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
