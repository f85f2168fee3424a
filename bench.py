"""Benchmark: walker-steps/s of phaseless AFQMC at M=300 on GB300.

Workload (the M=300 configuration): synthetic closed-shell Hamiltonian with
M=300 orbitals, N_up=N_dn=25, 1800 Cholesky vectors, 512 walkers, dt=0.005,
modified Gram-Schmidt every 5 steps, local energy every 10 steps.  One step
is one pass of the whole hot path over all walkers (force bias, fields, V,
propagation, overlap/LU, weights, and the periodic QR and energy).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|tf32|fp64|bf16-f32lu|tf32-f32lu]
    python bench.py --impl reference      # the CPU oracle on the host cores
    python bench.py --workload mcd [--config c2] [--impl reference]
        # modified Cholesky decomposition (Sec. 2.3) of the workload's
        # interaction over index pairs: Cholesky vectors per second

The default is the mixed path with BF16 tensor-core operands (the M=300
configuration's precision); the line also carries the same workload's FP64
path measured on the same GPU (a few steps) and the mixed path's energy bias
against it on identical walkers and fields.

Prints one JSON line.  Under torchrun (N > 1) the ranks hold one population
of N x 512 walkers, 512 per GPU (paper_1711_02242_gb300.dist): each rank
steps its share, the mixed estimator is summed over the ranks and, with
--pc-period, the comb spans all ranks (walkers move between GPUs).  Time is
the max over ranks and the value the walker-steps of all ranks per second
(weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

PHASES = ["force_bias", "fields", "v_assembly", "bhalf", "taylor", "overlap", "weight", "qr",
          "comb", "energy", "theta"]

# --precision -> afqmc_params.precision.  "bf16" / "tf32" keep S^-1 (the LU),
# log det, the overlap ratios, the weights and Gram-Schmidt in float64 and form
# Theta = Phi S^-1 in FP32; "-f64theta" forms Theta in float64 too; the
# "-f32lu" variants (opt-in) run the elimination and Gram-Schmidt in FP32.
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16": 2, "tf32-f32lu": 3, "bf16-f32lu": 4,
              "tf32-f64theta": 5, "bf16-f64theta": 6}
DTYPES = {"fp64": "f64", "tf32": "tf32/f32/f64", "bf16": "bf16/f32/f64",
          "tf32-f32lu": "tf32/f32/f64", "bf16-f32lu": "bf16/f32/f64",
          "tf32-f64theta": "tf32/f32/f64", "bf16-f64theta": "bf16/f32/f64"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 peak of GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA per
# clock x 2 FLOP x 2070 MHz = 1.259 TFLOP/s (a DFMA probe kernel measured
# 1.198 TFLOP/s on this machine, i.e. 2 FMA/clk/SM at the clock under load).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 likewise: 152 SMs x 128 FMA per clock x 2 FLOP x 2070 MHz = 80.5 TFLOP/s.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12

# DRAM bytes (read + write) per launch from one ncu capture of the M=300 step
# (energy: the exchange contraction, the phase's main kernel), with the SHA-256
# of the source file the kernel was built from and the precisions whose step
# runs that kernel; a figure whose source has changed since, or that belongs
# to another kernel at this precision, is reported as null.
GEMM_KERNEL = "__device__ __forceinline__ void gemm_body("
TRAFFIC = {
    "theta": [# k_theta_rows_f32 on the float64 S^-1 (the bf16 default path)
              {"bytes": (66.846720 + 26.307840) * 1e6, "precisions": ("bf16",),
               "function": "__global__ void __launch_bounds__(TH_T) k_theta_rows_f32(OverlapArgs a)",
               "sha": "95b521175a189697f17637210e88c7be80b91f899d89ffb387d05b3e718d9736"},
              # k_theta_rows (float64 Theta of the -f64theta mixed paths): its own
              # text is unchanged since this capture (DRAM 64.5 + 30.3 MB per launch)
              {"bytes": (64.544512 + 30.260480) * 1e6, "precisions": ("bf16-f64theta",),
               "function": "__global__ void __launch_bounds__(TH_T) k_theta_rows(OverlapArgs a)",
               "sha": "d7ee3083bab22e614e7aa9c51aff2886d255680c62a6454f637a089a17969ae7"}],
    # k_overlap<double> and k_mgs (float64, the bf16 default path), pinned to
    # their own text (captures in profiles/overlap_inverse_m300_bf16.md and
    # profiles/mgs_m300_bf16.md)
    "overlap": {"bytes": (8.244992 + 0.0) * 1e6, "precisions": ("bf16",),
                "function": "__global__ void __launch_bounds__(OV_T) k_overlap(OverlapArgs a)",
                "sha": "5905df615412e8d5881361e99808acd80656d2a0414eef96dd142e0f6e82e0bc"},
    "qr": {"bytes": (61.483264 + 34.291200) * 1e6, "precisions": ("bf16",),
           "function": "__global__ void __launch_bounds__(256) k_mgs(MgsArgs a)",
           "sha": "4e08b7f77fcd6fee61eeb48c18f47fe8220b9dacfe0af8c3a22f28d76f55f22f"},
    # the tensor-core kernels: pinned to the kernel's text (and its epilogue's),
    # unchanged since these captures (only their host launchers changed)
    "taylor": {"bytes": (218.472704 + 19.613440) * 1e6, "precisions": ("bf16", "bf16-f32lu", "bf16-f64theta"),
               "function": "__global__ void __launch_bounds__(kSeriesThreads, 1)",
               "sha": "e47766a88bc3d88a860c2cac6a6bb846bd1349fc46fd391771607944c29a3feb"},
    # the V contraction in the form the set-up chooses at M=300 (BN = 256 on
    # 128-row tiles, CTA pairs)
    "v_assembly": {"bytes": (183.425536 + 146.092288) * 1e6, "precisions": ("bf16", "bf16-f32lu", "bf16-f64theta"),
                   "function": [GEMM_KERNEL, "struct EpiVT {"],
                   "sha": "b34ba031fd47ee240c8c32d916b8c0c9eaed95718863e675b9597e6ba39dd815"},
    "energy": {"bytes": (42.981120 + 0.896512) * 1e6, "precisions": ("bf16", "bf16-f32lu", "bf16-f64theta"),
               "function": [GEMM_KERNEL, "struct EpiExchange {"],
               "sha": "a34fa5e7f96ce4c61663388be5935414dd273ca610993974abba5e0154a4a6d8"},
}


def pinned_copy(torch, a):
    """A float64 copy of the host array a in page-locked memory (a numpy view)."""
    a = np.ascontiguousarray(a, np.float64)
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t.numpy()


class ClockSampler:
    """nvidia-smi clock / throttle samples taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device="cpu") -> float:
    """The slowest rank's time (the job's time), via all_reduce(MAX)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


L2_BYTES = 129e6  # GB300 L2


def l2_note(w: workloads.Workload) -> str:
    """How the timed steps stand against L2: the packed Cholesky vectors and the
    walkers' orbitals are read every step; no flush between steps."""
    L_bytes = w.M * (w.M + 1) // 2 * w.nchol * 8
    phi_bytes = w.nwalkers * 2 * w.N * w.M * 8
    if L_bytes > L2_BYTES:
        return f"inputs larger than L2 (packed L {L_bytes / 1e6:.0f} MB float64)"
    size = lambda n: f"{n / 1e6:.1f} MB" if n >= 1e6 else f"{n / 1e3:.0f} KB"  # noqa: E731
    return (f"inputs fit in L2 (packed L {size(L_bytes)}, orbitals {size(phi_bytes)} float64): "
            "L2-resident steps, no flush")


def job_throughput(walkers_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Walker-steps of all ranks per second of the slowest rank."""
    return world * walkers_per_rank * steps / (ms_max * 1e-3)


def algorithmic_per_walker(w: workloads.Workload):
    """Algorithmic work of the step's kernels per walker (one spin block; the
    closed-shell walker's two blocks are the same matrix), as used for the
    roofline fractions:
      overlap  FP64: Gauss-Jordan inverse of S, 8 N^3 (in the trial-adapted
               basis S is the top block of Phi);
      theta    FP64: Theta's M - N non-trivial rows, 8 (M - N) N^2 (the top
               N rows are I);
      qr       FP64: modified Gram-Schmidt, 8 M N^2, every qr_period steps;
      v        tensor: V = sum_g x_g L_g over the M (M + 1) / 2 distinct
               elements, complex x real: 2 N_g M (M + 1);
      taylor   tensor: n products of complex M x M by M x N, 8 n M^2 N;
      energy   tensor: force bias 4 N_g N M and exchange 4 N_g N^2 M (the
               T_g = Lh_g Theta products), per evaluation."""
    M, N, G, n = w.M, w.N, w.nchol, w.taylor_order
    return {"overlap": 8 * N ** 3, "theta": 8 * (M - N) * N * N, "qr": 8 * M * N * N,
            "v_assembly": 2 * G * M * (M + 1), "taylor": 8 * n * M * M * N,
            "energy": 4 * G * N * M + 4 * G * N * N * M}


def bytes_per_walker(w: workloads.Workload, precision):
    """Algorithmic DRAM bytes per walker of the mixed path's FP32 kernels,
    which are bound by memory traffic, not by their FP32 arithmetic:
      theta  read Phi (2 N M float64) and S^-1 (N^2 complex: float64, or FP32
             on the -f32lu paths), write Theta (2 N M float64) and its
             BF16/TF32 copy (2 N Mp);
      qr     read and write Phi (2 x 2 N M float64), write its BF16/TF32 copy."""
    M, N = w.M, w.N
    Mp = (M + 15) // 16 * 16
    lo = 2 if precision.startswith("bf16") else 4
    sinv = 8 if precision.endswith("f32lu") else 16
    return {"theta": 2 * N * M * 8 + N * N * sinv + 2 * N * M * 8 + 2 * N * Mp * lo,
            "qr": 2 * (2 * N * M * 8) + 2 * N * Mp * lo}


def kernel_of_phase(precision):
    """Phase -> (kernel, bound, source file).  The elimination and the
    Gram-Schmidt sweep are FP64-pipe kernels on the float64 path and the
    bf16 / tf32 mixed paths, and so is Theta = Phi S^-1 on the float64 path
    and the -f64theta mixed paths; the bf16 / tf32 paths form Theta in FP32
    (against HBM), and the -f32lu paths also run the elimination (against the
    FP32 pipe) and the sweep (against HBM) in FP32."""
    k = dict(KERNEL_OF_PHASE)
    if precision in ("bf16", "tf32") or precision.endswith("f32lu"):
        k["theta"] = ("k_theta_rows_f32", "hbm", "walker_f64.cu")
    if precision.endswith("f32lu"):
        k["overlap"] = ("k_overlap<float>", "alu32", "walker_f64.cu")
        k["qr"] = ("k_mgs_f32", "hbm", "walker_f64.cu")
    return k


KERNEL_OF_PHASE = {"overlap": ("k_overlap", "alu", "walker_f64.cu"),
                   "theta": ("k_theta_rows", "alu", "walker_f64.cu"),
                   "qr": ("k_mgs", "alu", "walker_f64.cu"),
                   "v_assembly": ("tcgen05 V contraction (EpiV)", "tensor", "gemm_tc.cu"),
                   "taylor": ("k_taylor_series", "tensor", "taylor_tc.cu"),
                   "energy": ("force bias + tcgen05 exchange (EpiExchange) + k_eloc", "tensor",
                              "gemm_tc.cu")}


def source_sha(fname):
    import hashlib

    path = os.path.join(ROOT, "paper_1711_02242_gb300", "csrc", fname)
    try:
        with open(path, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None


def function_sha(fname, signature):
    """SHA-256 of one function's text (from `signature` to its closing brace)
    in a CUDA source file: a capture stays valid while that kernel's own source
    is unchanged, whatever else the file holds."""
    import hashlib

    path = os.path.join(ROOT, "paper_1711_02242_gb300", "csrc", fname)
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    i = text.find(signature)
    if i < 0:
        return None
    depth, j = 0, text.find("{", i)
    for k in range(j, len(text)):
        if text[k] == "{":
            depth += 1
        elif text[k] == "}":
            depth -= 1
            if depth == 0:
                return hashlib.sha256(text[i:k + 1].encode()).hexdigest()
    return None


def traffic_of(phase, src, precision):
    """The recorded DRAM bytes of a phase's kernel at this precision, if its
    source (the file, or the text of the kernel and of the device code it
    names, for entries that list them) is the one the counters were taken
    from."""
    import hashlib

    entries = TRAFFIC.get(phase)
    if not entries:
        return None
    for tr in entries if isinstance(entries, list) else [entries]:
        if precision not in tr.get("precisions", ("bf16",)):
            continue
        if "function" in tr:
            fns = tr["function"] if isinstance(tr["function"], (list, tuple)) else [tr["function"]]
            shas = [function_sha(src, f) for f in fns]
            sha = (shas[0] if len(shas) == 1 else
                   None if None in shas else hashlib.sha256("".join(shas).encode()).hexdigest())
        else:
            sha = source_sha(src)
        if tr.get("sha") == sha:
            return tr["bytes"]
    return None


def rooflines(w, phases, precision, K):
    """Roofline entry per timed phase that is one kernel family: algorithmic
    work per launch / device time per launch (CUDA events on the state's
    stream) against the peak of the pipe that bounds it."""
    pk, pk_kind = peaks()
    per = algorithmic_per_walker(w)
    per_bytes = bytes_per_walker(w, precision)
    out = []
    for ph, (kname, bound, src) in kernel_of_phase(precision).items():
        v = phases[ph]
        if v["count"] == 0 or v["ms"] <= 0:
            continue
        ms_launch = v["ms"] / v["count"]
        work = per[ph] * w.nwalkers
        if bound == "hbm":
            # bytes per launch / time, against the measured copy bandwidth
            peak, unit, src_peak = pk["hbm_gbs"], "GB/s", f"{pk_kind} HBM copy bandwidth"
            achieved = per_bytes[ph] * w.nwalkers / (ms_launch * 1e-3) / 1e9
            traffic = traffic_of(ph, src, precision)
            out.append({"phase": ph, "kernel": kname, "bound": bound, "achieved": achieved,
                        "peak": peak, "unit": unit, "frac": achieved / peak, "traffic": traffic,
                        "peak_source": src_peak, "ms_per_launch": ms_launch,
                        "launches_per_step": v["count"] / K,
                        "share_of_step": v["ms"] / sum(x["ms"] for x in phases.values())})
            continue
        if bound == "alu32":
            peak, unit, src_peak = FP32_PEAK_TFLOPS, "TFLOP/s", (
                "derived: 152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz")
            bound = "alu"
        elif bound == "alu" or precision == "fp64":
            peak, unit, src_peak = FP64_PEAK_TFLOPS, "TFLOP/s", (
                "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz")
            bound = "alu"
        else:
            base = pk["bf16_tflops_sustained"]
            peak = base if precision.startswith("bf16") else base / 2
            unit = "TFLOP/s"
            src_peak = (f"{pk_kind} bf16 sustained" if precision.startswith("bf16")
                        else f"{pk_kind} bf16 sustained / 2 (TF32 nominal ratio)")
        achieved = work / (ms_launch * 1e-3) / 1e12
        traffic = traffic_of(ph, src, precision)
        out.append({"phase": ph, "kernel": kname, "bound": bound, "achieved": achieved,
                    "peak": peak, "unit": unit, "frac": achieved / peak, "traffic": traffic,
                    "peak_source": src_peak, "ms_per_launch": ms_launch,
                    "launches_per_step": v["count"] / K,
                    "share_of_step": v["ms"] / sum(x["ms"] for x in phases.values())})
    out.sort(key=lambda d: -d["share_of_step"])
    return out


def flops_per_walker_step(w: workloads.Workload, s=1):
    """Algorithmic FLOPs per walker-step (packed symmetric V, real Lh, s spin
    blocks run): force bias, V, Taylor, B_half, overlap/Theta, QR/q,
    exchange/k_E."""
    M, N, G, n = w.M, w.N, w.nchol, w.taylor_order
    f_fb = 4 * s * G * N * M
    f_v = 2 * G * M * (M + 1)
    f_t = 8 * n * s * M * M * N
    f_b = 8 * s * M * M * N
    f_ov = 4 * s * N * N * M + 8 * s * M * N * N + (8 / 3) * s * N ** 3
    f_qr = (8 * s * M * N * N + f_ov) / w.qr_period if w.qr_period else 0
    f_e = (4 * s * G * N * N * M + 4 * s * N * M + f_fb) / w.energy_period if w.energy_period else 0
    return dict(force_bias=f_fb, v_assembly=f_v, taylor=f_t, bhalf=f_b, overlap=f_ov, qr=f_qr,
                energy=f_e, total=f_fb + f_v + f_t + f_b + f_ov + f_qr + f_e)


def make_inputs(w: workloads.Workload, rank=0):
    from paper_1711_02242_gb300.rhf import rhf_trial

    h1, L, H0 = w.hamiltonian()
    C, conv, grad = rhf_trial(h1, L, w.N, max_iter=25)
    return h1, L, H0, C, conv, grad


def run_gpu(args, w: workloads.Workload):
    import torch

    import paper_1711_02242_gb300 as pkg
    from paper_1711_02242_gb300 import build as b

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b.build()
    prec = PRECISIONS[args.precision]
    h1, L, H0, C, conv, grad = make_inputs(w)
    pc = args.pc_period if args.pc_period is not None else w.pc_period
    sharded = ws > 1
    if sharded:
        # one population of ws x W walkers: this rank steps the global walkers
        # [rank W, (rank + 1) W) (same seed everywhere, fields keyed by the
        # global index); the comb and the estimator span all ranks
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed,
                               qr_period=w.qr_period, energy_period=0, pc_period=0,
                               taylor_order=w.taylor_order, precision=prec, H0=H0,
                               use_graph=0 if args.no_graph else 1, walker0=rank * w.nwalkers)
    else:
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed,
                               qr_period=w.qr_period, energy_period=w.energy_period,
                               pc_period=pc, taylor_order=w.taylor_order, precision=prec, H0=H0,
                               use_graph=0 if args.no_graph else 1)
    stream = torch.cuda.Stream(device=dev)
    run = pkg.AfqmcRun(h1, L, C, p, device=dev, stream=stream)
    K = args.steps
    pop = None
    if sharded:
        from paper_1711_02242_gb300.dist import ShardedPopulation, StateShard

        pop = ShardedPopulation(StateShard(run), pc_period=pc, energy_period=w.energy_period)
    # warm-up: at least one whole graph block (capture + first replay)
    blk = math.lcm(*[x for x in (w.qr_period, pc, w.energy_period) if x]) or 1
    Wm = max(args.warmup, blk)
    Wm = -(-Wm // blk) * blk
    if pop is not None:
        pop.run(Wm)
    else:
        run.propagate(Wm)
    stream.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lib = pkg.lib()
    launches0 = pkg.afqmc_launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        e0.record(stream)
        if pop is not None:
            pop.run(K)
        else:
            run.propagate(K)
        e1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize(dev)
    barrier()
    launches = pkg.afqmc_launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    import ctypes

    # the same K steps again, launched one by one with CUDA events around
    # every phase on the state's stream: phase times and the dominant kernel
    nph = len(PHASES)
    ph_ms = (ctypes.c_double * nph)()
    ph_n = (ctypes.c_int64 * nph)()
    ph_k = (ctypes.c_int64 * nph)()
    pkg._check(lib.afqmc_profile_start(run.s, K))
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    run.propagate(K)
    p1.record(stream)
    pkg._check(lib.afqmc_profile_stop(run.s, ph_ms, ph_n, ph_k))
    ms_profiled = p0.elapsed_time(p1)
    # energy evaluations: afqmc_energy (local energies of every walker, the
    # estimator, and the 2-double read back)
    n_e = 5
    t0 = time.perf_counter()
    for _ in range(n_e):
        run.energy()
    s_energy = (time.perf_counter() - t0) / n_e
    ms_total = max_over_ranks(ms_total, device=dev)
    info = run.info()
    if pop is not None:
        E, wsum = pop.energy()  # the whole population's estimator
    else:
        E, wsum = run.energy()
    run.close()
    del run

    # end to end through the public API with host buffers: set-up (upload of
    # h1, L and the trial from pinned host memory), K steps, energy read back;
    # the workspace comes from the process's device-memory pool (a warm
    # process, as a caller running one walk after another)
    t_e2e = float("nan")
    if not args.no_e2e:
        h1_h, L_h, C_h = (pinned_copy(torch, a) for a in (h1, L, C))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        run2 = pkg.AfqmcRun(h1_h, L_h, C_h, p, device=dev, stream=stream)
        run2.propagate(K)
        run2.energy()
        t_e2e = time.perf_counter() - t0
        run2.close()

    phases = {PHASES[i]: {"ms": ph_ms[i], "count": int(ph_n[i]), "kernels": int(ph_k[i])}
              for i in range(len(PHASES))}
    prec_rep = None
    if prec != 0 and rank == 0 and not args.no_precision_report:
        prec_rep = precision_report(w, prec, h1, L, C, H0)
    fp64 = None
    if prec != 0 and rank == 0 and not args.no_fp64_compare:
        fp64 = fp64_compare(w, p, h1, L, C, dev, stream, args.fp64_steps)
    bias = None
    if prec != 0 and rank == 0 and not args.no_bias:
        bias = bias_report(device=dev, stream=stream, c2_inputs=(h1, L, H0, C))
    return dict(ms_total=ms_total, phases=phases, launches=launches, info=info, E=E, wsum=wsum,
                clocks=clk.summary(), e2e_s=t_e2e, trial_converged=conv, trial_grad=grad,
                h2d_bytes=h1.nbytes + L.nbytes + C.nbytes, world=ws, rank=rank, warmup=Wm,
                ms_profiled=ms_profiled, s_energy=s_energy, graph=not args.no_graph,
                sharded=sharded, pc_period=pc,
                precision_report=prec_rep, fp64=fp64, bias=bias)


def fp64_compare(w, p, h1, L, C, dev, stream, steps):
    """The FP64 path on the same workload and GPU: a few steps after one
    untimed step (its step is ~100x the mixed one)."""
    import dataclasses

    import torch

    import paper_1711_02242_gb300 as pkg

    q = pkg.Params.from_buffer_copy(p)
    q.precision = pkg.AFQMC_FP64
    q.use_graph = 0
    run = pkg.AfqmcRun(h1, L, C, q, device=dev, stream=stream)
    run.propagate(1)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run.propagate(steps)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    run.close()
    del run
    torch.cuda.empty_cache()
    return {"value": w.nwalkers * steps / (ms * 1e-3), "unit": "walker-steps/s",
            "ms_per_step": ms / steps, "steps": steps,
            "note": "the same workload on the FP64 path (every step in float64/complex128), "
                    "same GPU, kernel by kernel"}


class OracleSampler:
    """The oracle as it stands, stepping a bounded sample of the workload's
    walkers: the first n_walkers walkers of the population (the oracle skips
    the others, whose weight is set to 0) from the initial walkers, step after
    step with the workload's Gram-Schmidt and energy periods, so that a run of
    consecutive steps costs what the same steps of the whole walk cost per
    walker.  The set-up, like afqmc_init on the GPU, is untimed."""

    def __init__(self, w: workloads.Workload, n_walkers: int):
        from oracle import afqmc

        h1, L, H0, C, _, _ = make_inputs(w)
        p = afqmc.Params(dt=w.dt, seed=w.seed, qr_period=w.qr_period,
                         energy_period=w.energy_period, taylor_order=w.taylor_order)
        self.orc = afqmc.Oracle(h1, L, C, w.nwalkers, p, H0=H0)
        self.orc.weight[n_walkers:] = 0.0  # the oracle skips zero-weight walkers
        self.n = n_walkers

    def step(self):
        t0 = time.perf_counter()
        self.orc.step()
        return time.perf_counter() - t0


def precision_report(w: workloads.Workload, prec: int, h1, L, C, H0, nwalk=32):
    """Mixed path against the FP64 path on identical inputs: trial energy,
    local energies of identical perturbed walkers (Eqs. localenergy2/3), and
    the orbitals after one step on identical Philox fields."""
    import torch

    import paper_1711_02242_gb300 as pkg

    runs = {}
    for pr in (0, prec):
        p = pkg.default_params(w.M, w.N, w.nchol, nwalk, dt=w.dt, seed=w.seed, H0=H0,
                               qr_period=w.qr_period, energy_period=0, precision=pr)
        runs[pr] = pkg.AfqmcRun(h1, L, C, p)
    e_t = {pr: r.info().E_T for pr, r in runs.items()}
    rng = np.random.default_rng(11)
    phi = C[None] + 0.05 * (rng.standard_normal((nwalk,) + C.shape)
                            + 1j * rng.standard_normal((nwalk,) + C.shape))
    for r in runs.values():
        r.set_walkers(phi, np.ones(nwalk))
    el = {pr: r.local_energies() for pr, r in runs.items()}
    d = np.abs(el[prec] - el[0])
    for r in runs.values():
        r.set_walkers(np.broadcast_to(C, (nwalk,) + C.shape), np.ones(nwalk))
        r.propagate(1)
    p64 = runs[0].get_walkers()[0]
    pmx = runs[prec].get_walkers()[0]
    rel = float(np.linalg.norm(pmx - p64) / np.linalg.norm(p64))
    out = {"trial_energy_Ha": e_t[0], "dE_trial_mHa": 1e3 * (e_t[prec] - e_t[0]),
           "dEloc_mean_abs_mHa": 1e3 * float(d.mean()), "dEloc_max_mHa": 1e3 * float(d.max()),
           "dEloc_rel_mean": float((d / np.abs(el[0])).mean()),
           "phi_rel_err_one_step": rel, "walkers": nwalk,
           "note": "mixed minus FP64 on identical walkers and fields; the FP64 path is held "
                   "to the oracle at 1e-10"}
    for r in runs.values():
        r.close()
    del runs
    torch.cuda.empty_cache()
    return out


def bias_runs(w: workloads.Workload, precs, steps, energy_period, device=None, stream=None,
              h1=None, L=None, C=None, H0=0.0, groups=16):
    """Energy bias of the mixed precisions against the float64 path on
    identical Philox fields (same seed, same initial walkers, same step
    order): `steps` steps, a record every `energy_period`.  Without
    population control the walkers are independent, so the population is cut
    into `groups` groups of consecutive walkers, each an independent sample of
    the run; per group and record the mixed estimator sum W Re E_loc / sum W
    (Re E_loc capped as in the walk) is formed from the walkers' weights and
    local energies read back from the GPU, then

      run        time average over the records of E_mixed - E_fp64, the two
                 walks' group estimators (the walks separate only by the mixed
                 path's rounding);
      estimator  the same for the mixed estimator evaluated on the float64
                 walk's own walkers and weights (the evaluation's error alone);

    as the mean over groups with its standard error (spread over groups), in
    mHa."""
    import torch

    import paper_1711_02242_gb300 as pkg

    if h1 is None:
        h1, L, H0, C, _, _ = make_inputs(w)

    def mk(prec):
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                               qr_period=w.qr_period, energy_period=0,
                               taylor_order=w.taylor_order, precision=prec)
        return pkg.AfqmcRun(h1, L, C, p, device=device or "cuda:0", stream=stream)

    nrec = steps // energy_period
    r64 = mk(0)
    mixed = {pr: mk(PRECISIONS[pr]) for pr in precs}
    probe = {pr: mk(PRECISIONS[pr]) for pr in precs}
    half = math.sqrt(2.0 / w.dt)  # the estimator's cap, C = 2 (Eq. cap)
    gidx = np.array_split(np.arange(w.nwalkers), groups)

    def group_estimates(wt, el, e_t):
        er = np.clip(el.real, e_t - half, e_t + half)
        wr = wt.real
        return np.array([np.sum(wr[g] * er[g]) / np.sum(wr[g]) if np.sum(wr[g]) > 0 else np.nan
                         for g in gidx])

    e_t64 = r64.info().E_T
    e_t = {pr: r.info().E_T for pr, r in mixed.items()}
    g64, gmx, gpr = [], {pr: [] for pr in precs}, {pr: [] for pr in precs}
    for _ in range(nrec):
        r64.propagate(energy_period)
        wt64, el64 = r64.weights(), r64.local_energies()
        g64.append(group_estimates(wt64, el64, e_t64))
        for pr, r in mixed.items():
            r.propagate(energy_period)
            gmx[pr].append(group_estimates(r.weights(), r.local_energies(), e_t[pr]))
        phi, _, _ = r64.get_walkers()
        for pr, r in probe.items():
            r.set_walkers(phi, wt64)
            gpr[pr].append(group_estimates(wt64, r.local_energies(), e_t[pr]))
    g64 = np.array(g64)  # [records][groups]
    out = {}
    for pr in precs:
        d_run = 1e3 * np.nanmean(np.array(gmx[pr]) - g64, axis=0)  # per group, time-averaged
        d_est = 1e3 * np.nanmean(np.array(gpr[pr]) - g64, axis=0)
        ok = np.isfinite(d_run) & np.isfinite(d_est)
        n = int(np.count_nonzero(ok))
        out[pr] = {"bias_run_mHa": float(np.mean(d_run[ok])),
                   "se_run_mHa": float(np.std(d_run[ok], ddof=1) / math.sqrt(n)),
                   "bias_estimator_mHa": float(np.mean(d_est[ok])),
                   "se_estimator_mHa": float(np.std(d_est[ok], ddof=1) / math.sqrt(n)),
                   "dE_trial_mHa": 1e3 * (e_t[pr] - e_t64), "groups_used": n,
                   "status": int(mixed[pr].info().status)}
    res = {"steps": steps, "energy_period": energy_period, "records": nrec,
           "walkers": w.nwalkers, "groups": groups,
           "E_fp64_mean_Ha": float(np.nanmean(g64)),
           "alive_fp64_end": int(r64.info().alive), "precisions": out}
    for r in [r64, *mixed.values(), *probe.values()]:
        r.close()
    del r64, mixed, probe
    torch.cuda.empty_cache()
    return res


# workload: (mixed precisions, steps, energy period, walker groups)
BIAS_CASES = {"c0": (("bf16", "tf32"), 40, 2, 8), "c1": (("tf32", "bf16"), 100, 5, 16),
              "c2": (("bf16", "tf32"), 100, 5, 16)}


def bias_report(device=None, stream=None, c2_inputs=None):
    """bias_runs for the three single-system workloads (the M=12 one in both
    mixed precisions, M=100 in TF32 and BF16, M=300 in BF16 and TF32)."""
    rep = {}
    for name, (precs, steps, ep, ng) in BIAS_CASES.items():
        w = workloads.config(name)
        kw = {}
        if name == "c2" and c2_inputs is not None:
            kw = dict(zip(("h1", "L", "H0", "C"), c2_inputs))
        t0 = time.perf_counter()
        rep[name] = bias_runs(w, precs, steps, ep, device=device, stream=stream, groups=ng, **kw)
        rep[name]["seconds"] = time.perf_counter() - t0
    rep["note"] = ("mixed minus float64 on identical Philox fields (same seed and initial "
                   "walkers), no population control: 'run' compares the two walks' mixed "
                   "estimators, 'estimator' evaluates the mixed estimator on the float64 "
                   "walk's walkers and weights; time averages over the records per group of "
                   "walkers, mean and standard error over the independent groups")
    return rep


def cpu_sample(w: workloads.Workload, n_walkers=16, n_steps=20):
    """Oracle walker-steps/s on the first n_steps steps (two energy
    evaluations and four Gram-Schmidt passes at the M=300 periods, about 12 s
    on 16 Grace cores) of n_walkers walkers."""
    s = OracleSampler(w, n_walkers)
    dt = sum(s.step() for _ in range(n_steps))
    cores = len(os.sched_getaffinity(0))
    return dict(value=n_walkers * n_steps / dt, unit="walker-steps/s", cores=cores, kind="oracle",
                sample=f"steps 1-{n_steps} (Gram-Schmidt every {w.qr_period}, energy every "
                       f"{w.energy_period}) of {n_walkers} of the {w.nwalkers} walkers of the "
                       f"M={w.M} workload (set-up untimed), numpy float64, {cores} host threads",
                seconds=dt)


def workload_desc(w: workloads.Workload) -> str:
    return (f"M={w.M} N_up=N_dn={w.N} nchol={w.nchol} walkers={w.nwalkers} dt={w.dt} "
            f"qr/{w.qr_period} energy/{w.energy_period} taylor {w.taylor_order}; synthetic "
            f"Hamiltonian, Cholesky amplitude {workloads.l_amplitude(w.M, w.nchol):.3g} "
            f"(0.5 at M=12, scaled so that sum_g |L_g|_F^2 is the M=12 value)")


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    sample = args.ref_walkers
    s = OracleSampler(w, sample)
    for _ in range(args.warmup):
        s.step()
    dt = sum(s.step() for _ in range(args.steps))
    cores = len(os.sched_getaffinity(0))
    val = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": f"walker-steps/s at M={w.M}", "value": val,
        "unit": "walker-steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w), "sampled_walkers": sample,
                   "note": "the float64 oracle on the host cores, a bounded sample of the walkers"},
        "cpu_baseline": {"value": val, "unit": "walker-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} walkers, steps {args.warmup + 1}-"
                          f"{args.warmup + args.steps} of the walk (Gram-Schmidt every "
                          f"{w.qr_period}, energy every {w.energy_period})"},
        "e2e": {"value": val, "unit": "walker-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _inputs_parallel(ws, trial_iters=0):
    """Hamiltonians (and trials: core orbitals, or a few RHF iterations) for
    many workloads, generated on host threads."""
    import concurrent.futures as cf

    from paper_1711_02242_gb300.rhf import rhf_trial

    def one(w):
        h1, L, H0 = w.hamiltonian()
        if trial_iters:
            C, _, _ = rhf_trial(h1, L, w.N, max_iter=trial_iters)
        else:
            C = np.linalg.eigh(h1)[1][:, :w.N]
        return h1, L, H0, C

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        return list(ex.map(one, ws))


def run_batched(args):
    """16 uneven systems (M in {40..200}, N = M/8, nchol = 5M, walkers in
    {64..1024}) advanced by one CUDA graph launch per block of steps."""
    import torch

    import paper_1711_02242_gb300 as pkg
    from paper_1711_02242_gb300 import build as b

    b.build()
    prec = PRECISIONS[args.precision]
    ws_ = workloads.batched_systems()
    inputs = _inputs_parallel(ws_, trial_iters=10)
    runs = []
    for w, (h1, L, H0, C) in zip(ws_, inputs):
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                               qr_period=w.qr_period, energy_period=w.energy_period,
                               precision=prec, use_graph=1)
        runs.append(pkg.AfqmcRun(h1, L, C, p, stream=torch.cuda.Stream()))
    g = pkg.AfqmcGroup(runs)
    blk = 10
    K = -(-args.steps // blk) * blk

    def timed(mode, clk=None):
        # the block's capture chosen (default: four trial blocks, two each way)
        g.set_grouped(mode)
        g.propagate(4 * blk if mode == "auto" else blk)
        g.synchronize()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = pkg.afqmc_launch_count()
        if clk:
            clk.__enter__()
        e0.record(g.stream)
        g.propagate(K)
        e1.record(g.stream)
        torch.cuda.synchronize()
        if clk:
            clk.__exit__(None, None, None)
        return e0.elapsed_time(e1), pkg.afqmc_launch_count() - l0, g.tiles()

    clk = ClockSampler(0)
    ms, launches, (grouped_on, tiles) = timed("auto", clk)
    ms_grouped, _, (_, tiles_g) = timed(True)
    ms_branches, _, _ = timed(False)
    total_ws = sum(w.nwalkers for w in ws_)
    # the same systems one after the other, each with its own graph replay
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    s0.record(st)
    for r in runs:
        r.stream.wait_stream(st)
        r.propagate(K)
        st.wait_stream(r.stream)
    s1.record(st)
    torch.cuda.synchronize()
    ms_seq = s0.elapsed_time(s1)
    line = {
        "metric": "walker-steps/s, 16 uneven systems in one graph launch per block",
        "capture": "grouped" if grouped_on else "graph branches",
        "grouped": {"value": total_ws * K / (ms_grouped * 1e-3), "ms_per_step": ms_grouped / K,
                    "tiles": dict(zip(("force_bias", "v", "half_step_1", "half_step_2"), tiles_g)),
                    "note": "each of the step's four tensor-core contractions of all 16 systems "
                            "as one persistent launch over (system, tile); tile widths timed on "
                            "the systems' buffers"},
        "value": total_ws * K / (ms * 1e-3), "unit": "walker-steps/s", "n_gpus": 1, "steps": K,
        "warmup": blk, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": "16 systems, M in {40..200}, N=M/8, nchol=5M, walkers in {64..1024}",
                   "systems": [[w.M, w.N, w.nchol, w.nwalkers] for w in ws_],
                   "trial": "RHF, 10 DIIS iterations"},
        "one_by_one": {"value": total_ws * K / (ms_seq * 1e-3), "ms_per_step": ms_seq / K,
                       "note": "same systems propagated one after another (own graphs)"},
        "graph_branches": {"value": total_ws * K / (ms_branches * 1e-3),
                           "ms_per_step": ms_branches / K,
                           "note": "same block captured as each system's own kernels on its own "
                                   "stream (branches of one graph), no grouped launches"},
        "note": "value: the group's default capture, chosen by timing one block each way",
        "gpu_launches": launches, "clocks": clk.summary(),
        "e2e": None,
    }
    print(json.dumps(line))
    g.close()
    return 0


def run_serve(args):
    """A Poisson stream of AFQMC run requests (M uniform in [20, 300],
    N uniform in [2, M/8], nchol = 5M, 128-2048 walkers) served with
    continuous batching; p50/p99 run latency and aggregate throughput."""
    import torch

    import paper_1711_02242_gb300 as pkg
    from paper_1711_02242_gb300 import build as b
    from paper_1711_02242_gb300.serve import Request, Server, latency_stats

    b.build()
    prec = PRECISIONS[args.precision]
    stream = workloads.request_stream(count=args.requests, rate=args.rate, blocks=args.blocks,
                                      steps_per_block=args.steps_per_block)
    inputs = _inputs_parallel([w for _, w in stream])
    reqs = [Request(rid=i, arrival=t, h1=h1, L=L, trial=C, nwalkers=w.nwalkers, nsteps=w.nsteps,
                    seed=w.seed, energy_period=w.energy_period)
            for i, ((t, w), (h1, L, H0, C)) in enumerate(zip(stream, inputs))]
    free, _ = torch.cuda.mem_get_info()
    pool = int(min(0.6 * free, 120e9))
    srv = Server(pool, precision=prec, chunk_steps=args.steps_per_block,
                 max_active=args.slots or None)
    t0 = time.perf_counter()
    with ClockSampler(0) as clk:
        done = srv.run(reqs, realtime=True)
    makespan = time.perf_counter() - t0
    ws_total = sum(r.nwalkers * r.nsteps for r in done)
    lat = latency_stats(done)
    # FP64 one at a time: the first requests timed alone, the rest extrapolated
    # by algorithmic FLOPs (the FP64 path is bound by the FP64 pipe)
    n_fp = min(3, len(reqs))
    fl = lambda r: flops_per_walker_step(workloads.Workload(  # noqa: E731
        "r", M=r.trial.shape[0], N=r.trial.shape[1], nchol=r.L.shape[0], nwalkers=r.nwalkers,
        qr_period=5, energy_period=r.energy_period))["total"] * r.nwalkers * r.nsteps
    srv64 = Server(pool, precision=0, chunk_steps=args.steps_per_block)
    t1 = time.perf_counter()
    for r in reqs[:n_fp]:
        srv64.run([dataclasses_replace(r)], realtime=False)
    t_fp = time.perf_counter() - t1
    fp_rate = sum(fl(r) for r in reqs[:n_fp]) / t_fp
    t_fp_all = sum(fl(r) for r in reqs) / fp_rate
    line = {
        "metric": "p50/p99 run latency and walker-steps/s, served request stream",
        "value": ws_total / makespan, "unit": "walker-steps/s", "n_gpus": 1,
        "steps": int(np.mean([r.nsteps for r in reqs])), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{len(reqs)} requests, Poisson {args.rate}/s, M in [20,300], "
                               f"N in [2,M/8], nchol=5M, walkers in [128,2048], "
                               f"{args.blocks} blocks x {args.steps_per_block} steps",
                   "pool_GB": pool / 1e9, "trial": "core-Hamiltonian orbitals",
                   "slots": args.slots},
        "latency": lat, "makespan_s": makespan,
        "offered_walker_steps_per_s": ws_total / max(1e-9, max(r.arrival for r in reqs)),
        "fp64_one_at_a_time": {"measured_requests": n_fp, "seconds_measured": t_fp,
                               "estimated_seconds_all": t_fp_all,
                               "walker_steps_per_s": ws_total / t_fp_all},
        "clocks": clk.summary(), "gpu_launches": None, "e2e": None,
    }
    print(json.dumps(line))
    return 0


def mcd_flops_bytes(npair: int, nvec: int):
    """Algorithmic FP64 work of a decomposition into nvec vectors over npair
    indices: iteration k (k earlier vectors) takes npair k fused multiply-adds
    (2 npair k FLOP) and streams the k earlier vectors' components and one row
    of V, 8 npair (k + 1) bytes, plus the residual diagonal (read and write)
    and the new vector (write), 24 npair bytes."""
    ks = nvec * (nvec - 1) / 2
    return 2.0 * npair * ks, 8.0 * npair * (ks + nvec) + 24.0 * npair * nvec


def mcd_oracle_sample(W, nvec_sample, delta):
    """The oracle's decomposition of the host pair matrix, stopped after
    nvec_sample vectors (0: not stopped): seconds, vectors."""
    from oracle import mcd as omcd

    t0 = time.perf_counter()
    Lo, piv, dmax, resid, conv = omcd.modified_cholesky(W, delta, max_vectors=nvec_sample or None)
    return time.perf_counter() - t0, len(piv)


def run_mcd(args):
    """Modified Cholesky decomposition (Sec. 2.3, Eqs. chol and chol2) of the
    interaction v_pqrs = sum_g L_g[p,r] L_g[q,s] of the chosen workload's
    Cholesky vectors, over the M(M+1)/2 index pairs (afqmc_modified_cholesky_pairs),
    delta = 1e-6.  One step is one whole decomposition."""
    import torch

    w = workloads.config(args.config)
    M = w.M
    npair = M * (M + 1) // 2
    delta = 1e-6
    maxv = w.nchol + 64
    _, L, _ = w.hamiltonian()
    cores = len(os.sched_getaffinity(0))
    desc = (f"modified Cholesky (delta {delta:g}) of the M={M} interaction built from the "
            f"{w.nchol} Cholesky vectors of the walker-steps workload; {npair} index pairs "
            f"p<=r, pair matrix {npair * npair * 8 / 1e9:.1f} GB float64")
    ws_, rank, _ = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        if not torch.cuda.is_available():
            print(json.dumps({"impl": "reference", "unavailable": "the pair matrix is built on "
                              "the GPU (numpy would take minutes)"}))
            return 0
        W = workloads.interaction_pairs_device(L).cpu().numpy()
        nv = args.mcd_cpu_vectors
        secs = []
        for _ in range(args.steps):
            t, n = mcd_oracle_sample(W, nv, delta)
            secs.append(t)
        val = n / statistics.mean(secs)
        line = {"impl": "reference", "metric": f"Cholesky vectors/s, mCD at M={M}",
                "value": val, "unit": "vectors/s", "n_gpus": ws_, "steps": args.steps,
                "warmup": 0, "ms_per_step": 1e3 * statistics.mean(secs),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": desc, "sampled_vectors": n},
                "cpu_baseline": {"value": val, "unit": "vectors/s", "cores": cores,
                                 "kind": "oracle",
                                 "sample": f"{n} vectors of the decomposition (the whole "
                                           f"one unless --mcd-cpu-vectors caps it)"},
                "e2e": {"value": val, "unit": "vectors/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import ctypes

    import paper_1711_02242_gb300 as pkg
    from paper_1711_02242_gb300 import build as b

    b.build()
    dev = torch.device("cuda", 0)
    W = workloads.interaction_pairs_device(L, dev)
    torch.cuda.synchronize()
    nbytes = ctypes.c_size_t(0)
    pkg._check(pkg.lib().afqmc_mcd_pairs_workspace_size(M, maxv, ctypes.byref(nbytes)))
    work = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        Lv, piv, resid = pkg.afqmc_modified_cholesky_pairs(W, M, delta, maxv, workspace=work)
    torch.cuda.synchronize()
    K = args.steps
    l0 = pkg.afqmc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(st)
        for _ in range(K):
            Lv, piv, resid = pkg.afqmc_modified_cholesky_pairs(W, M, delta, maxv, workspace=work)
        e1.record(st)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    launches = (pkg.afqmc_launch_count() - l0) // K
    nvec = Lv.shape[0]
    flops, byts = mcd_flops_bytes(npair, nvec)
    # end to end: pair matrix from pinned host memory, decomposition, vectors
    # back to pinned host memory
    e2e = None
    if not args.no_e2e:
        Wh = torch.empty(W.shape, dtype=W.dtype, pin_memory=True)
        Wh.copy_(W)
        Wd = torch.empty_like(W)
        Lh = torch.empty((nvec, M, M), dtype=torch.float64, pin_memory=True)
        del W
        torch.cuda.synchronize()
        ke = max(1, K // 2)
        t0 = time.perf_counter()
        for _ in range(ke):
            Wd.copy_(Wh, non_blocking=True)
            Lv, piv, resid = pkg.afqmc_modified_cholesky_pairs(Wd, M, delta, maxv, workspace=work)
            Lh.copy_(Lv, non_blocking=True)
            torch.cuda.synchronize()
        s_e2e = (time.perf_counter() - t0) / ke
        e2e = {"value": nvec / s_e2e, "unit": "vectors/s", "h2d_bytes_per_step": Wh.nbytes,
               "d2h_bytes_per_step": Lh.nbytes,
               "includes": "pair matrix host->device, decomposition, vectors device->host "
                           "(pinned buffers)"}
        W = Wd
    pk_fp64 = FP64_PEAK_TFLOPS
    hbm = peaks()[0]["hbm_gbs"]
    line = {
        "metric": f"Cholesky vectors/s, mCD at M={M}", "value": nvec / (ms * 1e-3),
        "unit": "vectors/s", "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "vectors": nvec, "residual": resid,
                   "l2": f"input larger than L2 (pair matrix {npair * npair * 8 / 1e9:.1f} GB)"},
        "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": pk_fp64,
                     "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / pk_fp64,
                     "traffic": None, "kernel": "k_mcd_step",
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz",
                     "ms_per_launch": ms / max(1, launches),
                     "note": "one FMA per streamed float64 puts the step kernel on the FP64 "
                             "pipe (8 B/FMA x 0.6 TFMA/s = 4.8 TB/s < HBM); whole "
                             "decomposition time, launch gaps included"},
        "hbm_view": {"achieved": byts / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": byts / (ms * 1e-3) / 1e9 / hbm},
        "gpu_launches": launches, "clocks": clk.summary(), "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        Wc = W.cpu().numpy()
        t, n = mcd_oracle_sample(Wc, args.mcd_cpu_vectors, delta)
        line["cpu_baseline"] = {"value": n / t, "unit": "vectors/s", "cores": cores,
                                "kind": "oracle", "seconds": t,
                                "sample": (f"the first {n} of the {nvec} vectors" if n < nvec
                                           else "the whole decomposition") +
                                          " of the same pair matrix (numpy float64)"}
    print(json.dumps(line))
    return 0


def _case_main(a):
    """One contraction or kernel of the M=300 step, timed with CUDA events
    (random operands), for kernel profiling:
      v       V = sum_g x_g L_g as afqmc_contract with the M=300 shapes
              (A = 1024 x 1800 fields, B = 45150 x 1800 packed Cholesky
              vectors, C FP32: about 350 MB, B alone 162 MB in BF16);
      fb      the force-bias contraction (A = 1024 x 7600, B = 1800 x 7600);
      taylor  the sixth-order Taylor series of exp(V) on --walkers walkers,
              M = 300, N = 25 (afqmc_taylor_series; V 187 MB in BF16);
      mcd     the modified Cholesky decomposition over index pairs
              (delta = 1e-6) of the interaction of a seeded Hamiltonian with
              --orbitals M orbitals and 6M vectors (pair matrix 16.3 GB at
              M = 300, 1.3 GB at M = 160), one launch per vector;
      md      the M=100 walk with a trial of 1, 2 and 4 non-orthogonal
              determinants (rotations of the RHF determinant) in --dtype;
      bp      the M=300 walk with a back-propagation window of --window steps:
              time per step without and with the window, and afqmc_bp_end."""
    import torch

    import paper_1711_02242_gb300 as pkg
    from paper_1711_02242_gb300 import build as b

    b.build()
    if a.case == "taylor":
        return _case_taylor(a)
    if a.case == "mcd":
        return _case_mcd(a)
    if a.case == "bp":
        return _case_bp(a)
    if a.case == "md":
        return _case_md(a)
    if a.case == "ci":
        return _case_ci(a)
    if a.case == "v":
        m, n, k, pitch = 1024, 45150, 1800, 1800
    else:
        m, n, k, pitch = 1024, 1800, 25 * 304, 25 * 304
    dt = torch.bfloat16 if a.dtype == "bf16" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((m, pitch), generator=g, device="cuda").to(dt)
    B = torch.randn((n, pitch), generator=g, device="cuda").to(dt)
    ldc = (n + 3) // 4 * 4
    C = torch.empty((m, ldc), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    lib = pkg.lib()

    def call():
        pkg._check(lib.afqmc_contract(0 if a.dtype == "bf16" else 1, m, n, k,
                                      ctypes.c_void_p(A.data_ptr()), pitch,
                                      ctypes.c_void_p(B.data_ptr()), pitch, ctypes.c_float(1.0),
                                      ctypes.c_void_p(C.data_ptr()), ldc,
                                      ctypes.c_void_p(st.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream)))

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * m * n * k
    print(f"case {a.case} {a.dtype}: m={m} n={n} k={k}: {ms:.4f} ms/launch, "
          f"{flops / ms / 1e9:.1f} TFLOP/s, status {int(st.item())}")
    assert int(st.item()) == 0


def _case_taylor(a):
    import paper_1711_02242_gb300 as pkg
    import torch

    W, N, M, Mp, order = a.walkers, 25, 300, 304, 6
    dt = torch.bfloat16 if a.dtype == "bf16" else torch.float32
    g = torch.Generator(device="cuda").manual_seed(0)
    V = torch.zeros((W, M, 2 * Mp), device="cuda")
    V[:, :, :M] = torch.randn((W, M, M), generator=g, device="cuda") * (0.05 / M ** 0.5)
    V[:, :, Mp:Mp + M] = torch.randn((W, M, M), generator=g, device="cuda") * (0.05 / M ** 0.5)
    V = V.to(dt)
    T0 = torch.zeros((W, 2 * N, 2 * Mp), device="cuda")
    T0[:, :, :M] = torch.randn((W, 2 * N, M), generator=g, device="cuda")
    T0 = T0.to(dt)
    T1 = torch.empty_like(T0)
    S = torch.empty((W, 2 * N, Mp), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    lib = pkg.lib()

    def call():
        pkg._check(lib.afqmc_taylor_series(0 if a.dtype == "bf16" else 1, W, N, M, Mp, order,
                                           ctypes.c_void_p(V.data_ptr()),
                                           ctypes.c_void_p(T0.data_ptr()),
                                           ctypes.c_void_p(T1.data_ptr()),
                                           ctypes.c_void_p(S.data_ptr()), Mp, 0,
                                           ctypes.c_void_p(st.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream)))

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    vbytes = V.numel() * V.element_size()
    print(f"case taylor {a.dtype}: W={W} N={N} M={M} order={order}: {ms:.4f} ms/launch, "
          f"V {vbytes / 1e6:.0f} MB once from HBM: {vbytes / ms / 1e6:.0f} GB/s, "
          f"V per term (L2): {order * vbytes / ms / 1e6:.0f} GB/s, status {int(st.item())}")
    assert int(st.item()) == 0


def _case_mcd(a):
    import paper_1711_02242_gb300 as pkg
    import torch

    import workloads

    M = a.orbitals
    G = 6 * M
    _, L, _ = workloads.hamiltonian(M, G, 5000 + M, l_scale=workloads.l_amplitude(M, G))
    W = workloads.interaction_pairs_device(L)
    del L
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Lv, piv, resid = pkg.afqmc_modified_cholesky_pairs(W, M, 1e-6, G + 16)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    n = Lv.shape[0]
    print(f"case mcd M={M} pairs={W.shape[0]} vectors={n} residual={resid:.3e} "
          f"ms={min(times):.3f} per-vector-us={1e3 * min(times) / n:.2f}")


def _case_bp(a):
    import paper_1711_02242_gb300 as pkg
    import time

    import torch

    import workloads
    from paper_1711_02242_gb300.rhf import rhf_trial

    w = workloads.config("c2")
    h1, L, H0 = w.hamiltonian()
    C, _, _ = rhf_trial(h1, L, w.N, max_iter=25)
    prec = {"fp64": 0, "tf32": 1, "bf16": 2}[a.dtype]
    m = a.window
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                           qr_period=w.qr_period, energy_period=w.energy_period, precision=prec,
                           bp_steps=m)
    st = torch.cuda.Stream()
    run = pkg.AfqmcRun(h1, L, C, p, stream=st)
    run.propagate(10)
    st.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        st.synchronize()
        return e0.elapsed_time(e1)

    t_plain = timed(lambda: run.propagate(m))
    run.bp_begin()
    t_window = timed(lambda: run.propagate(m))
    t0 = time.perf_counter()
    rho, phl, wp, wsum, n = run.bp_end()
    t_end = 1e3 * (time.perf_counter() - t0)
    print(f"case bp {a.dtype} M={w.M} walkers={w.nwalkers} window={n}: "
          f"ms/step plain={t_plain / m:.3f} window-open={t_window / m:.3f}; "
          f"bp_end ms={t_end:.2f}; trace(rho_PRes)={np.trace(rho).real:.6f} "
          f"|sum W F|/sum W={abs(wp) / abs(wsum):.4f}; status={run.info().status}")
    run.close()


def _case_md(a):
    import paper_1711_02242_gb300 as pkg
    import scipy.linalg as sla
    import torch

    import workloads
    from paper_1711_02242_gb300.rhf import rhf_trial

    w = workloads.config("c1")
    h1, L, H0 = w.hamiltonian()
    C, _, _ = rhf_trial(h1, L, w.N, max_iter=25)
    rng = np.random.default_rng(11)
    q, _ = np.linalg.qr(np.hstack([C, rng.standard_normal((w.M, w.M - w.N))]))
    basis = np.hstack([C, q[:, w.N:]])

    def rotated():
        K = 0.02 * rng.standard_normal((w.M, w.M))
        return basis @ sla.expm(K - K.T)[:, :w.N]

    st = torch.cuda.Stream()
    steps = 10
    for nd in (1, 2, 4):
        up = np.array([C] + [rotated() for _ in range(nd - 1)])
        dn = np.array([C] + [rotated() for _ in range(nd - 1)])
        coef = np.array([1.0] + [0.3 / nd] * (nd - 1), np.complex128)
        p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                               qr_period=w.qr_period, energy_period=0, ndet=nd,
                               precision={"fp64": 0, "tf32": 1, "bf16": 2}[a.dtype])
        run = pkg.AfqmcRun(h1, L, (coef, up, dn), p, stream=st)
        run.propagate(2)
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        run.propagate(steps)
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / steps
        import time

        t0 = time.perf_counter()
        run.local_energies()
        te = 1e3 * (time.perf_counter() - t0)
        print(f"case md {a.dtype} M={w.M} N={w.N} nchol={w.nchol} walkers={w.nwalkers} ndet={nd}: "
              f"ms/step={ms:.2f} walker-steps/s={w.nwalkers / ms * 1e3:.0f} energy-eval ms={te:.2f} "
              f"status={run.info().status} alive={run.info().alive}")
        run.close()


def _case_ci(a):
    """A CI expansion about the RHF determinant on the M=100 workload (10 + 10
    electrons, 500 vectors, 1024 walkers): 1 + 2 x 8 singles and 8 doubles
    per spin (25 determinants, at most 2 columns each) evaluated relative to
    the reference; ms per step and per local-energy evaluation."""
    import time

    import paper_1711_02242_gb300 as pkg
    import torch

    import workloads
    from paper_1711_02242_gb300.rhf import rhf_trial

    w = workloads.config("c1")
    h1, L, H0 = w.hamiltonian()
    C, _, _ = rhf_trial(h1, L, w.N, max_iter=25)
    rng = np.random.default_rng(12)
    q, _ = np.linalg.qr(np.hstack([C, rng.standard_normal((w.M, w.M - w.N))]))
    virt = q[:, w.N:]
    up, dn, coef = [C], [C], [1.0]
    for s in range(2):
        for k in range(8):
            V = C.copy()
            V[:, w.N - 1 - k % w.N] = virt[:, k]
            (up if s == 0 else dn).append(V)
            (dn if s == 0 else up).append(C)
            coef.append(0.05 * (1 + k) / 8 * (1j if s else 1.0))
    for k in range(8):
        V = C.copy()
        V[:, w.N - 1] = virt[:, k]
        V[:, w.N - 2] = virt[:, k + 8]
        up.append(V)
        dn.append(V)
        coef.append(-0.02)
    nd = len(coef)
    st = torch.cuda.Stream()
    steps = 10
    p = pkg.default_params(w.M, w.N, w.nchol, w.nwalkers, dt=w.dt, seed=w.seed, H0=H0,
                           qr_period=w.qr_period, energy_period=0, ndet=nd,
                           precision={"fp64": 0, "tf32": 1, "bf16": 2}[a.dtype])
    run = pkg.AfqmcRun(h1, L, (np.array(coef, np.complex128), np.array(up), np.array(dn)), p,
                       stream=st)
    run.propagate(2)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    run.propagate(steps)
    e1.record(st)
    st.synchronize()
    ms = e0.elapsed_time(e1) / steps
    t0 = time.perf_counter()
    run.local_energies()
    te = 1e3 * (time.perf_counter() - t0)
    print(f"case ci {a.dtype} M={w.M} N={w.N} nchol={w.nchol} walkers={w.nwalkers} ndet={nd}: "
          f"ms/step={ms:.2f} walker-steps/s={w.nwalkers / ms * 1e3:.0f} energy-eval ms={te:.2f} "
          f"E_T={run.info().E_T:.6f} status={run.info().status} alive={run.info().alive}")
    run.close()


def run_peaks(args):
    """Dense float64 and float32 matrix-multiply throughput through PyTorch
    (cuBLAS; TF32 off for float32), the counterpart of the driver's BF16
    measurement for the FP64 and FP32 pipes: best of 5 after warm-up and 4 s
    back to back, n^3 with n = 8192 (float64: 16384 for the sustained loop's
    operands would not change the rate; 8192 keeps it short)."""
    import torch

    torch.backends.cuda.matmul.allow_tf32 = False
    dev = torch.device("cuda", 0)
    out = {}
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        n = 8192
        a = torch.randn((n, n), dtype=dt, device=dev)
        b = torch.randn((n, n), dtype=dt, device=dev)
        c = torch.empty((n, n), dtype=dt, device=dev)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        reps, t0 = 0, time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record()
            while time.perf_counter() - t0 < 4.0:
                for _ in range(4):
                    torch.matmul(a, b, out=c)
                reps += 4
                torch.cuda.synchronize()
            e1.record()
            torch.cuda.synchronize()
        sus = e0.elapsed_time(e1) / reps
        out[name] = {"n": n, "burst_tflops": 2 * n ** 3 / (best * 1e-3) / 1e12,
                     "sustained_tflops": 2 * n ** 3 / (sus * 1e-3) / 1e12,
                     "clocks": clk.summary()}
        del a, b, c
        torch.cuda.empty_cache()
    derived = {"fp64": FP64_PEAK_TFLOPS, "fp32": FP32_PEAK_TFLOPS}
    for k in out:
        out[k]["derived_tflops"] = derived[k]
        out[k]["frac_of_derived"] = out[k]["burst_tflops"] / derived[k]
    print(json.dumps({"metric": "dense GEMM TFLOP/s (torch.matmul, cuBLAS)", "peaks": out}))
    return 0


def dataclasses_replace(r):
    import dataclasses

    return dataclasses.replace(r, arrival=0.0, energies=None)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "batched", "serve", "mcd", "bias", "case", "peaks"],
                    help="c2: the M=300 walker-steps/s line; batched / serve: the grouped and "
                         "served forms; mcd: the modified Cholesky decomposition of the "
                         "workload's interaction (their own JSON lines)")
    ap.add_argument("--mcd-cpu-vectors", type=int, default=0,
                    help="mcd: stop the oracle's sample after this many vectors (0: the whole "
                         "decomposition, about 10 s of CPU at M=300)")
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--blocks", type=int, default=4)
    ap.add_argument("--steps-per-block", type=int, default=25)
    ap.add_argument("--slots", type=int, default=8, help="serve: runs advanced per tick (0: memory only)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="bf16", choices=list(PRECISIONS))
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64 path's own few-step measurement")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--config", default="c2", choices=sorted(workloads.CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass")
    ap.add_argument("--no-graph", action="store_true", help="launch kernels one by one")
    ap.add_argument("--no-precision-report", action="store_true")
    ap.add_argument("--no-bias", action="store_true",
                    help="skip the run-level bias of the mixed precisions against float64")
    ap.add_argument("--ref-walkers", type=int, default=16)
    ap.add_argument("--case", default="v", choices=["v", "fb", "taylor", "mcd", "bp", "md", "ci"],
                    help="--workload case: one kernel or contraction of the step, for profiling")
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "tf32", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--walkers", type=int, default=512)
    ap.add_argument("--orbitals", type=int, default=300)
    ap.add_argument("--window", type=int, default=20)
    ap.add_argument("--pc-period", type=int, default=None,
                    help="steps between combs (default: the workload's, 0 = off); under "
                         "torchrun the comb spans all ranks")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "mcd":
        return run_mcd(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "case":
        _case_main(args)
        return 0
    if args.workload == "bias":
        from paper_1711_02242_gb300 import build as b

        b.build()
        print(json.dumps({"metric": "mixed-precision energy bias vs float64, mHa",
                          "bias_vs_fp64": bias_report()}))
        return 0
    w = workloads.config(args.config)
    if args.impl == "reference":
        return run_reference(args, w)
    r = run_gpu(args, w)
    if r["rank"] != 0:
        return 0
    K = args.steps
    N = r["world"]
    ms_step = r["ms_total"] / K
    value = job_throughput(w.nwalkers, K, r["ms_total"], N)
    fl = flops_per_walker_step(w)
    # the dominant kernel (largest share of the profiled step) and the others
    roofs = rooflines(w, r["phases"], args.precision, K)
    top = roofs[0]
    roof = {k: top[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof.update(kernel=top["kernel"], peak_source=top["peak_source"],
                ms_per_launch=top["ms_per_launch"])
    line = {
        "metric": f"walker-steps/s at M={w.M}", "value": value, "unit": "walker-steps/s",
        "n_gpus": N, "steps": K, "warmup": r["warmup"], "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_desc(w),
                   "parallelism": (f"one population sharded over {N} GPUs ({w.nwalkers} "
                                   f"walkers each; comb every {r['pc_period'] or 'never'}, "
                                   "estimator summed over ranks)" if r["sharded"] else "1 GPU"),
                   "precision": args.precision, "l2": l2_note(w),
                   "trial": f"RHF (25 iterations, converged={r['trial_converged']}, "
                            f"|FD-DF|={r['trial_grad']:.2e})"},
        "roofline": roof,
        "rooflines_by_phase": roofs,
        "launch_mode": "CUDA graph per block of steps" if r["graph"] else "kernel by kernel",
        "energy_evals_per_s": w.nwalkers / r["s_energy"],
        "profiled_pass": {"ms_per_step": r["ms_profiled"] / K,
                          "note": "same K steps launched kernel by kernel with CUDA events "
                                  "around each phase; source of phases and roofline"},
        "phases_ms_per_step": {k: round(v["ms"] / K, 4) for k, v in r["phases"].items()},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "e2e": {"value": N * w.nwalkers * K / r["e2e_s"], "unit": "walker-steps/s",
                "h2d_bytes_per_step": r["h2d_bytes"] / K, "d2h_bytes_per_step": 16 / K,
                "includes": "afqmc_init from pinned host arrays (h1, L, trial upload and "
                            f"set-up), {K} steps, energy read back"},
        "energy": {"E": r["E"], "wsum": r["wsum"], "alive": int(r["info"].alive),
                   "E_T": r["info"].E_T, "nonfinite": int(r["info"].nonfinite)},
        "flops_per_walker_step": fl["total"],
    }
    if r["precision_report"]:
        line["precision_vs_fp64"] = r["precision_report"]
    if r.get("fp64"):
        line["fp64_same_gpu"] = r["fp64"]
    if r.get("bias"):
        line["bias_vs_fp64"] = r["bias"]
    if N == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample(w)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
