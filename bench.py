#!/usr/bin/env python3
"""Benchmark of the HICU hot path on GB300.

One step = one call of hicu_reconstruct (Algorithm 1 with centre-out stages: Gram,
principal subspace, JL-compressed descent steps with exact line search) on the
chosen workload.  The default line is the 3D knee-shaped volume (256 x 256 x 160,
8 coils, 5 x 5 x 5 kernel, n = 1000, rank 400; centre-out stage on the central
64 x 64 x 40 region: 10 outer iterations x 5 descent steps, p = 8; then full
k-space: 1 outer iteration x 20 descent steps, p = 8), i.e. 11 Gram + null-space
updates and 70 descent steps.  --workload brain / cine / batch give the other
configurations.  The metric is descent steps (GD iterations) per second.

  value   device time of K steps (CUDA events on the launch stream), inputs
          resident in HBM, L2 flushed between steps, max over ranks; no per-launch
          events inside this timed region (launches are only counted)
  e2e     the same call with pinned HOST input/output buffers: the library
          copies x0 and the mask in and the result out inside the timed call
  roofline  the kernel class with the largest device time: one reconstruction per
          class finds it, then a second pass of K steps brackets each of its
          launches with CUDA events on its launch stream
  accuracy  the timed split-BF16 reconstruction against the plain-FP32 GPU
          reconstruction of the same schedule, and both GPU forms against the FP64
          oracle on the workload scaled down with a shortened schedule
  cpu_baseline  the FP64 oracle on a bounded sample of the same workload,
          extrapolated to the schedule

Multi-GPU: replicas only (each rank reconstructs its own problem), no collective
on the data path; launched by torchrun with one process per GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "2d_brain_256"
# --workload name -> (synthetic problem, metric text); the knee volume is the default line
WORKLOADS = {
    "knee": ("knee3d_256x256x160", "HICU GD-iters/s (full hicu_reconstruct of one 256x256x160 8-coil volume)"),
    "brain": ("2d_brain_256", "HICU GD-iters/s (full hicu_reconstruct of one 256x256x8-coil slice)"),
    "cine": ("cine_192x144x24", "HICU GD-iters/s (full hicu_reconstruct of one 192x144x24-frame 8-coil cine)"),
    "dwi": ("msdwi_256_c32", "HICU GD-iters/s (full hicu_reconstruct of one 256x256 multi-shot diffusion slice, "
                             "4 shots x 8 coils, null space augmented with b0 null vectors)"),
}
# multi-shot diffusion slice: shots, coils per shot, b0 null vectors (Methods, Study IV)
DWI_SHOTS, DWI_COILS, DWI_Q0 = 4, 8, 40
# accuracy block: (scale-down factor per spatial axis, (iters, gd_steps, p) per stage) of the
# reconstruction compared with the FP64 oracle
ORACLE_CHECK = {"knee": (4, [(2, 2, 8), (1, 2, 8)]), "cine": (2, [(2, 2, 8), (1, 2, 8)]),
                "brain": (2, [(10, 5, 8), (2, 5, 32)]), "dwi": (4, [(3, 2, 8), (1, 4, 8)])}
UNIT = "GD-iters/s"
KERNEL_NAMES = {0: "gram", 1: "eig", 2: "conv_fp32", 3: "adjoint_fp32", 4: "jl", 5: "misc",
                6: "conv_tc", 7: "adjoint_tc", 8: "tridiag"}
# FP32 pipe: 152 SMs x 128 lanes, one FMA (2 flops) or one add/multiply per lane per clock
SMS, FP32_LANES = 152, 128
# Gram: each complex product conj(a) b is 4 real products, each formed exactly and accumulated in
# double-word arithmetic (1 multiply, 1 FMA for the error term, 8 adds of the two-sum): 40 FP32
# operations for the 8 algorithmic flops of one complex multiply-add (issued two per paired
# instruction; the FP32 pipe's operation rate is the bound)
GRAM_OPS_PER_CMAC = 40
# DRAM bytes (read + write) per launch from one ncu capture of the same kernel on the same
# workload (profiles/), averaged over the class's launches in one reconstruction (centre-region
# and full-size launches together, as the event timing averages them); a kernel changed since its
# capture has no entry.
NCU_TRAFFIC = {("knee3d_256x256x160", "conv_tc"): 293246606, ("knee3d_256x256x160", "adjoint_tc"): 570873406,
               ("knee3d_256x256x160", "gram"): 395651072}


def problem_seed(workload: str, rank: int) -> int:
    """Seed of the synthetic problem of a workload on a rank (replicas reconstruct different data)."""
    order = {"brain": 0, "cine": 1, "knee": 2, "dwi": 4}
    return 1000 * (1 + order[workload]) + rank


def workload_problem(workload: str, seed: int, scale: int = 1, sched=None):
    """(problem, b0 k-space or None) of a workload; `scale` shrinks the spatial axes and `sched`
    replaces the (iters, gd_steps, p) of its stages."""
    from synth.phantoms import make_msdwi, make_problem
    if workload == "dwi":
        n = 256 // scale
        pb, xb0 = make_msdwi(seed=seed, n=n, C=DWI_COILS, S=DWI_SHOTS)
    else:
        pb, xb0 = make_problem(WORKLOADS[workload][0], seed=seed, scale=scale), None
    if sched is not None:
        for st, (it, gd, p) in zip(pb.stages, sched):
            st.iters, st.gd_steps, st.p = it, gd, p
    return pb, xb0


def eig_kwargs(args, pb):
    """make_params keywords of the null-space route: the Gram and the principal subspace by
    tridiagonalisation (default), or the randomized SVD (Theory: rSVD) with l = r + max(r/2, 8)
    test vectors (at most n), warm started by the reconstruction."""
    if getattr(args, "eig_solver", "tridiag") != "rsvd":
        return {}
    n = pb.ncoil * pb.kernel[0] * pb.kernel[1] * pb.kernel[2]
    return {"eig_solver": "rsvd", "rsvd_cols": min(n, pb.rank + max(pb.rank // 2, 8)), "rsvd_seed": 23}


def dwi_q0_oracle(xb0):
    """The b0 null vectors Q0 (columns) by the oracle: the DWI_Q0 smallest eigenvectors of the b0
    Gram over the whole b0 k-space, kernel 5 x 5 over the coils."""
    from oracle import hicu_oracle as O
    C, nz, ny, nx = xb0.shape
    g0 = O.Geom((nx, ny, nz), C, (5, 5, 1))
    Q0, _ = O.nullspace(O.gram(xb0.astype(np.complex128), g0, O.full_region(g0)), g0.n - DWI_Q0)
    return Q0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def schedule(pb):
    return [(s.off, s.ext, s.iters, s.gd_steps, s.p) for s in pb.stages]


def gd_steps_per_recon(pb):
    return sum(s.iters * s.gd_steps for s in pb.stages)


def algorithmic_flops(pb, cls):
    """Algorithmic real flops per reconstruction for a kernel class (see design notes)."""
    C = pb.ncoil
    kx, ky, kz = pb.kernel
    n = C * kx * ky * kz
    tot = 0.0
    prev = pb.stages[0]
    for st in pb.stages:
        sx, sy, sz = (st.ext[a] if pb.circular[a] else st.ext[a] - pb.kernel[a] + 1 for a in range(3))
        s = sx * sy * sz
        if cls in (2, 6):   # two convolutions per step (H(y)Q~ and H(g)Q~), 8 n p s flops each
            tot += st.iters * st.gd_steps * 2 * 8.0 * n * st.p * s
        elif cls in (3, 7):  # one adjoint per step, same count
            tot += st.iters * st.gd_steps * 8.0 * n * st.p * s
        elif cls == 0 and st.iters > 0:
            # lag-form correlation: C^2 (2k-1)^d / 2 complex MACs per point of the previous outer
            # iteration's region: the previous stage's for a stage's first iteration, its own after
            points = prev.ext[0] * prev.ext[1] * prev.ext[2] + (st.iters - 1) * st.ext[0] * st.ext[1] * st.ext[2]
            lags = (2 * kx - 1) * (2 * ky - 1) * (2 * kz - 1)
            tot += 8.0 * (C * C * lags / 2.0) * points
        elif cls == 8:  # Householder tridiagonalisation of the n x n Hermitian Gram: 16 n^3 / 3
            tot += st.iters * 16.0 * n ** 3 / 3.0
        elif cls == 1:  # back-transformation of the r principal vectors: 8 n^2 r
            tot += st.iters * 8.0 * n * n * pb.rank
        if st.iters > 0:
            prev = st
    return tot


def _filter_len(pb):
    return pb.ncoil * pb.kernel[0] * pb.kernel[1] * pb.kernel[2]


def class_roofline(pb, wname, cls, ms, launches, recons, peaks):
    """Roofline of one kernel class from its summed event time `ms` over `launches` launches made by
    `recons` reconstructions: algorithmic work of those reconstructions / device time, against the
    peak of the pipe the kernel runs on."""
    fp32_ops = SMS * FP32_LANES * peaks.get("sm_max_mhz", 2070.0) * 1e6   # FP32 lane operations / s
    avg_s = ms / 1e3 / max(launches, 1)
    flops = algorithmic_flops(pb, cls) * recons
    ach = flops / max(ms / 1e3, 1e-12) / 1e12
    base = {"kernel": KERNEL_NAMES[cls], "avg_launch_us": avg_s * 1e6, "launches": launches}
    if cls in (6, 7):
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        base.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                     "peak_source": "measured bf16 cuBLAS GEMM, sustained (the kernel is timed inside a "
                                    "long reconstruction)",
                     "work": "8 n p s algorithmic flops per convolution (n p s complex MACs); the split-bf16 "
                             "form issues 4 tensor products per algorithmic one (hi and lo of the input "
                             "against [B_hi | B_lo])"})
    elif cls == 0:
        peak = fp32_ops * 8.0 / GRAM_OPS_PER_CMAC / 1e12
        base.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                     "peak_source": f"FP32 pipe {SMS} SMs x {FP32_LANES} lanes x max SM clock, "
                                    f"{GRAM_OPS_PER_CMAC} FP32 operations per double-word complex "
                                    "multiply-add (8 algorithmic flops)",
                     "work": "lag-form cross-correlation: C^2 (2k-1)^d / 2 complex MACs per region point "
                             "(8 flops each)"})
    elif cls in (2, 3):
        peak = 2.0 * fp32_ops / 1e12
        base.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                     "peak_source": "FP32 pipe, FMA = 2 flops, max SM clock",
                     "work": "8 n p s flops per convolution"})
    elif cls == 8:
        n = _filter_len(pb)
        per_step_us = avg_s * 1e6 / max(n - 2, 1)
        base.update({"bound": "latency", "achieved": per_step_us, "unit": "us per Householder step",
                     "peak": None, "frac": None, "n": n,
                     "algorithmic_tflops": ach,
                     "work": "16 n^3 / 3 flops per tridiagonalisation in n - 2 dependent Householder steps, "
                             "one barrier each, double-float arithmetic on the FP32 pipe"})
    else:
        base.update({"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None})
    tr = NCU_TRAFFIC.get((wname, base["kernel"]))
    base["traffic"] = tr
    if tr is not None:
        base["traffic_unit"] = "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    return base


def roofline_block(pb, wname, cls, ms, launches, eig_sweeps, recons, peaks, peak_src):
    r = class_roofline(pb, wname, cls, ms, launches, recons, peaks)
    r["peaks_source"] = peak_src
    r["timing"] = f"CUDA events around each launch of the class on its launch stream, {recons} reconstructions"
    if cls == 1 and eig_sweeps:
        r["jacobi_sweeps"] = eig_sweeps
    return r


def kernel_rooflines(pb, wname, per_class, peaks):
    out = {}
    for c in (6, 7, 0, 8, 2, 3):
        ms, nl = per_class.get(c, (0.0, 0))
        if nl:
            out[KERNEL_NAMES[c]] = class_roofline(pb, wname, c, ms, nl, 1, peaks)
    return out


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(",") for r in self.tmp.read().strip().splitlines() if r.strip()]
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------- rank aggregation

def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device) -> float:
    """The largest value over the ranks of the process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank_step * steps * world / seconds


# ------------------------------------------------------------------ oracle arm

def _slab(reg, geom, kernel, circular, max_out):
    """A region covering the first slab of `reg` (outermost non-trivial axis cut) whose valid
    outputs number about max_out; returns (region, fraction of reg's outputs)."""
    from oracle import hicu_oracle as O
    full = O.num_outputs(geom, reg)
    if full <= max_out:
        return reg, 1.0
    ax = 2 if reg.ext[2] > 1 else 1
    k = kernel[ax]
    out_ax = reg.ext[ax] if circular[ax] else reg.ext[ax] - k + 1
    keep = max(1, int(out_ax * max_out / full))
    ext = list(reg.ext)
    if circular[ax]:
        # a circular axis cannot be cut without changing the problem: keep it and cut y instead
        ax = 1
        k = kernel[1]
        out_ax = reg.ext[1] - k + 1
        keep = max(1, int(out_ax * max_out / full))
    ext[ax] = keep + (0 if circular[ax] else k - 1)
    sub = O.Region(tuple(reg.off), tuple(ext))
    return sub, O.num_outputs(geom, sub) / full


def oracle_sample(pb, seed=11, max_outputs=40000, target_s=10.0):
    """Time the FP64 oracle on a bounded sample of one reconstruction and extrapolate.

    Units timed: the Gram matrix of each stage's null-space region (Algorithm 1 step 2 reads
    H^(i-1): the first iteration of a stage uses the previous stage's region), one eigh, and
    one descent step on each stage's region.  A Gram or a step whose valid outputs exceed
    max_outputs runs on a slab of the region and its time is scaled by the ratio of outputs
    (both costs are linear in them).  The reconstruction is the sum over stages of iters x
    (Gram + eigh + gd_steps x step).  The sample is repeated until it has taken target_s of CPU
    time (at most 50 times) and the median extrapolation is kept.  Returns (GD-iters/s, CPU
    seconds of the sample, description).
    """
    from oracle import hicu_oracle as O
    og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    x = O.initial_estimate(pb.x0.astype(np.complex128), pb.mask,
                           "time_average" if pb.init == "time_average" else "zero_filled")
    total_s, recons, scaled = 0.0, [], False
    while True:
        sample_s = 0.0
        cache = {}

        def timed(kind, reg):
            nonlocal sample_s, scaled
            key = (kind, tuple(reg.off), tuple(reg.ext))
            if key in cache:
                return cache[key]
            sub, frac = _slab(reg, og, pb.kernel, pb.circular, max_outputs)
            scaled = scaled or frac < 1.0
            t0 = time.perf_counter()
            if kind == "gram":
                cache["G"] = O.gram(x, og, sub)
            else:
                f = O.as_filters(O.jl_compress(Q, O.jl_matrix(seed, 0, og.n, 8), "projector"), og)
                O.gd_step(x, pb.mask, og, sub, f)
            dt = time.perf_counter() - t0
            sample_s += dt
            cache[key] = dt / frac
            return cache[key]

        timed("gram", O.Region(pb.stages[0].off, pb.stages[0].ext))
        t0 = time.perf_counter()
        Q, _ = O.nullspace(cache["G"], pb.rank)
        t_eigh = time.perf_counter() - t0
        sample_s += t_eigh
        t_recon = 0.0
        prev = pb.stages[0]
        for st in pb.stages:
            rst = O.Region(st.off, st.ext)
            t_first = timed("gram", O.Region(prev.off, prev.ext))
            t_rest = timed("gram", rst) if st.iters > 1 else 0.0
            t_step = timed("step", rst)
            # the step above uses p = 8 filters; the step's cost is linear in p
            t_step *= st.p / 8.0
            t_recon += t_first + (st.iters - 1) * t_rest + st.iters * (t_eigh + st.gd_steps * t_step)
            prev = st
        recons.append(t_recon)
        total_s += sample_s
        if total_s >= target_s or len(recons) >= 50:
            break
    t_recon = statistics.median(recons)
    slab = " (large regions on slabs, times scaled by their share of outputs)" if scaled else ""
    desc = (f"per-stage Gram, one eigh (n={og.n}) and one descent step per stage{slab}, "
            f"{len(recons)} repetitions, {total_s:.1f} s of CPU, median extrapolated to the "
            f"{gd_steps_per_recon(pb)}-step schedule")
    return gd_steps_per_recon(pb) / t_recon, total_s, desc


def schedule_text(pb):
    def reg(st):
        if tuple(st.off) == (0, 0, 0) and tuple(st.ext) == tuple(pb.dims):
            return "full"
        return ("CO " if tuple(st.off) != (0,) * 3 and st.ext[1] < pb.dims[1] // 2 else "region ") + \
            "x".join(str(e) for e in st.ext if e > 1)
    return " + ".join(f"{reg(st)} {st.iters}x{st.gd_steps} p={st.p}" for st in pb.stages)


def workload_config(name, pb):
    kx, ky, kz = pb.kernel
    dims = "x".join(str(d) for d in pb.dims if d > 1)
    return {"workload": name, "image": dims, "coils": pb.ncoil,
            "kernel": "x".join(str(k) for k in pb.kernel if k > 1), "rank": pb.rank,
            "circular": "".join("xyz"[a] for a in range(3) if pb.circular[a]) or "none",
            "schedule": schedule_text(pb)}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads", 0) for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args, rank, world):
    """The oracle arm: every step is one bounded sample of the workload (per stage the Gram of its
    null-space region, one eigh and one descent step, regions above 10 000 valid outputs cut to a
    slab), timed on the host cores; `value` is the GD-iters/s of the whole schedule extrapolated
    from the sample (median over the timed steps), `ms_per_step` the measured time of one sample."""
    if rank != 0:
        return 0
    from synth.phantoms import make_problem
    wname, metric = WORKLOADS[args.workload]
    pb, _ = workload_problem(args.workload, problem_seed(args.workload, 0))
    vals, descs, step_s = [], [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, _, desc = oracle_sample(pb, max_outputs=10000, target_s=0.0)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(v)
            descs.append(desc)
            step_s.append(dt)
    value = statistics.median(vals)
    cores = blas_threads()
    sample = "per step: " + descs[-1]
    config = workload_config(wname, pb)
    config.update({"l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"})
    ekw = eig_kwargs(args, pb)
    config["null_space"] = (f"randomized SVD, l = {ekw['rsvd_cols']} (warm started)" if ekw
                            else "Gram + principal subspace by tridiagonalisation")
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_s) / len(step_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "extrapolated": True,
            "extrapolated_ms_per_reconstruction": 1e3 * gd_steps_per_recon(pb) / value,
            "note": "ms_per_step is the measured time of one bounded oracle sample; value is the "
                    "schedule's GD-iters/s extrapolated from it",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- profiling cases

def run_profile_case(kind: str, size: int) -> int:
    """Small fixed workloads for ncu captures of one kernel (no timing, no JSON line).

    eig / eig_cluster: the brain slice's Gram (n = 200), one cold solve then one warm
        split-criterion solve of a perturbed Gram on the grid / cluster solver (the warm one
        is the launch a reconstruction repeats: capture with -s 1 -c 1)
    tc_step: one split-BF16 descent step on a size x size x 8-coil slice, p = 32
    tc_step3d: one split-BF16 descent step on the knee-shaped 256 x 256 x 160 x 8-coil volume
        (5 x 5 x 5 kernel, p = 8); each step launches conv, adjoint, conv
    fgrad: the filter gradient H(x)^H R on the brain slice, p = 32
    principal: the principal subspace (tridiagonalisation path) of the brain slice's centre-region
        Gram (n = 200, r = 75) and of the cine workload's centre-region Gram (n = 1000, r = 300),
        twice each
    recon: one full reconstruction of the brain slice (for the launch list)
    recon_knee: one full reconstruction of the knee volume (for the launch list)
    gram_knee: the Gram of the knee volume's centre region (n = 1000), twice
    """
    import torch
    from paper_2004_08962_gb300 import build, hicu
    from synth.phantoms import _slice_2d, make_problem
    build.build()
    h = hicu.Handle()
    pb = make_problem(WORKLOAD)
    geom = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel)
    reg = hicu.make_region((0, 0, 0), pb.dims)
    if kind in ("eig", "eig_cluster"):
        solver = "grid" if kind == "eig" else "cluster"
        G = hicu.hicu_gram(h, geom, reg, torch.from_numpy(pb.x0).cuda())
        hicu.hicu_nullspace(h, G, pb.rank, split=True, solver=solver)
        rng = np.random.default_rng(3)
        E = torch.from_numpy(rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape)).cuda()
        G2 = G + (E + E.conj().T) * (1e-4 * G.abs().max())
        hicu.hicu_nullspace(h, G2, pb.rank, warm=True, split=True, solver=solver)
    elif kind == "tc_step":
        rng = np.random.default_rng(7)
        k, mask = _slice_2d(rng, size, 8, 4.0, n_ellipses=20)
        x = torch.from_numpy(k).cuda()
        m = torch.from_numpy(mask).cuda()
        g2 = hicu.make_geom((size, size, 1), 8, (5, 5, 1))
        r2 = hicu.make_region((0, 0, 0), (size, size, 1))
        f = torch.from_numpy((rng.standard_normal((32, 200)) + 1j * rng.standard_normal((32, 200)))
                             .astype(np.complex64) * 0.05).cuda()
        for _ in range(2):
            hicu.hicu_gd_step_filters(h, g2, r2, x, m, f, prec=hicu.HICU_SPLIT_BF16)
    elif kind == "tc_step3d":
        g3 = hicu.make_geom((256, 256, 160), 8, (5, 5, 5))
        r3 = hicu.make_region((0, 0, 0), (256, 256, 160))
        gen = torch.Generator(device="cuda").manual_seed(7)
        x = torch.randn((8, 160, 256, 256), dtype=torch.complex64, device="cuda", generator=gen)
        m = (torch.rand((160, 256, 256), device="cuda", generator=gen) < 0.2).to(torch.uint8)
        f = torch.randn((8, 1000), dtype=torch.complex64, device="cuda", generator=gen) * 0.03
        for _ in range(2):
            hicu.hicu_gd_step_filters(h, g3, r3, x, m, f, prec=hicu.HICU_SPLIT_BF16)
    elif kind == "principal":
        for name in (WORKLOAD, "cine_192x144x24"):
            pq = make_problem(name)
            gq = hicu.make_geom(pq.dims, pq.ncoil, pq.kernel, pq.circular)
            st = pq.stages[0]
            G = hicu.hicu_gram(h, gq, hicu.make_region(st.off, st.ext), torch.from_numpy(pq.x0).cuda())
            for _ in range(2):
                hicu.hicu_principal_subspace(h, G, pq.rank)
    elif kind == "fgrad":
        rng = np.random.default_rng(8)
        x = torch.from_numpy(pb.x0).cuda()
        Rb = torch.from_numpy((rng.standard_normal(hicu.out_shape(geom, reg) + (32,)) + 0j)
                              .astype(np.complex64)).cuda()
        for _ in range(2):
            hicu.hicu_conv_null_filter_grad(h, geom, reg, x, Rb)
    elif kind == "recon":
        params = hicu.make_params(pb.rank, schedule(pb), seed=11, jl=hicu.HICU_JL_PROJECTOR,
                                  prec=hicu.HICU_SPLIT_BF16)
        hicu.hicu_reconstruct(h, geom, torch.from_numpy(pb.x0).cuda(), torch.from_numpy(pb.mask).cuda(),
                              params)
    elif kind in ("recon_knee", "gram_knee"):
        pk = make_problem("knee3d_256x256x160", seed=problem_seed("knee", 0))
        gk = hicu.make_geom(pk.dims, pk.ncoil, pk.kernel, pk.circular)
        xk = torch.from_numpy(pk.x0).cuda()
        if kind == "recon_knee":
            params = hicu.make_params(pk.rank, schedule(pk), seed=11, jl=hicu.HICU_JL_PROJECTOR,
                                      prec=hicu.HICU_SPLIT_BF16)
            hicu.hicu_reconstruct(h, gk, xk, torch.from_numpy(pk.mask).cuda(), params)
        else:
            st = pk.stages[0]
            for _ in range(2):
                hicu.hicu_gram(h, gk, hicu.make_region(st.off, st.ext), xk)
    else:
        raise SystemExit(f"unknown profile case {kind}")
    torch.cuda.synchronize()
    hicu.hicu_check(h)
    h.close()
    print(f"profile case {kind} done")
    return 0


# ------------------------------------------------------------ batched workload

BATCH_METRIC = "HICU GD-iters/s (batched: 48 uneven 2D slices + 4 multi-shot 32-channel slices)"


def run_batch(args, rank, world):
    """The uneven batch (48 slices of 128^2..320^2 x 4..16 coils at R 3..5, plus 4 multi-shot
    256^2 slices stacked as 32 channels) through hicu_reconstruct_batched: aggregate descent
    steps per second, per-slice steps per second and completion latency percentiles, and the
    FP64 oracle's reconstruction of the cheapest slice for the NRMSE / SER check."""
    import torch
    from paper_2004_08962_gb300 import build, hicu
    from synth.phantoms import make_batch

    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    barrier()
    batch = make_batch(seed=4000 + 97 * rank)   # replicas: each rank reconstructs its own batch
    prec = hicu.HICU_FP32 if args.prec == "fp32" else hicu.HICU_SPLIT_BF16
    h = hicu.Handle()
    probs, outs, x0s, masks = [], [], [], []
    for pb in batch:
        per_coil = pb.mask.ndim == 4
        geom = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, mask_per_coil=per_coil)
        prm = hicu.make_params(pb.rank, schedule(pb), seed=pb.seed, jl=hicu.HICU_JL_PROJECTOR, prec=prec)
        x0 = torch.from_numpy(pb.x0).cuda()
        m = torch.from_numpy(pb.mask).cuda()
        out = torch.empty_like(x0)
        probs.append(hicu.make_problem_struct(geom, x0, m, prm, out))
        outs.append(out)
    steps_total = sum(gd_steps_per_recon(pb) for pb in batch)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        hicu.hicu_reconstruct_batched(h, probs, lanes=args.lanes)
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    barrier()
    sampler.start()
    hicu.hicu_profile_select(h, -1)
    _, _, launches0 = hicu.hicu_profile_read(h)
    stream = torch.cuda.current_stream()
    total_ms, reports = 0.0, []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep, _ = hicu.hicu_reconstruct_batched(h, probs, lanes=args.lanes)
        e1.record(stream)    # the call returns after every lane finished
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        reports.append(rep)
    _, _, launches1 = hicu.hicu_profile_read(h)
    barrier()
    clocks = sampler.stop()
    value = job_rate(steps_total, args.steps, world, max_over_ranks(total_ms, "cuda") / 1e3)
    if rank != 0:
        barrier()
        if world > 1:
            dist.destroy_process_group()
        h.close()
        return 0
    lat = [r["end_ms"] for rep in reports for r in rep]
    per_slice = [r["gd_steps"] / ((r["end_ms"] - r["start_ms"]) / 1e3) for rep in reports for r in rep]
    pct = lambda v, q: float(np.percentile(np.asarray(v), q))
    line = {"metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "bf16x2",
            "data": "synthetic",
            "config": {"workload": "batch_uneven_52", "slices": len(batch), "lanes": args.lanes,
                       "gd_steps_per_batch": steps_total,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "per_slice_gd_iters_per_s": {"p50": pct(per_slice, 50), "min": min(per_slice),
                                         "max": max(per_slice)},
            "completion_latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat)},
            "gpu_launches": (launches1 - launches0) // max(args.steps, 1),
            "clocks": clocks}
    if not args.no_cpu_baseline and world == 1:
        # FP64 oracle on the cheapest slice of the batch: NRMSE / SER of the GPU result, and its time
        from oracle import hicu_oracle as O
        order, cost = hicu.hicu_batch_order(probs)
        i = order[-1]
        pb = batch[i]
        og = O.Geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
        st = [O.StageSpec(O.Region(s.off, s.ext), s.iters, s.gd_steps, s.p) for s in pb.stages]
        t0 = time.perf_counter()
        ref = O.reconstruct(pb.x0, pb.mask, og, st, pb.rank, seed=pb.seed, jl_mode="projector")
        t_or = time.perf_counter() - t0
        x = outs[i].cpu().numpy()
        line["oracle_check"] = {"slice": pb.name, "nrmse": float(np.linalg.norm(x - ref) / np.linalg.norm(ref)),
                                "ser_db_gpu": O.ser_db(pb.x_full, x), "ser_db_oracle": O.ser_db(pb.x_full, ref)}
        line["cpu_baseline"] = {"value": gd_steps_per_recon(pb) / t_or, "unit": UNIT, "cores": blas_threads(),
                                "kind": "oracle", "sample": f"full reconstruction of the cheapest slice "
                                                            f"({pb.name}, {t_or:.1f} s of CPU)"}
    print(json.dumps(line), flush=True)
    barrier()
    if world > 1:
        dist.destroy_process_group()
    h.close()
    return 0


# ------------------------------------------------------------------- ablations

def run_ablation(args):
    """The JL p-sweep and the CO x JL ablation of the paper's Study I (Results, the JL / CO figure),
    re-run on the synthetic 2D brain slice.  For every variant the schedule is cut after a growing
    number of outer iterations; each cut reconstruction is timed with CUDA events (L2 flushed before
    it) and scored by its SER against the fully sampled k-space, giving SER against time.
      p sweep : p in {1, 2, 4, 8, 32, n - r} in both stages, and no compression (exact gradient)
      CO x JL : centre-out schedule or full k-space from the first iteration, JL (p = 8 / 32) or
                exact gradient
    Every variant runs the plain complex-FP32 convolutions: without compression (n filters) and at
    p = n - r the filter bank is larger than the split-BF16 adjoint keeps in shared memory, and one
    form for all keeps the times comparable.  Prints one JSON object."""
    import torch
    from oracle import hicu_oracle as O
    from paper_2004_08962_gb300 import build, hicu
    from synth.phantoms import make_problem
    build.build()
    pb = make_problem("2d_brain_256", seed=problem_seed("brain", 0))
    n = pb.ncoil * pb.kernel[0] * pb.kernel[1] * pb.kernel[2]
    h = hicu.Handle()
    geom = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
    x0 = torch.from_numpy(pb.x0).cuda()
    mask = torch.from_numpy(pb.mask).cuda()
    out = torch.empty_like(x0)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    prec = hicu.HICU_FP32
    co, full = pb.stages[0], pb.stages[1]
    cuts = [1, 5, 10, 20, 30, 40, 50, 52, 55, 60]

    def stages_for(co_on, p1, p2, upto):
        st = [((co.off, co.ext) if co_on else ((0, 0, 0), pb.dims)) + (co.iters, co.gd_steps, p1),
              ((0, 0, 0), pb.dims, full.iters, full.gd_steps, p2)]
        outp, left = [], upto
        for off, ext, it, gd, p in st:
            k = min(it, left)
            if k > 0:
                outp.append((off, ext, k, gd, p))
            left -= k
        return outp

    def curve(co_on, p1, p2, exact):
        pts = []
        for c in cuts:
            prm = hicu.make_params(pb.rank, stages_for(co_on, p1, p2, c), seed=11, jl=hicu.HICU_JL_PROJECTOR,
                                   prec=prec, jl_exact=exact)
            hicu.hicu_reconstruct(h, geom, x0, mask, prm, x_out=out)   # warm
            ms = timed_recons(lambda: hicu.hicu_reconstruct(h, geom, x0, mask, prm, x_out=out), 1, flush, stream)
            steps = sum(it * gd for _, _, it, gd, _ in stages_for(co_on, p1, p2, c))
            pts.append({"outer_iters": c, "gd_steps": steps, "ms": round(ms, 3),
                        "ser_db": round(O.ser_db(pb.x_full, out.cpu().numpy()), 4)})
        return pts

    res = {"ablation": "JL p-sweep and CO x JL on the synthetic 2D brain slice (256x256, 8 coils, 5x5, r = 75)",
           "prec": "fp32", "ser_db_zero_filled": round(O.ser_db(pb.x_full, pb.x0), 4),
           "schedule": "CO 64x64 50x5, then full 10x10; p applied to both stages", "p_sweep": [], "co_jl": []}
    for p in (1, 2, 4, 8, 32, n - pb.rank):
        res["p_sweep"].append({"p": p, "curve": curve(True, p, p, False)})
    res["p_sweep"].append({"p": "exact (no JL)", "curve": curve(True, 1, 1, True)})
    for co_on in (True, False):
        for jl_on in (True, False):
            res["co_jl"].append({"co": co_on, "jl": jl_on, "curve": curve(co_on, 8, 32, not jl_on)})
    torch.cuda.synchronize()
    hicu.hicu_check(h)
    h.close()
    print(json.dumps(res), flush=True)
    return 0


def run_nullspace_compare(args):
    """Time one null-space update (Algorithm 1 steps 2-3) by the two routes on the centre-out
    regions of the brain slice (n = 200, r = 75), the multi-shot diffusion slice (n = 800, r = 45)
    and the knee volume (n = 1000, r = 400):
      gram   : the lag-form Gram (hicu_gram) and the principal subspace by Householder
               tridiagonalisation (hicu_principal_subspace)
      rsvd   : the randomized SVD (hicu_principal_rsvd) with l = r + max(r/2, 8) test vectors, warm
               started from the previous call's vectors (the reconstruction's steady state)
    CUDA events around each call, median of 5 after a warm-up; the distance between the two
    subspaces (spectral norm of the projector difference) and each route's J.  One JSON object."""
    import torch
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    h = hicu.Handle()
    out = {"nullspace_compare": "one null-space update by the Gram route and by the randomized SVD", "cases": []}
    for wl in ("brain", "dwi", "knee"):
        pb, _ = workload_problem(wl, problem_seed(wl, 0))
        st = pb.stages[0]
        geom = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular)
        reg = hicu.make_region(st.off, st.ext)
        x = torch.from_numpy(pb.x0).cuda()
        r = pb.rank
        n = pb.ncoil * pb.kernel[0] * pb.kernel[1] * pb.kernel[2]
        l = min(n, r + max(r // 2, 8))

        def timed(fn, reps=5):
            fn()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                res = fn()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts), res

        def gram_route():
            G = hicu.hicu_gram(h, geom, reg, x)
            return hicu.hicu_principal_subspace(h, G, r, want_tail=True)

        t_gram, (Vg, eg, Jg) = timed(gram_route)
        Vr, er, Jr = hicu.hicu_principal_rsvd(h, geom, reg, x, r, l, seed=7, counter=0, want_tail=True)
        state = {"V": Vr, "k": 1}

        def rsvd_route():
            V, e, J = hicu.hicu_principal_rsvd(h, geom, reg, x, r, l, V_prev=state["V"], seed=7, counter=state["k"],
                                               want_tail=True)
            state["V"], state["k"] = V, state["k"] + 1
            return V, e, J

        t_rsvd, (Vr, er, Jr) = timed(rsvd_route)
        A, B = Vg.cpu().numpy().T, Vr.cpu().numpy().T
        dist = float(np.linalg.norm(A @ A.conj().T - B @ B.conj().T, 2))
        out["cases"].append({"workload": WORKLOADS[wl][0], "n": n, "r": r, "l": l,
                             "region": "x".join(str(e) for e in st.ext if e > 1),
                             "gram_route_ms": round(t_gram, 3), "rsvd_ms": round(t_rsvd, 3),
                             "subspace_distance": dist, "J_gram": float(Jg.item()), "J_rsvd": float(Jr.item())})
    hicu.hicu_check(h)
    h.close()
    print(json.dumps(out), flush=True)
    return 0


# -------------------------------------------------------------------- GPU arm

def timed_recons(one, steps, flush, stream):
    """Device time (ms) of `steps` reconstructions: CUDA events on the launch stream around each
    call, L2 flushed before each (outside the events), synchronised on both sides."""
    import torch
    total = 0.0
    torch.cuda.synchronize()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    return total


def accuracy_block(args, pb, hicu, h, geom, x_bf16, x_fp32):
    """NRMSE / SER of the timed split-BF16 reconstruction against the plain-FP32 GPU reconstruction
    of the same schedule, and (the full-size oracle reconstruction would take hours) both GPU
    forms against the FP64 oracle on the workload scaled down with a shortened schedule."""
    import torch
    from oracle import hicu_oracle as O
    from synth.phantoms import make_problem
    out = {}
    if x_bf16 is not None and x_fp32 is not None:
        out["split_bf16_vs_plain_fp32"] = {
            "nrmse": float(np.linalg.norm(x_bf16 - x_fp32) / np.linalg.norm(x_fp32)),
            "ser_db_split_bf16": O.ser_db(pb.x_full, x_bf16), "ser_db_plain_fp32": O.ser_db(pb.x_full, x_fp32),
            "ser_db_zero_filled": O.ser_db(pb.x_full, pb.x0)}
    if args.no_oracle_check:
        return out
    name = WORKLOADS[args.workload][0]
    scale, sched = ORACLE_CHECK[args.workload]
    ps, xb0 = workload_problem(args.workload, problem_seed(args.workload, 0), scale=scale, sched=sched)
    stages = [(st.off, st.ext, st.iters, st.gd_steps, st.p) for st in ps.stages]
    init = 1 if ps.init == "time_average" else 0
    og = O.Geom(ps.dims, ps.ncoil, ps.kernel, ps.circular)
    ost = [O.StageSpec(O.Region(off, ext), it, gd, p) for off, ext, it, gd, p in stages]
    Q0 = dwi_q0_oracle(xb0) if xb0 is not None else None
    ekw = eig_kwargs(args, ps)
    t0 = time.perf_counter()
    ref = O.reconstruct(ps.x0, ps.mask, og, ost, ps.rank, seed=5, jl_mode="projector", init=ps.init,
                        qplus=None if Q0 is None else (Q0, DWI_SHOTS),
                        rsvd=(ekw["rsvd_cols"], ekw["rsvd_seed"]) if ekw else None)
    t_or = time.perf_counter() - t0
    gs = hicu.make_geom(ps.dims, ps.ncoil, ps.kernel, ps.circular, mask_per_coil=ps.mask.ndim == 4)
    q0t = None if Q0 is None else torch.from_numpy(np.ascontiguousarray(Q0.T)).cuda()
    res = {"workload": f"{name} scaled 1/{scale} per spatial axis ({'x'.join(str(d) for d in ps.dims if d > 1)})",
           "schedule": " + ".join(f"{it}x{gd} p={p}" for it, gd, p in sched), "oracle_s": t_or,
           "ser_db_oracle": O.ser_db(ps.x_full, ref)}
    for tag, prec in (("split_bf16", hicu.HICU_SPLIT_BF16), ("plain_fp32", hicu.HICU_FP32)):
        prm = hicu.make_params(ps.rank, stages, seed=5, jl=hicu.HICU_JL_PROJECTOR, prec=prec, init=init,
                               qplus=q0t, qplus_blocks=DWI_SHOTS if q0t is not None else 0, **ekw)
        x = hicu.hicu_reconstruct(h, gs, torch.from_numpy(ps.x0).cuda(), torch.from_numpy(ps.mask).cuda(),
                                  prm).cpu().numpy()
        res[tag] = {"nrmse": float(np.linalg.norm(x - ref) / np.linalg.norm(ref)),
                    "max_abs_err_rel": float(np.max(np.abs(x - ref)) / np.max(np.abs(ref))),
                    "ser_db": O.ser_db(ps.x_full, x)}
    res["bounds"] = "NRMSE <= 1e-3 and SER within 0.05 dB of the oracle's"
    res["pass"] = all(res[t]["nrmse"] <= 1e-3 and abs(res[t]["ser_db"] - res["ser_db_oracle"]) <= 0.05
                      for t in ("split_bf16", "plain_fp32"))
    out["oracle_check"] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hicu", choices=["hicu", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the scaled-down oracle reconstruction of the accuracy block")
    ap.add_argument("--profile", default=None, choices=["eig", "eig_cluster", "tc_step", "tc_step3d", "principal",
                                                        "fgrad", "recon", "recon_knee", "gram_knee"],
                    help="run one small fixed case for an ncu capture and exit")
    ap.add_argument("--size", type=int, default=2048, help="image size of the tc_step profile case")
    ap.add_argument("--workload", default="knee", choices=["knee", "brain", "cine", "dwi", "batch"],
                    help="knee: 256x256x160 x 8 coils, 5x5x5 kernel (default line); brain: the 256x256x8 "
                         "slice; cine: 192x144x24 frames x 8 coils, 5x5x5 kernel, circular time; dwi: a "
                         "256x256 multi-shot diffusion slice (4 shots x 8 coils, augmented null space, "
                         "partial-Fourier final region); batch: the uneven 52-slice batch")
    ap.add_argument("--lanes", type=int, default=8, help="worker lanes of the batched workload")
    ap.add_argument("--ablation", action="store_true",
                    help="the JL p-sweep and CO x JL ablation on the brain slice (one JSON object, no bench line)")
    ap.add_argument("--nullspace-compare", action="store_true",
                    help="time one null-space update by the Gram route and by the randomized SVD "
                         "(brain, diffusion, knee)")
    ap.add_argument("--eig-solver", default="tridiag", choices=["tridiag", "rsvd"],
                    help="null-space route of the timed reconstruction: the Gram and the principal subspace "
                         "by tridiagonalisation, or the randomized SVD (its oracle check uses the oracle's "
                         "randomized SVD)")
    args = ap.parse_args()
    if args.eig_solver != "tridiag" and args.impl == "reference":
        ap.error("--eig-solver rsvd times the library's route; the reference arm samples the oracle's Gram route")
    if args.profile:
        return run_profile_case(args.profile, args.size)
    if args.ablation:
        return run_ablation(args)
    if args.nullspace_compare:
        return run_nullspace_compare(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.workload == "batch":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the reference arm times the oracle on single-problem workloads only"}))
            return 0
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world)
    wname, metric = WORKLOADS[args.workload]

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2004_08962_gb300 import build, hicu
    from synth.phantoms import make_problem

    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    pb, xb0 = workload_problem(args.workload, problem_seed(args.workload, rank))
    prec = hicu.HICU_FP32 if args.prec == "fp32" else hicu.HICU_SPLIT_BF16
    h = hicu.Handle()
    geom = hicu.make_geom(pb.dims, pb.ncoil, pb.kernel, pb.circular, mask_per_coil=pb.mask.ndim == 4)
    init = 1 if pb.init == "time_average" else 0
    q0, q0_ms = None, None
    if xb0 is not None:
        # the b0 null vectors: Gram and null space of the b0 k-space on the GPU (once per slice,
        # before the reconstruction; timed separately)
        c0 = xb0.shape[0]
        g0 = hicu.make_geom(pb.dims, c0, (5, 5, 1))
        xb0_t = torch.from_numpy(xb0).cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G0 = hicu.hicu_gram(h, g0, hicu.make_region((0, 0, 0), pb.dims), xb0_t)
        n0 = c0 * 25
        q0, _ = hicu.hicu_nullspace(h, G0, n0 - DWI_Q0)
        e1.record()
        e1.synchronize()
        q0_ms = e0.elapsed_time(e1)
    params = hicu.make_params(pb.rank, schedule(pb), seed=11, jl=hicu.HICU_JL_PROJECTOR, prec=prec, init=init,
                              qplus=q0, qplus_blocks=DWI_SHOTS if q0 is not None else 0, **eig_kwargs(args, pb))
    x0 = torch.from_numpy(pb.x0).cuda()
    mask = torch.from_numpy(pb.mask).cuda()
    xout = torch.empty_like(x0)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()
    steps_per = gd_steps_per_recon(pb)

    def one():
        hicu.hicu_reconstruct(h, geom, x0, mask, params, x_out=xout)

    for _ in range(args.warmup):
        one()

    # timed region: no per-launch events (profiling off); launches are only counted
    hicu.hicu_profile_select(h, -1)
    hicu.hicu_profile_read(h)
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler.start()
    total_ms = timed_recons(one, args.steps, flush, stream)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    _, _, all_launches = hicu.hicu_profile_read(h)
    tmax_s = max_over_ranks(total_ms, "cuda") / 1e3
    value = job_rate(steps_per, args.steps, world, tmax_s)
    x_main = xout.cpu().numpy() if rank == 0 else None

    # class times, one reconstruction per kernel class with events around that class's launches
    classes = [0, 1, 2, 3, 4, 5, 6, 7, 8]
    per_class = {}
    for c in classes:
        hicu.hicu_profile_select(h, c)
        one()
        ms, nl, _ = hicu.hicu_profile_read(h)
        per_class[c] = (ms, nl)
    hicu.hicu_profile_select(h, -1)
    dominant = max(per_class, key=lambda c: per_class[c][0])
    # roofline pass: the same K reconstructions with events around every launch of the dominant class
    hicu.hicu_profile_select(h, dominant)
    hicu.hicu_profile_eig_sweeps(h)
    roof_total_ms = timed_recons(one, args.steps, flush, stream)
    dom_ms, dom_launches, _ = hicu.hicu_profile_read(h)
    eig_sweeps = hicu.hicu_profile_eig_sweeps(h)
    hicu.hicu_profile_select(h, -1)

    # the plain complex-FP32 form of the same reconstruction, same timing rules
    fp32_ms, fp32_steps, x_fp32 = None, 0, None
    if args.prec == "bf16":
        params32 = hicu.make_params(pb.rank, schedule(pb), seed=11, jl=hicu.HICU_JL_PROJECTOR,
                                    prec=hicu.HICU_FP32, init=init, qplus=q0,
                                    qplus_blocks=DWI_SHOTS if q0 is not None else 0, **eig_kwargs(args, pb))
        out32 = torch.empty_like(x0)
        one32 = lambda: hicu.hicu_reconstruct(h, geom, x0, mask, params32, x_out=out32)
        one32()
        fp32_steps = min(args.steps, 5)
        fp32_ms = timed_recons(one32, fp32_steps, flush, stream)
        x_fp32 = out32.cpu().numpy() if rank == 0 else None
    fp32_value = None if fp32_ms is None else job_rate(steps_per, fp32_steps, world,
                                                        max_over_ranks(fp32_ms, "cuda") / 1e3)

    # end-to-end through the C ABI with pinned host buffers (copies inside the call)
    x0h = torch.from_numpy(pb.x0).pin_memory()
    mh = torch.from_numpy(pb.mask).pin_memory()
    outh = torch.empty_like(x0h).pin_memory()
    hicu.hicu_reconstruct(h, geom, x0h, mh, params, x_out=outh)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hicu.hicu_reconstruct(h, geom, x0h, mh, params, x_out=outh)
        e2e_s += time.perf_counter() - t0
    e2e_value = job_rate(steps_per, args.steps, world, max_over_ranks(e2e_s, "cuda"))
    h2d = pb.x0.nbytes + pb.mask.nbytes
    d2h = pb.x0.nbytes

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    roof = roofline_block(pb, wname, dominant, dom_ms, dom_launches, eig_sweeps, args.steps, peaks, peak_src)
    roof["timed_pass_ms_per_step"] = roof_total_ms / args.steps
    extra_roofs = kernel_rooflines(pb, wname, per_class, peaks)
    config = workload_config(wname, pb)
    config.update({"l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"})
    ekw = eig_kwargs(args, pb)
    config["null_space"] = (f"randomized SVD, l = {ekw['rsvd_cols']} (warm started)" if ekw
                            else "Gram + principal subspace by tridiagonalisation")
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "fp32" else "bf16x2",
            "data": "synthetic",
            "config": config,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": all_launches,
            "roofline": roof,
            "class_ms_per_step": {KERNEL_NAMES[c]: round(v[0], 3) for c, v in per_class.items()},
            "class_launches_per_step": {KERNEL_NAMES[c]: v[1] for c, v in per_class.items()},
            "kernel_rooflines": extra_roofs,
            "plain_fp32": None if fp32_ms is None else {
                "value": fp32_value, "unit": UNIT, "ms_per_step": fp32_ms / fp32_steps, "steps": fp32_steps,
                "speedup_of_split_bf16": value / fp32_value},
            "clocks": clocks,
            "peaks_source": peak_src}
    if q0_ms is not None:
        line["b0_null_space_ms"] = q0_ms
    if world == 1:
        line["accuracy"] = accuracy_block(args, pb, hicu, h, geom, x_main if args.prec == "bf16" else None,
                                          x_fp32)
    if world == 1 and not args.no_cpu_baseline:
        v, _, desc = oracle_sample(pb)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                "sample": desc, "extrapolated": True}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
