#!/usr/bin/env python3
"""Benchmark of HEALPix spherical-harmonic synthesis at Planck resolution.

Workload: Nside = 2048 (50,331,648 pixels, 8191 rings), L = 4096, a batch of
8 maps of seeded Gaussian a_lm (Re, Im ~ N(0, C_l/2), C_l = 1/(l+1)^2), FP64,
requested accuracy eps = 1e-10.  A step is one synthesis of the whole batch
(Legendre stage + ring FFT stage) on inputs already resident in HBM; the
adjoint of the same batch and the plain one-map-per-launch synthesis are
timed the same way and reported beside it.  Inputs (1.07 GB of a_lm, 3.2 GB
of maps, 4.3 GB of q) are far larger than the 129 MB L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (the transform is replicated, not sharded); value is
the whole-job ms per map: the slowest rank's time over all maps of all
ranks.  ``--impl reference`` times the CPU oracle (the only reference
implementation: the paper ships no code) on a bounded ring sample of the
same workload and extrapolates to ms per map.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L=4096 HEALPix synthesis ms/map, % HBM roofline; batched & adjoint vs plain"
UNIT = "ms/map"

# GB300 FP64 pipe: 152 SMs x 2 DFMA/clock/SM x 2 flop x 2.070 GHz max SM clock
# (2 DFMA/clock/SM is NVIDIA's published 1.25 TFLOP/s FP64 rate for GB300
# divided over 152 SMs at 2070 MHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# DRAM traffic of the dominant kernel from an ncu capture (see profiles/),
# in the unit `achieved` is computed over (the kernel's launches of one step);
# valid only while the kernel's source files are unchanged.
NCU_TRAFFIC = {
    "legendre_synth_kernel": {
        "sources": ["paper_1110_4874_gb300/csrc/shtb_legendre.cu"],
        "sha256": "2716a9eb2679dc0a7730c490c671b800e69d7688a7fb6465ffbe4592e8d7cacb",
        # 410.5 MB measured at Nside=512, L=1024; every array scales with Nside*L (x16)
        "bytes": 16 * 410_475_008,
        "profile": "profiles/legendre_synth_nside512_l1024_b8.md",
    },
    # butterfly kernels: DRAM bytes of one synthesis of 8 maps at Nside=2048,
    # L=4096, scaled from an ncu capture of the same kernels at Nside=512,
    # L=1024 (all launches of one synthesis) by the stored elements each
    # kernel processes (dense interpolation elements for the levels, stored
    # residual elements for the residual blocks); keyed on the item bodies and
    # each kernel's own definition
    "bf_level_kernel": {
        "sources": ["paper_1110_4874_gb300/csrc/shtb_bf_items.cuh",
                    "paper_1110_4874_gb300/csrc/shtb_butterfly.cu::bf_level_kernel"],
        "sha256": "06b9e7a09d16be7486aa7ceb73c12caeb7b8b8df50f1ac49a2d63b093e7f3852",
        # (2153.0 + 811.7) MB x 4,266,029,163 / 140,986,926 dense elements
        "bytes": round((2_153_000_000 + 811_700_000) * 4_266_029_163 / 140_986_926),
        "profile": "profiles/bf_level_kernel_nside2048_l4096_b8.md",
    },
    "bf_r_kernel": {
        "sources": ["paper_1110_4874_gb300/csrc/shtb_bf_items.cuh",
                    "paper_1110_4874_gb300/csrc/shtb_butterfly.cu::bf_r_kernel"],
        "sha256": "a7f9b65a4a54b5fe181a4a547c65b3fad4279508730af57d9a3c50c700017a62",
        # (447.3 + 193.9) MB x 787,402,057 / 46,195,210 stored residual elements
        "bytes": round((447_300_000 + 193_900_000) * 787_402_057 / 46_195_210),
        "profile": "profiles/bf_level_kernel_nside2048_l4096_b8.md",
    },
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def file_sha256(path):
    with open(os.path.join(ROOT, path), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def kernel_text(src, name):
    """The text of the __global__ function `name` in a CUDA source: from its
    __global__ through the brace that closes its body."""
    i = src.find(name + "(")
    while i >= 0:
        g = src.rfind("__global__", 0, i)
        if g >= 0 and ";" not in src[g:i] and "}" not in src[g:i]:
            depth = 0
            for k in range(src.index("{", i), len(src)):
                depth += {"{": 1, "}": -1}.get(src[k], 0)
                if depth == 0:
                    return src[g:k + 1]
        i = src.find(name + "(", i + 1)
    raise KeyError(name)


def sources_sha256(paths):
    """One digest over several sources: a path stands for the whole file,
    "path::kernel" for that kernel's definition only (a single whole file:
    its own sha256)."""
    if len(paths) == 1 and "::" not in paths[0]:
        return file_sha256(paths[0])
    h = hashlib.sha256()
    for path in paths:
        fname, _, kernel = path.partition("::")
        with open(os.path.join(ROOT, fname), "rb") as fh:
            data = fh.read()
        h.update(kernel_text(data.decode(), kernel).encode() if kernel else data)
    return h.hexdigest()


# ------------------------------------------------------------ clock sampling
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi every 200 ms while the timed region runs."""

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- CPU oracle
def oracle_sample(nside, lmax, nmaps_sample, nrings_sample, seed, nthreads=0):
    """Time the CPU oracle on a ring sample of one map and extrapolate to ms
    per map (cost per ring scales with the ring count of the sample)."""
    import numpy as np

    import oracle
    from paper_1110_4874_gb300 import synthetic

    rings = oracle.healpix_rings(nside)
    idx = np.unique(np.linspace(0, rings.nrings - 1, nrings_sample).round().astype(int))
    sub = rings.subset(idx)
    a = synthetic.gaussian_alm(lmax, nmaps_sample, seed=seed)
    t0 = time.perf_counter()
    oracle.synthesize(sub, lmax, a, nthreads=nthreads)
    dt = time.perf_counter() - t0
    ms_per_map = dt * 1e3 / nmaps_sample * rings.nrings / idx.size
    cores = nthreads if nthreads > 0 else oracle.max_threads()
    sample = (f"{idx.size} of {rings.nrings} rings (evenly spaced, poles and equator included) "
              f"of {nmaps_sample} map(s), oracle synthesis (double-double one-step Legendre "
              f"recurrence + direct per-ring DFT), {dt:.1f} s, scaled by {rings.nrings}/{idx.size}")
    return ms_per_map, cores, sample


# -------------------------------------------------------------- our arm
def reduce_max(x, dist, device):
    """The largest of the ranks' values of x (each rank's own time); x
    itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def ms_per_map(ms_slowest, steps, nmaps, world):
    """Whole-job time per map: every rank transforms nmaps maps per step, so
    the job's maps are steps * nmaps * world in the slowest rank's time."""
    return ms_slowest / (steps * nmaps * world)


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    import paper_1110_4874_gb300 as sh
    from paper_1110_4874_gb300 import synthetic

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, L, B = args.nside, args.lmax, args.nmaps

    t0 = time.perf_counter()
    eps_plan = args.eps
    built_on = "host" if args.host_build else "gpu"
    try:
        try:
            plan = sh.Plan(N, L, eps_plan, leaf_cols=args.leaf_cols, gpu_build=not args.host_build,
                           nthreads=build_threads(world, not args.host_build),
                           residual_recurrence=args.residual_recurrence)
        except sh.ShtbError as e:
            # the GPU builder needs pinned staging per host worker; where the
            # host cannot give it (SHTB_ENOMEM), the same plan is built with
            # host IDs.  Any other error, a CUDA fault above all, propagates.
            if args.host_build or e.code != sh.SHTB_ENOMEM:
                raise
            built_on = f"host (GPU builder: {e})"
            plan = sh.Plan(N, L, eps_plan, leaf_cols=args.leaf_cols,
                           nthreads=build_threads(world, False),
                           residual_recurrence=args.residual_recurrence)
    except sh.ShtbError as e:
        if e.code != sh.SHTB_ENOTSUP or eps_plan <= 0:
            raise
        eps_plan = 0.0                      # compressed plans unavailable: exact operator
        plan = sh.Plan(N, L, eps_plan)
    plan_s = time.perf_counter() - t0
    st = plan.stats()
    plan.reserve(B)

    alm_h = torch.from_numpy(synthetic.gaussian_alm(L, B, seed=2000 + 100 * rank)).pin_memory()
    alm = alm_h.to(dev)
    maps = torch.empty((B, plan.npix), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(fn, steps):
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return reduce_max(e0.elapsed_time(e1), dist, dev)

    synth = lambda: plan.synthesize(alm, out=maps)  # noqa: E731
    for _ in range(args.warmup):
        synth()
    # ---- headline: batched synthesis, with stage events for the roofline
    sh.shtb_profile_enable(plan.handle, True)
    sh.shtb_profile_read(plan.handle)
    launches0 = plan.stats()["kernel_launches"]
    with ClockSampler(local) as clk:
        ms_total = timed(synth, args.steps)
    launches = plan.stats()["kernel_launches"] - launches0
    stages, ncalls = sh.shtb_profile_read(plan.handle)
    sh.shtb_profile_enable(plan.handle, False)
    clocks = clk.summary()
    value = ms_per_map(ms_total, args.steps, B, world)

    # ---- adjoint of the same batch
    f = torch.from_numpy(synthetic.gaussian_map(plan.npix, B, seed=3000 + rank)).to(dev)
    aout = torch.empty((B, plan.nalm), dtype=torch.complex128, device=dev)
    adj = lambda: plan.adjoint(f, out=aout)  # noqa: E731
    adj()
    ms_adj = ms_per_map(timed(adj, args.steps), args.steps, B, world)

    # ---- analysis (quadrature + Jacobi refinement) of the same batch
    analysis = None
    if not args.no_patterns:
        analysis = {"maps": B}
        for k in (0, 3):
            ana = lambda: plan.analyze(f, niter=k, out=aout)  # noqa: E731
            analysis[f"niter{k}_ms_per_map"] = round(event_ms(ana, 1) / B, 3)

    # ---- plain: one map per launch
    def plain():
        for b in range(B):
            plan.synthesize(alm[b:b + 1], out=maps[b:b + 1])
    plain()
    sh.shtb_profile_enable(plan.handle, True)
    sh.shtb_profile_read(plan.handle)
    ms_plain = ms_per_map(timed(plain, args.steps), args.steps, B, world)
    plain_stages, plain_calls = sh.shtb_profile_read(plan.handle)
    sh.shtb_profile_enable(plan.handle, False)

    # ---- end to end through the C ABI with host buffers (copies inside)
    maps_h = torch.empty((B, plan.npix), dtype=torch.float64).pin_memory()
    sh.shtb_synthesize_host(plan.handle, alm_h, maps_h, B)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sh.shtb_synthesize_host(plan.handle, alm_h, maps_h, B)
    e2e_s = reduce_max(time.perf_counter() - t0, dist, dev)
    e2e = {"value": ms_per_map(e2e_s * 1e3, args.steps, B, world), "unit": UNIT,
           "h2d_bytes_per_step": int(alm_h.numel() * alm_h.element_size()),
           "d2h_bytes_per_step": int(maps_h.numel() * maps_h.element_size())}

    # ---- roofline of the dominant kernel (FP64-bound on GB300), on the
    # algorithmic count of the butterfly: 4 flop per map per stored dense
    # element (two FMAs on the real and imaginary parts); identity entries
    # are a copy and count no flop
    groups = [8] * (B // 8) + ([B % 8] if B % 8 else [])
    ncall = max(ncalls, 1)
    if st["compressed"]:
        per_step = {   # kernel -> (algorithmic flops per step, ms per step)
            "bf_level_kernel": (B * 4.0 * st["n_dense"], stages["bf_levels"] / ncall),
            # stored blocks: 4B flop per element; regenerated: 4B + 4 (one recurrence step)
            "bf_r_kernel": (B * 4.0 * st["n_rstored"] + (4.0 * B + 4.0) * st["n_rgen"],
                            stages["bf_residual"] / ncall),
        }
    else:
        per_step = {"legendre_synth_kernel": (sum(4.0 * st["n_recurrence"] * (1 + g) for g in groups),
                                              stages["legendre_synth"] / ncall)}
    kname = max(per_step, key=lambda k: per_step[k][1])
    flops, kms = per_step[kname]
    achieved = flops / (kms * 1e-3) / 1e12
    traffic = None
    rec = NCU_TRAFFIC.get(kname)
    if rec and rec["bytes"] and rec["sha256"] == sources_sha256(rec["sources"]):
        traffic = rec["bytes"]
    dfma_gflops, _ = sh.shtb_measure_fp64_peak(local)
    peak_meas = dfma_gflops / 1e3
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "kernel": f"{kname} (FP64 pipe)",
                "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz",
                "peak_measured_dfma": round(peak_meas, 4),
                "frac_of_measured_dfma": round(achieved / peak_meas, 4),
                "count": "4 flop per map per stored dense element; identity entries are copies",
                "per_kernel_tflops": {k: round(f / (t * 1e-3) / 1e12, 4) if t else None
                                      for k, (f, t) in per_step.items()}}
    if st["compressed"]:
        with_ident = B * (4.0 * st["n_dense"] + 2.0 * st["n_ident"])
        roofline["frac_counting_identity_adds"] = round(
            with_ident / (per_step["bf_level_kernel"][1] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4)
    flops_leg = sum(f for f, _ in per_step.values())
    # ring stage: a real FFT of each ring's length plus the fold of the L+1
    # orders (2.5 J log2 J + 4 (L + 1) flop per ring and map)
    flops_phi = B * (st["phi_flops_per_map"] + 4.0 * (L + 1) * plan.nrings)
    phi_ms = stages["phi_synth"] / ncall
    roofline["ring_stage"] = {"flops_per_step": flops_phi, "ms_per_step": round(phi_ms, 3),
                              "achieved": round(flops_phi / (phi_ms * 1e-3) / 1e12, 4) if phi_ms else None,
                              "frac": round(flops_phi / (phi_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4)
                              if phi_ms else None}
    # whole-step HBM view (algorithmic bytes of the batch over the step time)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    step_bytes = (st["plan_read_bytes"] * len(groups) + B * st["nalm"] * 16 * 3
                  + B * plan.nrings * (L + 1) * 16 * 2 + B * plan.npix * 8)
    step_ms = ms_total / args.steps
    hbm = {"bytes_per_step": step_bytes, "achieved_gbs": round(step_bytes / (step_ms * 1e-3) / 1e9, 1),
           "peak_gbs": hbm_peak, "peak_source": "measured (MEASURED_PEAKS.json)" if hbm_peak else None,
           "frac": round(step_bytes / (step_ms * 1e-3) / 1e9 / hbm_peak, 4) if hbm_peak else None}
    # whole step against its roofline time T* = max(bytes / BW, flops / F64)
    t_star = max(step_bytes / (hbm_peak * 1e9) if hbm_peak else 0.0,
                 (flops_leg + flops_phi) / (FP64_PEAK_TFLOPS * 1e12)) * 1e3
    roofline["whole_step"] = {"flops": flops_leg + flops_phi, "bytes": step_bytes,
                              "t_star_ms": round(t_star, 3), "t_ms": round(step_ms, 3),
                              "t_star_over_t": round(t_star / step_ms, 4)}

    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian a_lm, C_l = 1/(l+1)^2)",
        "config": workload_config(args, world),
        "roofline": roofline, "hbm": hbm, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clocks,
        "details": {"adjoint_ms_per_map": round(ms_adj, 4), "plain_ms_per_map": round(ms_plain, 4),
                    "batched_over_plain": round(ms_plain / value, 3),
                    "stage_ms_per_step": {k: round(v / max(ncalls, 1), 3) for k, v in stages.items() if v},
                    "plain_stage_ms_per_map": {k: round(v / max(plain_calls, 1), 3)
                                               for k, v in plain_stages.items() if v},
                    "eps_plan": eps_plan, "compressed": bool(st["compressed"]),
                    "plan_build_s": round(plan_s, 2), "plan_built_on": built_on,
                    "plan_device_gb": round(st["plan_device_bytes"] / 1e9, 3),
                    "n_recurrence": st["n_recurrence"], "n_dense": st["n_dense"],
                    "n_rstored": st["n_rstored"], "n_ident": st["n_ident"],
                    "depth_hist": st["depth_hist"][:12],
                    "legendre_flops_per_step": flops_leg},
    }
    plan.close()
    del alm, maps, f, aout
    torch.cuda.empty_cache()
    if analysis is not None:
        out["details"]["analysis"] = analysis
    if rank == 0 and not args.no_patterns:
        out["details"]["batched_serving"], plan_c4 = batched_serving(sh, synthetic, dev)
        out["details"]["differentiation"] = differentiation(sh, synthetic, dev, plan_c4)
        out["details"]["regenerated_residual"] = regenerated_residual(sh, synthetic, dev, plan_c4)
        plan_c4.close()
        out["details"]["polarised"] = polarised_synthesis(sh, synthetic, dev)
        out["details"]["plan_build"] = plan_build_compare(sh)
        out["details"]["nside512_l1024"] = mid_size(sh, synthetic, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ms_cpu, cores, sample = oracle_sample(N, L, 1, args.cpu_rings, seed=2000)
        out["cpu_baseline"] = {"value": round(ms_cpu, 1), "unit": UNIT, "cores": cores,
                               "kind": "oracle", "sample": sample}
    return out


def mid_size(sh, synthetic, dev, N=512, L=1024, B=16, reps=5):
    """Nside=512, L=1024 at eps = 1e-10 and 1e-12: 16 maps sharing one plan
    in one call against the same maps one per call (ms/map each)."""
    import torch
    out = {}
    for eps in (1e-10, 1e-12):
        plan = sh.Plan(N, L, eps, leaf_cols=32, gpu_build=True)
        plan.reserve(B)
        alm = torch.from_numpy(synthetic.gaussian_alm(L, B, seed=2000)).to(dev)
        maps = torch.empty((B, plan.npix), dtype=torch.float64, device=dev)

        def plain():
            for b in range(B):
                plan.synthesize(alm[b:b + 1], out=maps[b:b + 1])
        ms_b = event_ms(lambda: plan.synthesize(alm, out=maps), reps) / B
        ms_1 = event_ms(plain, reps) / B
        out[f"eps{eps:g}"] = {"batched_ms_per_map": round(ms_b, 4), "plain_ms_per_map": round(ms_1, 4),
                              "batched_over_plain": round(ms_1 / ms_b, 3), "maps": B,
                              "n_dense": plan.stats()["n_dense"]}
        plan.close()
        del alm, maps
        torch.cuda.empty_cache()
    return out


def event_ms(fn, reps):
    """Mean CUDA-event time of fn on the current stream (one warm-up call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batched_serving(sh, synthetic, dev, reps=5):
    """Pattern 2 on the uneven request mix: 64 requests, Nside drawn from
    {64, ..., 1024} and 1-8 maps each (numpy default_rng(3000)), L = 2 Nside,
    eps = 1e-10; one persistent launch (graph replay) against the plain
    one-request-per-launch loop on the same plans.  Returns the summary and
    the Nside=1024 plan (reused for the differentiation workload)."""
    import numpy as np
    import torch

    rng = np.random.default_rng(3000)
    sizes = (64, 128, 256, 512, 1024)
    t0 = time.perf_counter()
    plans = {n: sh.Plan(n, 2 * n, 1e-10) for n in sizes}
    build_s = time.perf_counter() - t0
    reqs = []
    for i in range(64):
        n = int(rng.choice(sizes))
        b = int(rng.integers(1, 9))
        alm = torch.from_numpy(synthetic.gaussian_alm(2 * n, b, seed=3000 + 10 * i)).to(dev)
        reqs.append((plans[n], alm, torch.empty((b, plans[n].npix), dtype=torch.float64, device=dev)))
    nmaps = sum(int(r[1].shape[0]) for r in reqs)
    t0 = time.perf_counter()
    batch = sh.shtb_batch_create(reqs, autotune=True)
    create_s = time.perf_counter() - t0
    info = sh.shtb_batch_info(batch)
    stream = torch.cuda.current_stream()

    def plain():
        for p, alm, maps in reqs:
            p.synthesize(alm, out=maps)

    ms_plain = event_ms(plain, reps)
    want = [m.clone() for _, _, m in reqs]
    ms_batch = event_ms(lambda: sh.shtb_batch_run(batch, stream), reps)
    sh.shtb_batch_status(batch, stream)
    diff = max(float((m - w).abs().max() / w.abs().max()) for (_, _, m), w in zip(reqs, want))
    sh.shtb_batch_destroy(batch)
    # each schedule family on its own: the one persistent launch (warps per
    # block x work order) and the stage-kernel graph
    families = {}
    for name, kw in (("persistent_w4", dict(schedule=0, warps_per_block=4, lpt=True)),
                     ("persistent_w8", dict(schedule=0, warps_per_block=8, lpt=True)),
                     ("graph_4_streams", dict(schedule=1, streams=4))):
        bb = sh.shtb_batch_create(reqs, autotune=False, **kw)
        families[name] = round(event_ms(lambda: sh.shtb_batch_run(bb, stream), reps), 3)
        sh.shtb_batch_status(bb, stream)
        families[name + "_bitwise_equal"] = all(torch.equal(m, w) for (_, _, m), w in zip(reqs, want))
        sh.shtb_batch_destroy(bb)
    for n in sizes[:-1]:
        plans[n].close()
    return ({"requests": 64, "maps": nmaps, "plans": len(sizes), "eps": 1e-10,
             "batched_ms": round(ms_batch, 3), "plain_ms": round(ms_plain, 3),
             "batched_over_plain": round(ms_plain / ms_batch, 3),
             "maps_per_s_batched": round(nmaps / (ms_batch * 1e-3), 1),
             "max_rel_diff_vs_plain": diff, "schedule": info, "families_ms": families,
             "plan_build_s": round(build_s, 1), "create_and_tune_s": round(create_s, 1)},
            plans[sizes[-1]])


def differentiation(sh, synthetic, dev, plan, reps=5):
    """Pattern 3: loss = 0.5 ||Y a - d||^2 at Nside=1024, L=2048, 4 maps,
    d = Y a_true + 0.1 N(0, 1) per pixel; forward + backward through the
    autograd Function (backward = the adjoint kernels), and a directional
    derivative check (exact for a quadratic loss up to rounding)."""
    import numpy as np
    import torch

    B, L = 4, plan.lmax
    a_true = torch.from_numpy(np.stack([synthetic.gaussian_alm(L, 1, seed=4100 + b)[0] for b in range(B)])).to(dev)
    a0 = torch.from_numpy(np.stack([synthetic.gaussian_alm(L, 1, seed=4000 + b)[0] for b in range(B)])).to(dev)
    noise = torch.from_numpy(np.random.default_rng(4200).normal(0.0, 0.1, (B, plan.npix))).to(dev)
    with torch.no_grad():
        d = plan.synthesize(a_true) + noise

    def loss_of(a):
        r = sh.synthesize(a, plan) - d
        return 0.5 * (r * r).sum()

    a = a0.clone().requires_grad_(True)

    def step():
        a.grad = None
        loss_of(a).backward()

    ms = event_ms(step, reps)
    g = a.grad.detach().clone()
    v = torch.from_numpy(synthetic.gaussian_alm(L, B, seed=4300)).to(dev)
    v[:, :L + 1] = v[:, :L + 1].real.to(v.dtype)     # Im a_l0 is ignored by the transform
    h = 1e-3
    with torch.no_grad():
        fd = (loss_of(a0 + h * v) - loss_of(a0 - h * v)) / (2 * h)
    dd = float((g.conj() * v).real.sum())
    return {"nside": plan.nside, "lmax": L, "maps": B, "eps": plan.eps,
            "fwd_bwd_ms": round(ms, 3), "fwd_bwd_ms_per_map": round(ms / B, 3),
            "directional_derivative_rel_err": abs(float(fd) - dd) / abs(dd)}


def regenerated_residual(sh, synthetic, dev, plan, B=8, reps=5):
    """The same compressed operator (Nside=1024, L=2048, eps=1e-10) with its
    residual blocks regenerated by the recurrence from two start values per
    (block, column) instead of stored: synthesis and adjoint of B maps against
    the stored plan, plan memory of both, and the largest relative RMS
    differences."""
    import torch
    L = plan.lmax
    regen = sh.Plan(plan.nside, L, plan.eps, gpu_build=True, residual_recurrence=True)
    a = torch.from_numpy(synthetic.gaussian_alm(L, B, seed=4400)).to(dev)
    m0 = torch.empty((B, plan.npix), dtype=torch.float64, device=dev)
    m1 = torch.empty_like(m0)
    ms_stored = event_ms(lambda: plan.synthesize(a, out=m0), reps) / B
    ms_regen = event_ms(lambda: regen.synthesize(a, out=m1), reps) / B
    diff = max(float(((m1[b] - m0[b]).norm() / m0[b].norm()).item()) for b in range(B))
    a0 = torch.empty_like(a)
    a1 = torch.empty_like(a)
    ms_adj_stored = event_ms(lambda: plan.adjoint(m0, out=a0), reps) / B
    ms_adj_regen = event_ms(lambda: regen.adjoint(m0, out=a1), reps) / B
    adiff = max(float(((a1[b] - a0[b]).norm() / a0[b].norm()).item()) for b in range(B))
    s0, s1 = plan.stats(), regen.stats()
    regen.close()
    return {"nside": plan.nside, "lmax": L, "maps": B, "eps": plan.eps,
            "stored_ms_per_map": round(ms_stored, 3), "regenerated_ms_per_map": round(ms_regen, 3),
            "stored_plan_gb": round(s0["plan_device_bytes"] / 1e9, 3),
            "regenerated_plan_gb": round(s1["plan_device_bytes"] / 1e9, 3),
            "n_rstored": s0["n_rstored"], "n_rgen": s1["n_rgen"], "max_rel_rms_vs_stored": diff,
            "adjoint_stored_ms_per_map": round(ms_adj_stored, 3),
            "adjoint_regenerated_ms_per_map": round(ms_adj_regen, 3), "adjoint_max_rel_rms_vs_stored": adiff}


def polarised_synthesis(sh, synthetic, dev, reps=5):
    """Spin-2 (Q, U from E, B) synthesis at Nside=512, L=1024, eps=1e-10,
    4 pairs, beside a scalar synthesis of the same 8 coefficient sets on a
    scalar plan of the same size."""
    import numpy as np
    import torch

    N, L, P = 512, 1024, 4
    t0 = time.perf_counter()
    plan = sh.Plan(N, L, 1e-10, spin=2)
    build_s = time.perf_counter() - t0
    eb = np.stack([np.stack([synthetic.gaussian_alm(L, 1, seed=7000 + 2 * p)[0],
                             synthetic.gaussian_alm(L, 1, seed=7001 + 2 * p)[0]]) for p in range(P)])
    a = torch.from_numpy(eb).to(dev)
    out = torch.empty((P, 2, plan.npix), dtype=torch.float64, device=dev)
    ms = event_ms(lambda: plan.synthesize_spin(a, out=out), reps)
    st = plan.stats()
    plan.close()
    scalar = sh.Plan(N, L, 1e-10)
    flat = a.reshape(2 * P, -1)
    maps = torch.empty((2 * P, scalar.npix), dtype=torch.float64, device=dev)
    ms_scalar = event_ms(lambda: scalar.synthesize(flat, out=maps), reps)
    scalar.close()
    return {"nside": N, "lmax": L, "pairs": P, "eps": 1e-10, "ms": round(ms, 3),
            "ms_per_pair": round(ms / P, 3), "scalar_ms_per_map": round(ms_scalar / (2 * P), 3),
            "plan_build_s": round(build_s, 2), "plan_device_gb": round(st["plan_device_bytes"] / 1e9, 3),
            "n_dense": st["n_dense"], "n_rstored": st["n_rstored"]}


def plan_build_compare(sh, N=512, L=1024, eps=1e-10):
    """Plan build time at Nside=512, L=1024: the IDs on the host cores vs
    batched on the GPU (the same plan up to pivoting near-ties)."""
    out = {"nside": N, "lmax": L, "eps": eps}
    for name, gb in (("host_s", False), ("gpu_s", True)):
        t0 = time.perf_counter()
        p = sh.Plan(N, L, eps, gpu_build=gb)
        out[name] = round(time.perf_counter() - t0, 2)
        out["n_dense_" + name[:-2]] = p.stats()["n_dense"]
        p.close()
    return out


def build_threads(world, gpu_build):
    """Host threads for one rank's plan build: the library's default (all
    cores, twice that for the GPU builder, whose workers also wait on their
    GPU batches) on one rank; the node's cores shared out when several ranks
    build at once."""
    if world <= 1:
        return 0
    cores = max(1, (os.cpu_count() or 1) // world)
    return 2 * cores if gpu_build else cores


def workload_config(args, world):
    """The workload both arms report (the same object for ours and the
    reference): the synthesis size, batch, requested tolerance and layout."""
    N, L, B = args.nside, args.lmax, args.nmaps
    gb = lambda x: round(x / 1e9, 2)  # noqa: E731
    a_bytes, m_bytes = 16 * B * (L + 1) * (L + 2) / 2, 8 * B * 12 * N * N
    cfg = {"workload": f"HEALPix synthesis Nside={N} L={L} batch of {B} maps",
           "nside": N, "lmax": L, "nmaps": B, "eps": args.eps, "leaf_cols": args.leaf_cols,
           "parallelism": f"replicas x{world}",
           "l2": (f"a_lm {gb(a_bytes)} GB and maps {gb(m_bytes)} GB per step, "
                  + ("both larger than the 129 MB L2" if min(a_bytes, m_bytes) > 129e6
                     else "not both larger than the 129 MB L2"))}
    if getattr(args, "residual_recurrence", False):
        cfg["residual_blocks"] = "regenerated by the recurrence"
    return cfg


def run_reference(args):
    """The CPU oracle as the reference arm: each step a bounded ring sample."""
    vals = []
    cores, sample = None, None
    for _ in range(args.warmup):
        oracle_sample(args.nside, args.lmax, 1, max(4, args.ref_rings // 4), seed=2000)
    t0 = time.perf_counter()
    for s in range(args.steps):
        v, cores, sample = oracle_sample(args.nside, args.lmax, 1, args.ref_rings, seed=2000 + s)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    return {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall * 1e3 / args.steps, 1),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian a_lm, C_l = 1/(l+1)^2)", "impl": "reference",
        "config": workload_config(args, args.gpus),
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nside", type=int, default=2048)
    ap.add_argument("--lmax", type=int, default=4096)
    ap.add_argument("--nmaps", type=int, default=8)
    ap.add_argument("--eps", type=float, default=1e-10)
    ap.add_argument("--leaf-cols", type=int, default=32, help="rings per butterfly leaf block")
    ap.add_argument("--cpu-rings", type=int, default=64, help="ring sample of the CPU baseline")
    ap.add_argument("--ref-rings", type=int, default=16, help="ring sample per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--residual-recurrence", action="store_true",
                    help="plan that regenerates its residual blocks by the recurrence (less plan memory)")
    ap.add_argument("--host-build", action="store_true",
                    help="build the plan's interpolative decompositions on the host, not the GPU")
    ap.add_argument("--no-patterns", action="store_true",
                    help="skip the batched-serving and differentiation measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    out = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
