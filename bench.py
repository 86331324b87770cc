#!/usr/bin/env python
"""Benchmark of the multiple-scattering hot path on GB300.

One step = the whole hot path on the 400-disk workload (M = 400 sound-soft
disks, radii U[0.5, 1.5] in a 100 x 100 square, gap 0.2, k = 2 pi, N = 20,
16 400 unknowns, one plane wave): Bessel diagonals and Toeplitz generators
(recomputed from the device-resident geometry), preconditioned right-hand
side, restarted GMRES to relres 1e-10 with the block-Toeplitz product, and
the far field at 360 angles.  The FP64 path is the timed step; the same
steps are then timed with FP32 inner sweeps and FP64 refinement (MSD_MIXED)
for the "FP64 vs mixed" half of the metric.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "block-matvec GB/s (% HBM peak) & solve time at relres 1e-10, FP64 vs mixed"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12  # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
TF32_OVER_BF16 = 1.1 / 2.25                    # nominal dense TF32 / bf16 tensor rate
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the FP64
# product kernel (window length 7, generator rows staged by bulk copies) on
# this workload, from an ncu capture (216.05 MB read + 5.78 MB written); the
# algorithmic stream is 207.7 MB
K3_FP64_DRAM_BYTES_PER_LAUNCH = 221831168
K3_FP64_TRAFFIC_SOURCE = ("copied from an ncu capture of the same kernel on this workload "
                          "(profiles/k_bt_matvec_random400.md, current kernel), not measured in this run")
WORKLOAD = ("random400_k2pi: M=400 sound-soft disks, a~U[0.5,1.5], centres U[-50,50]^2 gap 0.2, "
            "k=2pi, N=20 (16400 unknowns), 1 plane wave, GMRES (restart length sized to HBM) to relres 1e-10, "
            "far field T=360")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def start_clock_sampler(dev: int):
    try:
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        return subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def stop_clock_sampler(p):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        return None
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 7:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        for n, v in zip(names, f[3:7]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# The CPU baseline (the oracle, as it stands) is timed on one fixed sample
# of the 400-disk product: CPU_SAMPLE_ROWS target block rows, evenly spaced,
# applied to one seeded vector, split over a spawn process pool with one
# worker per host core (each worker single-threaded).  The reference arm
# runs one pass of this sample per step; the cpu_baseline of the main line
# repeats the same pass for about ten seconds.
CPU_SAMPLE_ROWS = 64


def _oracle_rows(payload):
    """Worker: the oracle's preconditioned block rows `rows` applied to x."""
    import oracle.msd_oracle as O_
    centres, radii, bc, k, N, x, rows = payload
    return O_.preconditioned_rows(centres, radii, bc, k, N, x, rows)


class OracleSample:
    def __init__(self, cl):
        import multiprocessing as mp
        import numpy as np
        self.cl = cl
        self.cores = os.cpu_count() or 1
        self.rows = [int(r) for r in np.linspace(0, cl.M - 1, CPU_SAMPLE_ROWS).round()]
        self.x = np.random.default_rng(0).standard_normal((cl.ntot, 1)) + 0j
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores)   # spawned: safe after CUDA is initialised
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
        self.chunks = [self.rows[i::self.cores] for i in range(self.cores) if self.rows[i::self.cores]]
        self.pass_once()   # imports the oracle in every worker (untimed)
        self.bytes_per_pass = algorithmic_bytes_fp64(cl) * len(self.rows) / cl.M
        self.description = (f"{len(self.rows)} evenly spaced target block rows of the 400-disk FP64 product "
                            f"(oracle preconditioned_rows, NumPy/SciPy) per pass, split over {self.cores} "
                            "single-threaded spawn workers")

    def pass_once(self) -> float:
        cl = self.cl
        t0 = time.perf_counter()
        self.pool.map(_oracle_rows, [(cl.centres, cl.radii, cl.bc, cl.k, cl.N, self.x, ch) for ch in self.chunks])
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def algorithmic_bytes_fp64(cl, R=1):
    M, L, n = cl.M, 4 * cl.N + 1, cl.n
    return 16.0 * (M * (M - 1) * L + 2.0 * M * n * R)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1409_8186_gb300 import workloads as W
    cl = W.random_cluster_400()
    smp = OracleSample(cl)
    for _ in range(max(0, args.warmup)):
        smp.pass_once()
    times = [smp.pass_once() for _ in range(args.steps)]
    smp.close()
    t = sum(times) / len(times)
    gbs = smp.bytes_per_pass / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "what": "the CPU oracle's FP64 block-row products; one step = one "
                       "pass over the fixed row sample (value = algorithmic bytes of the sampled rows / wall time)"},
            "ms_per_full_product_extrapolated": t * 1e3 * cl.M / len(smp.rows),
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": smp.cores, "kind": "oracle",
                             "sample": smp.description},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(local_ms: float, local_bytes: float, dist, device="cpu"):
    """Whole-job throughput across ranks: the slowest rank's time and the
    algorithmic bytes of every rank's block products (replicas: each rank
    runs its own copy of the workload).  Returns (max_ms, GB/s)."""
    import torch
    t = torch.tensor([local_ms, local_bytes], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized():
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = t[1:].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        max_ms, all_bytes = float(mx.item()), float(tot.item())
    else:
        max_ms, all_bytes = local_ms, local_bytes
    return max_ms, all_bytes / (max_ms * 1e-3) / 1e9


def profile_only(what: str):
    """Minimal runs for ncu captures: 'matvec' = three FP64 then three FP32
    products of the 400-disk operator; 'fp64' / 'mixed' = one solve;
    'sweep600' = one FP32 sweep of the mixed solve capped at 600 Arnoldi
    steps (after a 5-step solve that builds the plans), with its wall time
    per step;
    'tc' / 'tcs' = three tensor-core FP32 products with 64 columns on the
    first 800 sites of the 4000-disk lattice (generators 0.31 GB, above L2;
    the expanding kernel / the shift-GEMM kernel);
    'recompute' = three FP32 products of the same operator with recomputed
    generators."""
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    if what in ("tc", "tcs", "recompute"):
        cl = W.lattice_4000(M=800)
        pb = msd.Problem(cl)
        R = 64 if what in ("tc", "tcs") else 1
        if what == "tc":
            pb.set_tile(R, msd.MSD_FP32, 0, 64)
        elif what == "tcs":
            pb.set_tile(R, msd.MSD_FP32, 0, 8)
        else:
            pb.set_generator_mode(msd.MSD_GEN_RECOMPUTE)
        g = torch.Generator(device="cpu").manual_seed(0)
        x = torch.randn(cl.ntot, R, dtype=torch.complex128, generator=g).to(torch.complex64).cuda()
        for _ in range(3):
            pb.matvec(x, msd.MSD_FP32)
        torch.cuda.synchronize()
        return
    cl = W.random_cluster_400()
    pb = msd.Problem(cl)
    if what == "sweep600":
        import time
        beta = [cl.meta["beta"]]
        pb.solve(beta, tol=1e-10, precision=msd.MSD_MIXED, maxit=5, max_refine=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = pb.solve(beta, tol=1e-10, precision=msd.MSD_MIXED, maxit=600, max_refine=1)
        torch.cuda.synchronize()
        steps = max(1, int(res.iters.max()))
        print(json.dumps({"steps": steps, "wall_us_per_step": round((time.perf_counter() - t0) * 1e6 / steps, 1)}))
        return
    if what == "matvec":
        g = torch.Generator(device="cpu").manual_seed(0)
        x64 = torch.randn(cl.ntot, 1, dtype=torch.complex128, generator=g).cuda()
        x32 = x64.to(torch.complex64)
        for x, p in ((x64, msd.MSD_FP64), (x32, msd.MSD_FP32)):
            for _ in range(3):
                pb.matvec(x, p)
    else:
        prec = msd.MSD_FP64 if what == "fp64" else msd.MSD_MIXED
        res = pb.solve([cl.meta["beta"]], tol=1e-10, precision=prec)
        print("status", res.status, "iters", int(res.iters[0]), "relres", float(res.relres[0]))
    torch.cuda.synchronize()


def products_table(reps: int = 3, only: str = ""):
    """One JSON line per (workload, columns R, precision, kernel, generator
    mode): the block-Toeplitz kernel's own time (CUDA events around each
    launch, averaged over `reps` products after one untimed product) and the
    whole product (column scaling + kernel + split reduction), with the
    algorithmic FLOP rate and generator+vector bandwidth.  Kernels: the
    autotuned plan ("auto", its shape reported), the cost-model CUDA-core
    shape ("model"), and each tensor-core column tile ("tcNN")."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    F64, F32 = msd.MSD_FP64, msd.MSD_FP32
    peaks = measured_peaks() or {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * TF32_OVER_BF16  # measured bf16 x nominal ratio
    cases = [
        ("random400 (M=400, N=20)", W.random_cluster_400, [(F64, 1), (F32, 1)], False),
        ("random200_k10 (M=200, N=22)", W.cluster_200, [(F64, 16), (F32, 16)], False),
        ("batched6 (6 of the 256 batched clusters)", lambda: W.batched_clusters(count=6), [(F32, 32)], False),
        ("batched256 (all 256 batched clusters, 3.1 M unknowns)", lambda: W.batched_clusters(count=256),
         [(F32, 32)], False),
        ("lattice4000 (M=4000, N=15)", W.lattice_4000, [(F64, 1), (F32, 1), (F32, 64)], True),
    ]
    for name, make, shapes, try_recompute in cases:
        if only and only not in name:
            continue
        cl = make()
        for gen in (["streamed", "recompute"] if try_recompute else ["streamed"]):
            for prec, R in shapes:
                kinds = ["auto", "model"]
                if prec == F32:
                    kinds += [f"tc{rc}" for rc in (16, 32, 64) if R % rc == 0]
                    if R % 8 == 0 and gen == "streamed":
                        kinds += ["tcs", "tcsw"]
                for kind in kinds:
                    os.environ["MSD_AUTOTUNE"] = "0" if kind == "model" else "1"
                    pb = msd.Problem(cl)
                    if gen == "recompute":
                        pb.set_generator_mode(msd.MSD_GEN_RECOMPUTE)
                    if kind in ("tcs", "tcsw"):
                        pb.set_tile(R, prec, 0 if kind == "tcs" else 1, 8)
                    elif kind.startswith("tc"):
                        pb.set_tile(R, prec, 0, int(kind[2:]))
                    dt = torch.complex128 if prec == F64 else torch.complex64
                    g = torch.Generator(device="cpu").manual_seed(R)
                    x = torch.randn(pb.ntot, R, dtype=torch.complex128, generator=g).to(dt).cuda()
                    y = torch.empty_like(x)
                    info, tuned = pb.plan_info(R, prec)
                    pb.matvec(x, prec, out=y)
                    torch.cuda.synchronize()
                    msd.msd_matvec_timing(pb.handle, 1)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        pb.matvec(x, prec, out=y)
                    e1.record()
                    torch.cuda.synchronize()
                    kms, nl, fl, by = msd.msd_matvec_timing(pb.handle, 0)
                    prod_ms = e0.elapsed_time(e1) / reps
                    kms /= max(nl, 1)
                    fl /= max(nl, 1)
                    by /= max(nl, 1)
                    tf = fl / (kms * 1e-3) / 1e12
                    gbs = by / (kms * 1e-3) / 1e9
                    if prec == F64:
                        bound, peak = "fp64 alu", FP64_PEAK_TFLOPS
                    elif info["KB"] < 4:  # tensor cores (all kernels): 3 TF32 products per real multiply-add
                        bound, peak = "tf32 tensor (3x executed)", tf32_peak / 3.0
                    else:
                        bound, peak = "fp32 alu", FP32_PEAK_TFLOPS
                    print(json.dumps({
                        "workload": name, "R": R, "precision": "fp64" if prec == F64 else "fp32",
                        "kernel": kind, "shape": info, "generators": gen,
                        "kernel_ms": round(kms, 4), "product_ms": round(prod_ms, 4),
                        "tflops": round(tf, 2), "bound": bound, "peak_frac": round(tf / peak, 3),
                        "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4)}), flush=True)
                    pb.close()
                    del pb, x, y
                    torch.cuda.empty_cache()
    os.environ.pop("MSD_AUTOTUNE", None)


def grad_timing(reps: int = 3):
    """One JSON line per precision: the adjoint gradient of the far-field
    misfit on the 200-disk workload (M = 200, k = 10, N = 22, 16 incidences,
    360 far-field samples; target = the perturbed configuration's far field):
    forward solve, far field, misfit, adjoint solve, pair and per-disk
    gradient kernels, timed with CUDA events around the whole C-ABI call
    (host outputs), after one untimed call."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    cl = W.cluster_200()
    betas, th = W.angles(16), W.angles(360)
    tgt = W.perturbed_target(cl, seed=40)
    pt = msd.Problem(tgt)
    rt = pt.solve(betas, tol=1e-13, precision=msd.MSD_MIXED)
    Ft = pt.farfield(rt.rho, th).cpu().numpy()
    pt.close()
    pb = msd.Problem(cl)
    for prec, name in ((msd.MSD_FP64, "fp64"), (msd.MSD_MIXED, "mixed")):
        pb.grad_farfield_misfit(betas, th, Ft, tol=1e-12, precision=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            J, dO, da, dk = pb.grad_farfield_misfit(betas, th, Ft, tol=1e-12, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"workload": "random200_k10 (M=200, N=22, 16 incidences, 360 samples)",
                          "what": "J and dJ/d(centres, radii, k) by the adjoint method, solves to relres 1e-12",
                          "precision": name, "ms_per_gradient": round(e0.elapsed_time(e1) / reps, 2),
                          "J": float(J[0]), "grad_norm": float(np.sqrt((dO ** 2).sum() + (da ** 2).sum() + dk[0] ** 2))}),
              flush=True)
    pb.close()


def batched_timing(count: int = 16):
    """Batched solves: `count` clusters of the batched recipe (mixed
    Dirichlet/Neumann, k ~ U[1, 8], N = ceil(k) + 8, area fraction 0.2, gap
    0.01; M restricted to 50..150 so that a solve ends in minutes) with 32
    incidences each, in one batch (count x 32 systems), to relres 1e-10,
    plain FP64 and mixed precision; CUDA events around each solve."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    cls = W.batched_clusters(count=count, m_lo=50, m_hi=150)
    R = 32
    betas = np.stack([W.angles(R)] * len(cls))
    pb = msd.Problem(cls)
    for prec, name in ((msd.MSD_FP64, "fp64"), (msd.MSD_MIXED, "mixed")):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = pb.solve(betas, tol=1e-10, precision=prec, maxit=8000)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"workload": f"batched recipe, {count} clusters (M 50..150), {R} incidences each",
                          "systems": int(len(cls) * R), "unknowns": int(pb.ntot), "precision": name,
                          "solve_ms": round(e0.elapsed_time(e1), 1), "status": int(res.status),
                          "iters_max": int(res.iters.max()), "refine_steps": int(res.refine_steps.max()),
                          "relres_max": float(res.relres.max())}), flush=True)
    pb.close()


def batched_full(groups: int = 8, take: int = 256, maxit: int = 20000, check_rows: int = 2, only_group: int = -1,
                 fp64_groups=()):
    """The batched workload as specified: 256 seeded clusters (M ~ U{50..800},
    unit radii, area fraction 0.2, gap 0.01, k ~ U[1, 8], N = ceil(k) + 8,
    Dirichlet/Neumann per disk ~ Bernoulli(1/2)), 32 incidences each,
    mixed-precision solve (FP32 inner sweeps, FP64 refinement) to relres
    1e-10.  The clusters are ordered by M and solved as `groups` batched
    problems of consecutive sizes (each group's Krylov basis and generators
    fit in HBM together with a long restart); one JSON line per group and
    one for the whole batch.  Every cluster is checked on `check_rows`
    sampled target disks: the oracle's residual of the GPU densities on
    those rows must be within the stopping bound (1.05e-10 ||P^-1 b||).
    The groups listed in `fp64_groups` are solved a second time in FP64 (the
    plain GPU solve the mixed one is compared with)."""
    import numpy as np
    import torch
    import oracle.msd_oracle as O_
    from paper_1409_8186_gb300 import msd, workloads as W
    cls = W.batched_clusters(count=256)
    order = sorted(range(len(cls)), key=lambda i: cls[i].M)[:take]
    R = 32
    betas_all = W.angles(R)
    chunks = np.array_split(np.array(order), groups)
    tot_ms, worst_rel, worst_check, tot_iters = 0.0, 0.0, 0.0, 0
    rows_done = 0
    for gi, idx in enumerate(chunks):
        if only_group >= 0 and gi != only_group:
            continue
        sub = [cls[i] for i in idx]
        pb = msd.Problem(sub)
        betas = np.stack([betas_all] * len(sub))
        info32, _ = pb.plan_info(R, msd.MSD_FP32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = pb.solve(betas, tol=1e-10, precision=msd.MSD_MIXED, maxit=maxit)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        rho = res.rho.cpu().numpy()
        worst = 0.0
        for c, cl in enumerate(sub):
            o0 = pb.row_offset(c)
            b = O_.preconditioned_rhs(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas[c])
            bn = np.linalg.norm(b, axis=0)
            tg = sorted(set([0, cl.M - 1] + list(np.random.default_rng(c).choice(cl.M, check_rows, replace=False))))
            rows = O_.preconditioned_rows(cl.centres, cl.radii, cl.bc, cl.k, cl.N, rho[o0:o0 + cl.ntot], tg)
            for i, p in enumerate(tg):
                r = b[p * cl.n:(p + 1) * cl.n] - rows[i]
                worst = max(worst, float((np.linalg.norm(r, axis=0) / bn).max()))
        fp64 = None
        if gi in fp64_groups:
            torch.cuda.synchronize()
            e0.record()
            r64 = pb.solve(betas, tol=1e-10, precision=msd.MSD_FP64, maxit=maxit)
            e1.record()
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1)
            fp64 = {"solve_ms": round(ms64, 1), "status": int(r64.status), "iters_max": int(r64.iters.max()),
                    "relres_max": float(r64.relres.max()), "mixed_speedup": round(ms64 / ms, 2)}
            del r64
        tot_ms += ms
        worst_rel = max(worst_rel, float(res.relres.max()))
        worst_check = max(worst_check, worst)
        tot_iters = max(tot_iters, int(res.iters.max()))
        rows_done += pb.ntot
        print(json.dumps({"workload": f"batched recipe, group {gi + 1}/{len(chunks)} (M {sub[0].M}..{sub[-1].M})",
                          "clusters": len(sub), "systems": len(sub) * R, "unknowns": int(pb.ntot),
                          "fp32_product_shape": info32, "solve_ms": round(ms, 1), "status": int(res.status),
                          "iters_max": int(res.iters.max()), "iters_median": float(np.median(res.iters)),
                          "refine_steps": int(res.refine_steps.max()), "relres_max": float(res.relres.max()),
                          "sampled_residual_max": worst, "fp64": fp64}), flush=True)
        pb.close()
        del pb, res, rho
        torch.cuda.empty_cache()
    print(json.dumps({"workload": f"batched recipe, {len(order)} clusters x {R} incidences, mixed precision to relres 1e-10",
                      "groups": len(chunks), "unknowns_per_column": int(rows_done), "solve_ms_total": round(tot_ms, 1),
                      "iters_max": tot_iters, "relres_max": worst_rel, "sampled_residual_max": worst_check,
                      "all_within_bound": bool(worst_check <= 1.05e-10 and worst_rel <= 1e-10)}), flush=True)


def lattice_solve(R: int = 8, maxit: int = 30000, check_rows: int = 6):
    """The 4000-disk lattice (radius 0.3, spacing 1, jitter 0.02, k = 5,
    N = 15, 124,000 unknowns) with R incidences, mixed-precision solve to
    relres 1e-10 (restart sized to HBM, up to 4000); CUDA events around the
    solve; the oracle's residual on sampled target rows of every column."""
    import numpy as np
    import torch
    import oracle.msd_oracle as O_
    from paper_1409_8186_gb300 import msd, workloads as W
    cl = W.lattice_4000()
    pb = msd.Problem(cl)
    betas = W.angles(R)
    info32, _ = pb.plan_info(R, msd.MSD_FP32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = pb.solve(betas, tol=1e-10, precision=msd.MSD_MIXED, maxit=maxit)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rho = res.rho.cpu().numpy()
    b = O_.preconditioned_rhs(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas)
    bn = np.linalg.norm(b, axis=0)
    tg = sorted(set([0, cl.M - 1] + list(np.random.default_rng(5).choice(cl.M, check_rows, replace=False))))
    rows = O_.preconditioned_rows(cl.centres, cl.radii, cl.bc, cl.k, cl.N, rho, tg)
    worst = max(float((np.linalg.norm(b[p * cl.n:(p + 1) * cl.n] - rows[i], axis=0) / bn).max())
                for i, p in enumerate(tg))
    print(json.dumps({"workload": f"lattice4000 (M=4000, N=15, 124000 unknowns), {R} incidences, mixed to 1e-10",
                      "fp32_product_shape": info32, "solve_ms": round(ms, 1), "status": int(res.status),
                      "iters_max": int(res.iters.max()), "refine_steps": int(res.refine_steps.max()),
                      "relres_max": float(res.relres.max()), "sampled_residual_max": worst}), flush=True)


def nearfield_timing(n: int = 512):
    """Scattered field (Prop. 4.3, kernel K8) of the 400-disk solution on an
    n x n grid over [-55, 55]^2 (points inside disks return 0): CUDA events
    around the C-ABI call with device buffers, after one untimed call."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    cl = W.random_cluster_400()
    pb = msd.Problem(cl)
    res = pb.solve([cl.meta["beta"]], tol=1e-10, precision=msd.MSD_MIXED)
    g = np.linspace(-55.0, 55.0, n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = torch.from_numpy(np.stack([X.ravel(), Y.ravel()], axis=1)).cuda()
    u = torch.empty((n * n, 1), dtype=torch.complex128, device="cuda")
    msd.msd_nearfield(pb.handle, 0, res.rho, 1, pts, u)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        msd.msd_nearfield(pb.handle, 0, res.rho, 1, pts, u)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    print(json.dumps({"workload": f"random400 solution, {n}x{n} grid over [-55,55]^2", "points": n * n,
                      "disks": cl.M, "modes": cl.n, "ms": round(ms, 3),
                      "point_disk_pairs_per_s": n * n * cl.M / (ms * 1e-3)}), flush=True)
    pb.close()


def dort_timing():
    """Time reversal (section 7): the whole msd_dort call (batched solve of
    n_alpha incidences to relres 1e-12, far field at the opposite angles,
    T = conj(F)^T F, eigenvalues) and the eigen stage alone (msd_dort_eigen
    on the same F), CUDA events after one untimed call.  Workloads: the
    three small sound-soft disks of the example with 512 mirror angles; a
    100-disk cluster (radii 0.5..1, k = 2) with 256 angles; the eigen stage
    of random 1024 and 2048 matrices."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    scenes = [(W.dort_three_disks(0), 512, "three small sound-soft disks (example), 512 angles"),
              (W.random_cluster(seed=21, M=100, half_side=20.0, rmin=0.5, rmax=1.0, gap=0.3, k=2.0, N=10),
               256, "random100_k2 (M=100, N=10), 256 angles")]
    for cl, n, name in scenes:
        pb = msd.Problem(cl)
        for prec, pname in ((msd.MSD_FP64, "fp64"), (msd.MSD_MIXED, "mixed")):
            ms, (eig, F, _, st) = timed(lambda: pb.dort(n, precision=prec, want_T=False))
            ms_e, _ = timed(lambda: pb.dort_eigen(F))
            e = eig.cpu().numpy()[0]
            print(json.dumps({"workload": name, "unknowns": int(pb.ntot), "n_alpha": n, "precision": pname,
                              "dort_ms": round(ms, 3), "eigen_ms": round(ms_e, 3), "status": int(st),
                              "significant": int((e > 1e-3 * e[0]).sum()),
                              "top": [float(x) for x in e[:4]]}), flush=True)
        pb.close()
    pb = msd.Problem(W.four_disks())
    rng = np.random.default_rng(0)
    for n in (1024, 2048):
        F = torch.from_numpy(rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))).cuda()
        ms_e, _ = timed(lambda: pb.dort_eigen(F), reps=2)
        print(json.dumps({"workload": f"eigen stage, random {n} x {n} complex F", "n_alpha": n,
                          "eigen_ms": round(ms_e, 3), "householder_launches": 2 * (n - 2)}), flush=True)
    pb.close()


def formulation_timing(reps: int = 5):
    """Integral-equation formulations on the 400-disk workload: the
    preconditioned product (CUDA events around msd_matvec, device buffers)
    with the default rows and with the Brakhage-Werner rows (one
    block-Toeplitz product over 2R columns), FP64 and FP32, R = 1 and 16;
    then a mixed-precision solve to relres 1e-10 with each formulation."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    cl = W.random_cluster_400()
    pb = msd.Problem(cl)
    rng = np.random.default_rng(0)
    for kind in (None, "cfie", "bwie"):
        pb.set_formulation(kind) if kind else pb.set_formulation(None)
        for prec in (msd.MSD_FP64, msd.MSD_FP32):
            for R in (1, 16):
                dt = torch.complex128 if prec == msd.MSD_FP64 else torch.complex64
                x = torch.from_numpy(rng.standard_normal((cl.ntot, R)) + 1j * rng.standard_normal((cl.ntot, R))).to(
                    device="cuda", dtype=dt)
                y = torch.empty_like(x)
                msd.msd_matvec(pb.handle, R, prec, x, y)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    msd.msd_matvec(pb.handle, R, prec, x, y)
                e1.record()
                torch.cuda.synchronize()
                print(json.dumps({"workload": "random400 (M=400, N=20)", "formulation": kind or "default",
                                  "precision": "fp64" if prec == msd.MSD_FP64 else "fp32", "R": R,
                                  "product_ms": round(e0.elapsed_time(e1) / reps, 3)}), flush=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = pb.solve([cl.meta["beta"]], tol=1e-10, precision=msd.MSD_MIXED)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"workload": "random400 (M=400, N=20)", "formulation": kind or "default",
                          "mixed_solve_ms": round(e0.elapsed_time(e1), 1), "iters": int(res.iters[0]),
                          "status": int(res.status)}), flush=True)
    pb.close()


def penetrable_timing(reps: int = 5):
    """Penetrable obstacles on the geometry of the paper's example (400 unit
    disks on a square lattice of spacing 3 without its middle row and column,
    k+ = 1, k- = 2, N = 10, a point source at the origin): the transmission
    product (two block-Toeplitz launches, CUDA events around the C-ABI call
    with device buffers) and the FP64 and mixed solves to relres 1e-10."""
    import numpy as np
    import torch
    from paper_1409_8186_gb300 import msd, workloads as W
    cl = W.penetrable_lattice()
    pb = msd.Problem(cl)
    pb.set_penetrable(2.0)
    rng = np.random.default_rng(0)
    xp = torch.from_numpy(rng.standard_normal((cl.ntot, 1)) + 1j * rng.standard_normal((cl.ntot, 1))).cuda()
    xm = torch.from_numpy(rng.standard_normal((cl.ntot, 1)) + 1j * rng.standard_normal((cl.ntot, 1))).cuda()
    pb.penetrable_matvec(xp, xm)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        pb.penetrable_matvec(xp, xm)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"workload": f"penetrable lattice (M={cl.M}, N={cl.N}, k+=1, k-=2)", "unknowns": 2 * int(pb.ntot),
                      "what": "FP64 transmission product, R=1", "product_ms": round(e0.elapsed_time(e1) / reps, 3)}),
          flush=True)
    th = W.angles(360)
    for prec, name in ((msd.MSD_FP64, "fp64"), (msd.MSD_MIXED, "mixed")):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rp, _, res = pb.solve_penetrable(sources=[[0.0, 0.0]], tol=1e-10, precision=prec, maxit=8000)
        F = pb.farfield(rp, th)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"workload": f"penetrable lattice (M={cl.M}, N={cl.N}, k+=1, k-=2), point source at 0",
                          "precision": name, "solve_and_farfield_ms": round(e0.elapsed_time(e1), 1),
                          "iters": int(res.iters[0]), "relres": float(res.relres[0]), "status": int(res.status),
                          "rcs_db_at_0": float(10 * np.log10(2 * np.pi * abs(F[0, 0, 0].item()) ** 2))}), flush=True)
    pb.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", choices=["matvec", "fp64", "mixed", "sweep600", "tc", "tcs", "recompute"],
                    default=None,
                    help="run a minimal workload for a profiler capture and print no JSON line")
    ap.add_argument("--products", action="store_true",
                    help="print a table (JSON lines) of block-product kernels over the workloads instead")
    ap.add_argument("--products-only", default="",
                    help="with --products: only the workloads whose name contains this text")
    ap.add_argument("--grad", action="store_true",
                    help="print the timing (JSON lines) of the far-field misfit gradient instead")
    ap.add_argument("--batched", action="store_true",
                    help="print FP64 and mixed batched solve times (JSON lines) instead")
    ap.add_argument("--batched-full", action="store_true",
                    help="solve all 256 batched clusters (32 incidences, mixed precision) and print JSON lines")
    ap.add_argument("--groups", type=int, default=8, help="with --batched-full: batched problems of similar M")
    ap.add_argument("--take", type=int, default=256, help="with --batched-full: the smallest TAKE clusters only")
    ap.add_argument("--only-group", type=int, default=-1, help="with --batched-full: run this group only")
    ap.add_argument("--fp64-groups", type=str, default="",
                    help="with --batched-full: comma-separated groups also solved in FP64")
    ap.add_argument("--lattice-solve", type=int, default=0, metavar="R",
                    help="solve the 4000-disk lattice with R incidences (mixed precision) and print a JSON line")
    ap.add_argument("--nearfield", action="store_true",
                    help="print the timing (JSON line) of the near field on a grid instead")
    ap.add_argument("--penetrable", action="store_true",
                    help="print product and solve times (JSON lines) of the penetrable example instead")
    ap.add_argument("--formulations", action="store_true",
                    help="print product and solve times (JSON lines) of the integral-equation formulations instead")
    ap.add_argument("--dort", action="store_true",
                    help="print the timing (JSON lines) of the time-reversal matrix and its eigenvalues instead")
    args = ap.parse_args()
    if args.dort:
        return dort_timing()
    if args.formulations:
        return formulation_timing()
    if args.penetrable:
        return penetrable_timing()
    if args.nearfield:
        return nearfield_timing()
    if args.lattice_solve:
        return lattice_solve(R=args.lattice_solve)
    if args.batched_full:
        fg = tuple(int(v) for v in args.fp64_groups.split(",") if v.strip())
        return batched_full(groups=args.groups, take=args.take, only_group=args.only_group, fp64_groups=fg)
    if args.batched:
        return batched_timing()
    if args.products:
        return products_table(only=args.products_only)
    if args.grad:
        return grad_timing()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_only:
        return profile_only(args.profile_only)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1409_8186_gb300 import msd, workloads as W

    cl = W.random_cluster_400()
    beta = np.array([[cl.meta["beta"]]])
    thetas = W.angles(360)
    pb = msd.Problem(cl)
    h = pb.handle
    cen_d = torch.from_numpy(np.ascontiguousarray(cl.centres)).cuda()
    rad_d = torch.from_numpy(np.ascontiguousarray(cl.radii)).cuda()
    rho = torch.empty((cl.ntot, 1), dtype=torch.complex128, device="cuda")
    F = torch.empty((1, 360, 1), dtype=torch.complex128, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    stats = (msd.msd_stats * 1)()

    def step(precision):
        msd.msd_update_geometry(h, cen_d, rad_d, None)
        o = msd.msd_opts(1e-10, 0, 3000, 0, 0.0, precision, 0)
        st = msd.msd_solve_planewaves(h, 1, beta, o, rho, stats)
        msd.msd_farfield(h, rho, 1, thetas, F)
        return st

    def timed(precision, K, W_):
        for _ in range(W_):
            step(precision)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        msd.msd_matvec_timing(h, 1)
        l0 = msd.msd_kernel_launches()
        sampler = start_clock_sampler(local) if precision == msd.MSD_FP64 else None
        ms, iters, statuses = [], [], []
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            statuses.append(step(precision))
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            iters.append(stats[0].iters)
        clocks = stop_clock_sampler(sampler)
        launches = msd.msd_kernel_launches() - l0
        kms, kl, kfl, kby = msd.msd_matvec_timing(h, 0)
        if dist:
            dist.barrier()
        return dict(ms=ms, iters=iters, status=statuses, relres=stats[0].relres, clocks=clocks, launches=launches,
                    kernel_ms=kms, kernel_launches=kl, kernel_flops=kfl, kernel_bytes=kby)

    r64 = timed(msd.MSD_FP64, args.steps, args.warmup)
    rmx = timed(msd.MSD_MIXED, args.steps, args.warmup)

    total_ms, value = aggregate(sum(r64["ms"]), r64["kernel_bytes"], dist, device="cuda")

    # end to end through the C ABI with host buffers (host->device inputs,
    # device->host densities and far field inside the timed region)
    cen_h = np.ascontiguousarray(cl.centres)
    rad_h = np.ascontiguousarray(cl.radii)
    rho_h = np.empty((cl.ntot, 1), np.complex128)
    F_h = np.empty((1, 360, 1), np.complex128)

    def step_e2e():
        msd.msd_update_geometry(h, cen_h, rad_h, None)
        o = msd.msd_opts(1e-10, 0, 3000, 0, 0.0, msd.MSD_FP64, 0)
        msd.msd_solve_planewaves(h, 1, beta, o, rho_h, stats)
        msd.msd_farfield(h, rho_h, 1, thetas, F_h)

    step_e2e()
    torch.cuda.synchronize()
    msd.msd_matvec_timing(h, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    _, _, _, e2e_bytes = msd.msd_matvec_timing(h, 0)
    h2d = cen_h.nbytes + rad_h.nbytes + beta.nbytes + thetas.nbytes + rho_h.nbytes
    d2h = rho_h.nbytes + F_h.nbytes

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    kern_s = r64["kernel_ms"] * 1e-3
    achieved_tf = r64["kernel_flops"] / kern_s / 1e12 if kern_s > 0 else 0.0
    kern_gbs = r64["kernel_bytes"] / kern_s / 1e9 if kern_s > 0 else 0.0
    mix_kern_s = rmx["kernel_ms"] * 1e-3
    mix_tf = rmx["kernel_flops"] / mix_kern_s / 1e12 if mix_kern_s > 0 else None

    # the other steps of the path, each timed alone after the timed region
    # (CUDA events around 10 calls; update_geometry includes its host-side
    # flag check)
    rhs_buf = torch.empty((cl.ntot, 1), dtype=torch.complex128, device="cuda")
    stage_ms = {}
    for sname, fn in (("k1_k2_update_geometry", lambda: msd.msd_update_geometry(h, cen_d, rad_d, None)),
                      ("k5_rhs_planewave", lambda: msd.msd_rhs_planewave(h, 1, beta, rhs_buf)),
                      ("k6_farfield_360", lambda: msd.msd_farfield(h, rho, 1, thetas, F))):
        fn()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(10):
            fn()
        s1.record()
        torch.cuda.synchronize()
        stage_ms[sname] = round(s0.elapsed_time(s1) / 10, 4)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        smp = OracleSample(cl)
        t_cpu, passes = 0.0, 0
        while t_cpu < 10.0:
            t_cpu += smp.pass_once()
            passes += 1
        smp.close()
        cpu_gbs = smp.bytes_per_pass * passes / t_cpu / 1e9
        cpu = {"value": cpu_gbs, "unit": "GB/s", "cores": smp.cores, "kind": "oracle",
               "sample": smp.description + f"; {passes} passes",
               "ms_per_full_product_extrapolated": t_cpu / passes * 1e3 * cl.M / len(smp.rows)}

    ms_step = total_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}", "l2": "flushed between steps (256 MB write)",
                   "step": "K1 diagonals + K2 generators + K5 rhs + GMRES with K3 products + K6 far field"},
        "hbm_frac_whole_step": value / hbm,
        "solve_ms_fp64": statistics.median(r64["ms"]), "solve_ms_mixed": statistics.median(rmx["ms"]),
        "mixed_speedup": statistics.median(r64["ms"]) / statistics.median(rmx["ms"]),
        "iters_fp64": r64["iters"][-1], "iters_mixed": rmx["iters"][-1],
        "relres_fp64": r64["relres"], "relres_mixed": rmx["relres"],
        "status_fp64": r64["status"][-1], "status_mixed": rmx["status"][-1],
        "stage_ms": stage_ms,
        "matvec_fp64": {"kernel_ms_avg": r64["kernel_ms"] / max(1, r64["kernel_launches"]),
                        "launches": r64["kernel_launches"], "GB_s": kern_gbs, "hbm_frac": kern_gbs / hbm,
                        "TFLOP_s": achieved_tf},
        "matvec_fp32": {"kernel_ms_avg": rmx["kernel_ms"] / max(1, rmx["kernel_launches"]),
                        "launches": rmx["kernel_launches"],
                        "GB_s": rmx["kernel_bytes"] / 2 / mix_kern_s / 1e9 if mix_kern_s > 0 else None,
                        "TFLOP_s": rmx["kernel_flops"] / mix_kern_s / 1e12 if mix_kern_s > 0 else None},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tf / FP64_PEAK_TFLOPS, "traffic": K3_FP64_DRAM_BYTES_PER_LAUNCH,
                     "traffic_source": K3_FP64_TRAFFIC_SOURCE,
                     "kernel": "k_bt_matvec<double2,1,1> (FP64 block-Toeplitz product)",
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"},
        "roofline_mixed": {"bound": "alu", "achieved": mix_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": mix_tf / FP32_PEAK_TFLOPS if mix_tf else None, "traffic": None,
                           "kernel": "FP32 block-Toeplitz product inside the mixed-precision solve "
                                     "(autotuned CUDA-core shape)",
                           "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_bytes / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s / args.steps * 1e3},
        "gpu_launches": int(r64["launches"]),
        "clocks": r64["clocks"],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
