"""Benchmark: converged slab S_N solves/s (FPSA source iteration) on the precision workload.

Workload (one step = one pass of the whole path over one problem):
  1 cm slab, 2000 LD cells, S64 Gauss-Legendre, screened-Rutherford scattering
  (eta = 1e-5) expanded to L = 63, sigma_s0 = 1000/cm, sigma_a = 0.01/cm,
  isotropic unit source on z < 0.5, vacuum edges; synthetic, seeded inputs.
  A step is fpsa_set_xs (upload, sweep coefficients, FP block assembly, block
  cyclic-reduction factorization) followed by fpsa_solve to a relative change of
  phi_0 below 1e-10 (FPSA source iteration). Default: mixed precision (FP32 inner
  FPSA solves with tensor-core contractions inside FP64 refinement) and the WFD
  angular Laplacian; the same workload with MPD and with the plain FP64 path is
  reported under "secondary".

  value : solves/s with inputs already resident in device memory (torch CUDA
          tensors passed to the C ABI), device-timed with CUDA events on the
          library's stream.
  e2e   : the same step through the same C ABI with HOST numpy inputs/outputs, so
          the host->device input copies and the device->host flux copy are inside
          the timed region.
  The factors of one step (2000 blocks of 128 x 128: 131 MB in FP32 on the default
  mixed path, 262 MB in FP64) exceed the L2 (126 MB), so each step streams its
  working set from HBM.

Multi-GPU (torchrun): every rank solves its own replica of the problem (the
workload does not shard); value = solves of all ranks / max rank time.

--impl reference runs the FP64 CPU oracle (the only other place this file runs
oracle code) on rank 0 on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

# The oracle's CPU timings are reported as single-core: numpy's BLAS (and any OpenMP
# pool) in this process runs one thread, set before numpy loads its BLAS.
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_var] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "precision_srk_slab: 1 cm, K=2000 LD cells, S64, SRK eta=1e-5, L=63, sigma_s0=1000, sigma_a=0.01, Q=1 on z<0.5, vacuum"
METRIC = "converged slab S_N solves/s (FPSA-SI, tol 1e-10 rel. change of phi_0)"
TOL = 1e-10
# Per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel on this workload, measured by ncu for each row-slice cap of the BCR solve (the
# launch shape that changes its units; one block per SM), keyed by (kernel, precision,
# solve_max_slices). A shape missing here reports traffic null.
NCU_TRAFFIC = {("k_bcr_solve_flow_s", "mixed", 1): 224.14e6, ("k_bcr_solve_flow_s", "mixed", 2): 223.64e6,
               ("k_bcr_solve_flow_s", "mixed", 4): 222.42e6}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, device=None):
    """Max of a per-rank time over all ranks (torch.distributed, any backend); identity
    when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps_per_rank, max_ms):
    """Weak scaling with one replica per rank: units of all ranks / slowest rank's time."""
    return world * steps_per_rank / (max_ms * 1e-3)


def read_golden(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    vals, its10 = [], None
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                if "relative change 1e-10" in line:
                    its10 = int(line.rsplit(":", 1)[1])
                continue
            vals.append(float(line))
    return np.array(vals), its10


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running; start()
    returns once the first sample has arrived (at most 3 s), so that the sampling loop
    is already running when the timed region begins."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
            self.first = threading.Event()
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=3.0)
            n = len(self.lines)
            self.pre = self.lines[n - 1:n]  # the last sample before the timed region
            del self.lines[:n]
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # a timed region shorter than the sampling interval may hold no sample: then the
        # one taken just before it stands in (samples = 0 says so)
        lines = [ln for ln in self.lines if ln]
        in_region = len(lines)
        for ln in lines or getattr(self, "pre", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": in_region}


def run_config(args, world):
    """The workload's `config` object, the same on both arms (how the GPU arm computes,
    its precision and launch shapes, is reported beside it)."""
    return {"workload": WORKLOAD, "laplacian": args.laplacian, "tol": TOL,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": ("working set larger than L2, no flush: each step rewrites and each BCR solve "
                   "launch reads %s" % ("the 262 MB of FP64 factors" if args.precision == "fp64" else
                                        "the 131 MB of FP32 factors and the 17 MB coarse inverse"))}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed as it stands on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import iterations as oit
    from paper_1907_13013_gb300 import inputs
    p = inputs.precision_srk_slab()
    _, n_it = read_golden("precision_srk_slab_fpsa_%s_phi0.txt" % args.laplacian)
    sample_its = 3

    def step():
        t0 = time.perf_counter()
        # FP operator assembly + sparse LU (the setup), then `sample_its` FPSA iterations
        _, n = oit.fpsa_source_iteration(p, args.laplacian, tol=0.0, max_it=sample_its)
        t_all = time.perf_counter() - t0
        t1 = time.perf_counter()
        _, n = oit.fpsa_source_iteration(p, args.laplacian, tol=0.0, max_it=sample_its + 2)
        t_more = time.perf_counter() - t1
        per_it = max((t_more - t_all) / 2.0, 0.0)
        setup = max(t_all - sample_its * per_it, 0.0)
        return setup + n_it * per_it

    for _ in range(args.warmup):
        step()
    est = [step() for _ in range(args.steps)]
    s_per_solve = float(np.mean(est))
    v = 1.0 / s_per_solve
    sample = ("per step: oracle FP setup + %d and %d FPSA iterations, extrapolated to the oracle's %d "
              "iterations to 1e-10 (mean of %d steps)" % (sample_its, sample_its + 2, n_it, args.steps))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * s_per_solve,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": run_config(args, world), "precision": "fp64",
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": v, "unit": "solves/s"},
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline_sample(laplacian):
    """One full oracle solve of the workload (about 10-30 s of single-threaded CPU work)."""
    from oracle import iterations as oit
    from paper_1907_13013_gb300 import inputs
    p = inputs.precision_srk_slab()
    t0 = time.perf_counter()
    _, n = oit.fpsa_source_iteration(p, laplacian, tol=TOL)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "one complete FP64 oracle FPSA-SI (%s) solve of the workload, %d iterations, %.1f s"
                      % (laplacian.upper(), n, dt)}


def _oracle_solve_seconds(laplacian):
    """One complete oracle solve of the workload in this (worker) process; its seconds."""
    from oracle import iterations as oit
    from paper_1907_13013_gb300 import inputs
    p = inputs.precision_srk_slab()
    t0 = time.perf_counter()
    oit.fpsa_source_iteration(p, laplacian, tol=TOL)
    return time.perf_counter() - t0


def _import_oracle(_):
    from oracle import iterations  # noqa: F401
    from paper_1907_13013_gb300 import inputs  # noqa: F401
    return os.getpid()


def cpu_baseline_all_cores(laplacian):
    """Throughput of the oracle on every host core: one complete solve per core at once, in
    processes started by spawn (the parent has a CUDA context), each single-threaded."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_import_oracle, range(cores))
        t0 = time.perf_counter()
        secs = pool.map(_oracle_solve_seconds, [laplacian] * cores)
        wall = time.perf_counter() - t0
    return {"value": cores / wall, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": "%d complete FP64 oracle FPSA-SI (%s) solves of the workload, one per core at once; "
                      "wall %.1f s (single solves %.1f - %.1f s)" % (cores, laplacian.upper(), wall, min(secs),
                                                                     max(secs))}


def balance_defect(p, phi, r, tab):
    """Particle balance of the converged LD solution for right-hand side r: |emission -
    absorption - leakage| / emission (exact for the discrete solution; tab = the S_N tables)."""
    mu, w, M = tab["mu"], tab["w"], tab["M"]
    pos, neg = mu > 0, mu < 0
    jr = (w[pos] * mu[pos]) @ (M[pos] @ phi[r, -1, 1])
    jl = (w[neg] * -mu[neg]) @ (M[neg] @ phi[r, 0, 0])
    h, Q = p["h"], p["Q"][r]
    sa = p["sigma_t"] - p["sigma_s"][:, 0]
    emission = np.sum(h * (Q[:, 0, 0] + Q[:, 1, 0]) / 2)
    absorption = np.sum(sa * h * (phi[r, :, 0, 0] + phi[r, :, 1, 0]) / 2)
    return float(abs(emission - absorption - jl - jr) / emission)


def scale_secondary(binding, inputs, dev, stream, hbm, bf16, precisions, K=20000, methods=("fpsa", "gmres"),
                    inner=0):
    """The Scale workload (full size: K = 20000, S256, L = 255, HG g = 0.99, c = 0.9999,
    64 seeded sources): one set_xs and one solve per (precision, method), FPSA-SI and
    GMRES(30) right-preconditioned by the FP solve, timed by the host clock around both,
    with CUDA events around every launch (the library's profiler) for the per-kernel
    times; the particle balance of the converged flux for 3 of the right-hand sides.
    A smaller K (same recipe) serves the ncu captures of its kernels."""
    import torch
    p = inputs.scale_slab(K=K)
    K, N, L, R = p["h"].size, p["N"], p["L"], p["Q"].shape[0]
    tab = binding.tables(N, L, "mpd")
    out = {"workload": "scale_slab: 1 cm, K=%d, S256, L=255, HG g=0.99, c=0.9999, sigma_t=100, "
                       "64 rhs Q~U[0,1), vacuum, MPD, tol 1e-10" % K, "solves": {}}
    d_st = torch.tensor(p["sigma_t"], device=dev)
    d_ss = torch.tensor(p["sigma_s"], device=dev)
    d_q = torch.tensor(p["Q"], device=dev)
    phi = torch.zeros((R, K, 2, L + 1), dtype=torch.float64, device=dev)
    for prec in precisions:
        ctx = binding.Context([K], p["h"], N, L, n_rhs=R, laplacian="mpd", precision=prec, device=dev.index,
                              stream=stream.cuda_stream)
        for meth, kw in [m for m in (("fpsa", {"inner_iterations": inner}), ("gmres", {"restart": 30}))
                         if m[0] in methods]:
            ctx.profile_enable(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_xs(d_st, d_ss, d_q)
            try:
                _, st = ctx.solve(meth, tol=TOL, max_iterations=400, raise_on_notconv=False, out=phi, **kw)
            except binding.FpsaError as e:  # e.g. the FP64 GMRES(30) basis does not fit beside the FP64 factors
                out["solves"]["%s_%s" % (prec, meth)] = {"status": e.code, "error": str(e)}
                continue
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            prof = ctx.profile_read()
            ph = phi.cpu().numpy()
            phases = {k: v for k, v in prof.items() if v["timed"]}
            dom = max(phases, key=lambda k: phases[k]["ms"])
            per = phases[dom]["ms"] / phases[dom]["timed"]
            esize = 4 if prec == "mixed" else 8
            n2 = 2 * N
            if dom == "bcr_solve":
                # the factors once per solve (every eliminated cell: A^{-1} forward, its inflow
                # columns backward, two couplings), whatever the number of right-hand sides
                byt = esize * K * (n2 * n2 + n2 * N + 2 * (N // 2) ** 2)
                kname = "k_bcr_solve_flow"
                if ctx.get_tuning()["solve_engine"] == 2:
                    # tensor-core solve: the split factors (4 bytes an element) once per tile of
                    # 64 right-hand sides, and the vector passes (rhs read and Y written forward,
                    # Y read and written backward) of every right-hand side
                    kname = "k_bcr_solve_tc"
                    byt = K * (-(-R // 64) * 4 * (n2 * n2 + n2 * N + 4 * (N // 2) ** 2) + 4 * R * 4 * n2)
                roof = {"kernel": kname, "bound": "hbm", "achieved": byt / (per * 1e-3) / 1e9,
                        "peak": hbm, "unit": "GB/s", "algorithmic_bytes": byt}
            elif dom == "contract" and prec == "mixed":
                # tensor-core contractions, split BF16 with three products: an N x N GEMM over
                # every column (K x 2 per rhs) is 3 x 2 N^2 flop a column; FPSA-SI launches two
                # such GEMMs per contraction launch, a GMRES operator four in three launches
                gemms = 2.0 if meth == "fpsa" else 4.0 / 3.0
                fl = gemms * 3 * 2.0 * N * N * 2 * K * R
                roof = {"kernel": "k_tc_*_big (tensor-core contractions)", "bound": "tensor",
                        "achieved": fl / (per * 1e-3) / 1e12, "peak": bf16, "unit": "TFLOP/s",
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)"}
            elif dom == "contract":
                # 2 N (L+1) flop per column, K x 2 columns per rhs, 64 rhs, per contraction launch
                fl = 2.0 * N * (L + 1) * 2 * K * R
                roof = {"kernel": "contractions (SIMT)", "bound": "alu", "achieved": fl / (per * 1e-3) / 1e12,
                        "peak": 1.20, "unit": "TFLOP/s", "peak_source": "FP64 FMA-chain probe on GB300 (1.20 TFLOP/s)"}
            elif dom == "residual" and prec == "mixed" and ctx.get_tuning()["residual_engine"] == 2:
                # the tensor-core residual: two contractions of 36 BF16 digit-pair products of
                # 2 N^2 flop per column; a refinement step launches the residual and the
                # accumulation of the correction, so the phase's launches are two per step
                fl = 2 * 36 * 2.0 * N * N * 2 * K * R / 2
                roof = {"kernel": "k_mixed_residual_tc", "bound": "tensor", "achieved": fl / (per * 1e-3) / 1e12,
                        "peak": bf16, "unit": "TFLOP/s",
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)",
                        "note": "achieved over the residual phase's launch pairs (residual + accumulation)"}
            elif dom == "residual" and prec == "mixed":
                # the FP64 refinement residual: both contractions fold the mirror ordinates, N^2
                # FP64 multiply-adds per column; a refinement step launches the residual and the
                # accumulation of the correction, so the phase's launches are two per step
                fl = 2.0 * N * N * 2 * K * R / 2
                roof = {"kernel": "k_mixed_residual", "bound": "alu", "achieved": fl / (per * 1e-3) / 1e12,
                        "peak": 1.20, "unit": "TFLOP/s", "peak_source": "FP64 FMA-chain probe on GB300 (1.20 TFLOP/s)",
                        "note": "achieved over the residual phase's launch pairs (residual + accumulation)"}
            else:
                roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s"}
            if roof.get("achieved") is not None:
                roof["frac"] = roof["achieved"] / roof["peak"]
            roof["avg_launch_ms"] = per
            sweep_roof = None
            if "sweep" in phases and phases["sweep"]["timed"]:
                # one sweep = the maps and apply launches; algorithmic bytes per cell-angle:
                # the source read and the flux written at both LD nodes (4 values)
                t_sweep = phases["sweep"]["ms"] / (phases["sweep"]["timed"] / 2.0)
                byt_s = 4 * esize * K * N * R
                sweep_roof = {"kernel": "k_sweep_maps + k_sweep_apply", "bound": "hbm", "ms_per_sweep": t_sweep,
                              "algorithmic_bytes": byt_s, "achieved": byt_s / (t_sweep * 1e-3) / 1e9, "peak": hbm,
                              "unit": "GB/s", "frac": byt_s / (t_sweep * 1e-3) / 1e9 / hbm}
            out["solves"]["%s_%s" % (prec, meth)] = {
                "sweep_roofline": sweep_roof,
                "value": 1.0 / wall, "unit": "solves/s (64 rhs each)", "wall_s": wall, "setup_ms": st["setup_ms"],
                "solve_ms": st["solve_ms"], "iterations": st["iterations"], "outer_iterations": st["outer_iterations"],
                "sweeps": st["sweeps"], "status": st["status"],
                "cell_angles_per_s": st["cell_angles"] / wall,
                "profile_ms": {k: round(v["ms"], 1) for k, v in phases.items()}, "roofline": roof,
                "balance_defect_max_rhs_0_17_63": max(balance_defect(p, ph, r, tab) for r in (0, 17, R - 1))}
        ctx.close()
        torch.cuda.empty_cache()
    return out


def batching_secondary(binding, inputs, n_slabs, hbm, mode="graph"):
    """The first n_slabs of the seeded 4096-slab Batching recipe through the batch driver
    (groups by (N, L), memory-bounded waves; each round of waves, one per N, solved as
    one CUDA graph launch): wall time of context creation, upload, assembly,
    factorization and solve, after one untimed run (and the same with the waves solved
    from host threads on concurrent streams, for comparison); the
    particle balance of every converged slab; then one more pass with CUDA events around
    every launch (the library's profiler), its groups one after another, for the roofline
    of the BCR solve (the dominant kernel) of the largest-N group."""
    import torch
    from paper_1907_13013_gb300 import batch
    probs = inputs.batch_slabs(n_slabs, seed=0)

    def run(graph):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", graph=graph).solve(tol=TOL,
                                                                                            max_iterations=200)
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    graph = mode == "graph"
    run(graph)  # untimed
    (phis, stats), wall = run(graph)
    # the same slabs with every wave's solve driven from its own host thread and stream
    (phis_t, _), wall_t = run(False) if graph else ((phis, stats), wall)
    agree = max(float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)[..., 0]).max())
                for a, b in zip(phis, phis_t))
    cells = sum(q["h"].size for q in probs)
    by_n = {}
    for q in probs:
        by_n[q["N"]] = by_n.get(q["N"], 0) + 1
    tabs = {}
    defect = 0.0
    for q, ph in zip(probs, phis):
        if q["N"] not in tabs:
            tabs[q["N"]] = binding.tables(q["N"], q["L"], "wfd")
        qq = dict(q, Q=q["Q"][None])
        defect = max(defect, balance_defect(qq, np.asarray(ph)[None], 0, tabs[q["N"]]))
    # profiled pass: groups one at a time (max_streams=1), so the event pairs time each
    # kernel alone
    _, pst = batch.BatchSolver(probs, precision="mixed", laplacian="wfd", max_streams=1,
                               profile=True).solve(tol=TOL, max_iterations=200)
    nmax = max(by_n)
    roof = None
    grp = [w for w in pst if w["N"] == nmax]
    if grp:
        ms = sum(w["profile"]["bcr_solve"]["ms"] for w in grp)
        nl = sum(w["profile"]["bcr_solve"]["timed"] for w in grp)
        # one BCR solve reads, for every cell of the group: A^{-1} ((2N)^2 forward), its
        # 2N x N inflow columns (backward) and two N/2 x N/2 couplings, FP32
        byt_per_solve = [4 * w["cells"] * ((2 * nmax) ** 2 + 2 * nmax * nmax + 2 * (nmax // 2) ** 2) for w in grp]
        solves = [w["profile"]["bcr_solve"]["timed"] for w in grp]
        byt = sum(b * n for b, n in zip(byt_per_solve, solves))
        achieved = byt / (ms * 1e-3) / 1e9
        roof = {"kernel": "k_bcr_solve_flow (N = %d group, 2N = %d)" % (nmax, 2 * nmax), "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "avg_launch_ms": ms / max(nl, 1), "algorithmic_bytes_per_launch": byt / max(nl, 1),
                "phase_ms": {k: round(sum(w["profile"][k]["ms"] for w in grp), 1) for k in grp[0]["profile"]
                             if grp[0]["profile"][k]["timed"]}}
    return {"workload": "batch_slabs(%d, seed=0): the first %d of the seeded 4096-slab recipe (K ~ U{100..5000}, "
                        "N in {16,32,64,128}, L = N-1, two HG regions), mixed WFD, tol 1e-10" % (n_slabs, n_slabs),
            "value": n_slabs / wall, "unit": "slabs/s", "wall_s": wall, "cells": int(cells),
            "mode": ("one CUDA graph launch per round of waves (every N's refinement loop a device-side while node)"
                     if graph else "every wave's solve from its own host thread and stream"),
            "graph_rounds": 1 + max(s.get("graph_round", 0) for s in stats) if graph else None,
            "threads_value": n_slabs / wall_t, "threads_vs_graph_max_rel_diff": agree,
            "slabs_per_N": {str(k): v for k, v in sorted(by_n.items())}, "waves": len(stats),
            "balance_defect_max": defect, "roofline": roof}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--laplacian", default="wfd", choices=["mpd", "wfd"])
    ap.add_argument("--no-secondary", action="store_true", help="skip the MPD and FP64 comparison runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", default="auto", choices=["library", "auto"],
                    help="launch shapes: the library's own, or those fpsa_autotune picks on this workload "
                         "(before the warm-up, outside the timed region)")
    ap.add_argument("--no-scale", action="store_true", help="skip the full-size Scale workload line")
    ap.add_argument("--scale-fp64", action="store_true", help="add the FP64 forms to the Scale line (minutes)")
    ap.add_argument("--batch-only", type=int, default=0, metavar="B",
                    help="run only the Batching line on the first B slabs of the recipe and print it: the small "
                         "case of the Batching kernels' ncu captures")
    ap.add_argument("--scale-inner", type=int, default=0,
                    help="Scale line: FP32 FPSA iterations per FP64 refinement step (0: the library's default)")
    ap.add_argument("--scale-methods", default="fpsa,gmres", help="Scale line: methods, comma-separated")
    ap.add_argument("--batch-mode", default="graph", choices=["graph", "threads"],
                    help="Batching line: one CUDA graph per round of waves, or the waves from host threads")
    ap.add_argument("--scale-only", type=int, default=0, metavar="K",
                    help="run only the Scale recipe with K cells (mixed FPSA-SI and GMRES(30)) and print its "
                         "line: the small case of the Scale kernels' ncu captures")
    ap.add_argument("--batch-slabs", type=int, default=256, help="Batching line: slabs of the recipe (0: skip)")
    ap.add_argument("--solve-slices", type=int, default=0, choices=[0, 1, 2, 4],
                    help="row-slice cap of the BCR solve after tuning (0: keep the tuned / library value)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    if world > 1:
        dist.barrier()
    from paper_1907_13013_gb300 import binding, inputs

    if args.scale_only or args.batch_only:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    if args.batch_only:
        out = batching_secondary(binding, inputs, args.batch_only, peaks.get("hbm_gbs", 6800.0), args.batch_mode)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.scale_only:
        out = scale_secondary(binding, inputs, dev, torch.cuda.current_stream(), peaks.get("hbm_gbs", 6800.0),
                              peaks.get("bf16_tflops_sustained", 1676.4),
                              ("mixed", "fp64") if args.scale_fp64 else ("mixed",), K=args.scale_only,
                              methods=tuple(args.scale_methods.split(",")), inner=args.scale_inner)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return

    p = inputs.precision_srk_slab()
    K, N, L = p["h"].size, p["N"], p["L"]
    stream = torch.cuda.current_stream()
    ctx = binding.Context([K], p["h"], N, L, laplacian=args.laplacian, precision=args.precision,
                          device=local, stream=stream.cuda_stream)
    d_st = torch.tensor(p["sigma_t"], device=dev)
    d_ss = torch.tensor(p["sigma_s"], device=dev)
    d_q = torch.tensor(p["Q"][None], device=dev)
    d_phi = torch.zeros((1, K, 2, L + 1), dtype=torch.float64, device=dev)
    h_st = torch.tensor(p["sigma_t"]).pin_memory().numpy()
    h_ss = torch.tensor(p["sigma_s"]).pin_memory().numpy()
    h_q = torch.tensor(p["Q"][None]).pin_memory().numpy()
    h_phi = torch.zeros((1, K, 2, L + 1), dtype=torch.float64).pin_memory().numpy()
    stats = {}

    def step_device():
        ctx.set_xs(d_st, d_ss, d_q)
        _, s = ctx.solve("fpsa", tol=TOL, out=d_phi)
        stats.update(s)

    def step_host():
        ctx.set_xs(h_st, h_ss, h_q)
        _, s = ctx.solve("fpsa", tol=TOL, out=h_phi)
        stats.update(s)

    def timed(fn, k):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dev)

    if args.tune == "auto":
        ctx.set_xs(d_st, d_ss, d_q)
        ctx.autotune(tol=TOL, repeats=3)
    if args.solve_slices:
        ctx.set_tuning(dict(ctx.get_tuning(), solve_max_slices=args.solve_slices))
    shape = ctx.get_tuning()
    for _ in range(args.warmup):
        step_device()
    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile_enable(False)  # reset launch counters, no events
    ms = timed(step_device, args.steps)
    prof_counts = ctx.profile_read()
    clocks = sampler.stop()
    launches = sum(v["launches"] for v in prof_counts.values())
    dev_stats = dict(stats)
    # end to end: host inputs / outputs through the same C ABI
    for _ in range(1):
        step_host()
    ms_e2e = timed(step_host, args.steps)
    # per-kernel durations: the same steps again with CUDA events around every launch
    ctx.profile_enable(True)
    ms_prof = timed(step_device, args.steps)
    prof = ctx.profile_read()
    ctx.profile_enable(False)

    # parity of the benchmarked result against the stored oracle flux
    ref, its_ref = read_golden("precision_srk_slab_fpsa_%s_phi0.txt" % args.laplacian)
    phi0 = d_phi[0, :, :, 0].cpu().numpy().ravel()
    rel_err = float(np.abs(phi0 - ref).max() / np.abs(ref).max())

    # roofline of the dominant kernel class (algorithmic bytes / FLOPs per launch)
    esize = 4 if args.precision == "mixed" else 8
    n2 = 2 * N
    phases = {k: v for k, v in prof.items() if v["timed"]}
    dom = max(phases, key=lambda k: phases[k]["ms"])
    per_launch_ms = phases[dom]["ms"] / phases[dom]["timed"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    if dom == "bcr_solve":
        # forward: every eliminated cell below the coarse level reads its full (2N)^2
        # inverse; backward: its 2N x N inflow columns; plus its N/2 x N/2 couplings (2 per
        # cell); the coarse cells (those the library's coarse step covers, the rule of
        # plan_coarse: the lowest level c with ceil(K / 2^c) <= N/4 and two levels above
        # it, staged FP32 solves of one slab) are one read of the dense inverse G
        nl = max(1, (K - 1).bit_length())
        m_c = 0
        if (2 * N) * (2 * N) * esize <= 64 * 1024:
            for c in range(1, nl - 1):
                if -(-K // (1 << c)) <= N // 4:
                    m_c = -(-K // (1 << c))
                    break
        kf = K - m_c
        byt = esize * (kf * n2 * n2 + kf * n2 * N + 2 * kf * (N // 2) ** 2 + (m_c * n2) ** 2)
        achieved = byt / (per_launch_ms * 1e-3) / 1e9
        kname = "k_bcr_solve_flow_s" if (2 * N) * (2 * N) * esize <= 64 * 1024 else "k_bcr_solve_flow"
        traffic = NCU_TRAFFIC.get((kname, args.precision, shape["solve_max_slices"]))
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic, "algorithmic_bytes": byt}
    elif dom == "bcr_invert":
        flops = 2.0 * n2 ** 3 * K / 12.0  # per launch: K blocks over 12 launches on average
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        peak = 74.0 if esize == 4 else 1.20  # FMA-chain probe on this GB300 (not in MEASURED_PEAKS.json)
        roof = {"kernel": "k_bcr_invert_reg", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "FP32 / FP64 FMA-chain probe on GB300 (74 / 1.20 TFLOP/s)"}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None}
    roof["avg_launch_ms"] = per_launch_ms
    roof["peak_source"] = roof.get("peak_source", "MEASURED_PEAKS.json hbm_gbs (STREAM-style copy, burst)")

    secondary = {}
    if not args.no_secondary:
        for name, lap, prec in (("mpd", "mpd", args.precision), ("fp64", args.laplacian, "fp64")):
            if (lap, prec) == (args.laplacian, args.precision):
                continue
            c2 = binding.Context([K], p["h"], N, L, laplacian=lap, precision=prec, device=local,
                                 stream=stream.cuda_stream)
            st2 = {}

            def step2():
                c2.set_xs(d_st, d_ss, d_q)
                _, s = c2.solve("fpsa", tol=TOL, out=d_phi)
                st2.update(s)

            if args.tune == "auto":
                c2.set_xs(d_st, d_ss, d_q)
                c2.autotune(tol=TOL, repeats=2)

            for _ in range(3):
                step2()
            n2steps = 10
            ms2 = timed(step2, n2steps)
            ref2, _ = read_golden("precision_srk_slab_fpsa_%s_phi0.txt" % lap)
            err2 = float(np.abs(d_phi[0, :, :, 0].cpu().numpy().ravel() - ref2).max() / np.abs(ref2).max())
            secondary[name] = {"laplacian": lap, "precision": prec, "value": whole_job_rate(world, n2steps, ms2),
                               "unit": "solves/s", "steps": n2steps, "ms_per_step": ms2 / n2steps,
                               "iterations": st2["iterations"],
                               "setup_ms": st2["setup_ms"], "solve_ms": st2["solve_ms"],
                               "max_rel_err_vs_oracle": err2, "tuning": c2.get_tuning()}
            c2.close()

    if not args.no_secondary and rank == 0 and world == 1:
        if not args.no_scale:
            secondary["scale"] = scale_secondary(binding, inputs, dev, stream, hbm,
                                                 peaks.get("bf16_tflops_sustained", 1676.4),
                                                 ("mixed", "fp64") if args.scale_fp64 else ("mixed",),
                                                 methods=tuple(args.scale_methods.split(",")), inner=args.scale_inner)
        if args.batch_slabs > 0:
            secondary["batching"] = batching_secondary(binding, inputs, args.batch_slabs, hbm, args.batch_mode)

    value = whole_job_rate(world, args.steps, ms)
    h2d = 8 * (K + K * (L + 1) + 2 * K * (L + 1))
    d2h = 8 * 2 * K * (L + 1)
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64 (bf16x3 tensor-core contractions)",
        "data": "synthetic",
        "config": run_config(args, world), "precision": args.precision,
        "tuning": dict(shape, source=args.tune),
        "cell_angles_per_s": dev_stats["cell_angles"] * world * args.steps / (ms * 1e-3),
        # the same numerator over the sweep kernels' own event time
        "sweep_cell_angles_per_s": (dev_stats["cell_angles"] * world * args.steps
                                    / (phases["sweep"]["ms"] * 1e-3) if phases.get("sweep") else None),
        "iterations": dev_stats["iterations"], "oracle_iterations_1e-10": its_ref,
        "setup_ms": dev_stats["setup_ms"], "solve_ms": dev_stats["solve_ms"],
        "max_rel_err_vs_oracle": rel_err,
        "e2e": {"value": whole_job_rate(world, args.steps, ms_e2e), "unit": "solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roof,
        "profile": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["timed"] / args.steps}
                    for k, v in phases.items()},
        "profiled_ms_per_step": ms_prof / args.steps,
        "clocks": clocks,
        "secondary": secondary,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_sample(args.laplacian)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.laplacian)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
