#!/usr/bin/env python
"""Throughput of the stage-parallel Radau IIA heat step on GB300.

Metric: stage-DoF updates per second per IRK step at 1e-10 FGMRES residual
(Q * interior DoFs / time of one full step: stage right-hand side, FGMRES with
the FP32 multigrid preconditioner of Eq. (irk:P), solution update), with the
roofline of the dominant kernel and p50/p99 step latency.

Default workload: 3D heat, degree 3 on 64^3 cells (7,189,057 nodes), Radau IIA
Q=3, tau=1e-3, Chebyshev degree 3, all stages batched, V-cycle replayed from a
CUDA graph, launch shapes autotuned; outer solver (stage operator, Krylov
vectors, stage combinations, update) in native FP64, multigrid in FP32.
Synthetic manufactured-solution data.  One step = one irk_step call.
Multi-GPU: replicas only (each rank advances its own copy of the problem; no
collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synthetic import HEAT3D_K4_N32_Q3, HEAT2D_K2_N16_Q2, HEAT3D_K2_N48_Q3, heat3d_k3_n64  # noqa: E402

WORKLOADS = {w.name: w for w in (HEAT3D_K4_N32_Q3, HEAT2D_K2_N16_Q2, HEAT3D_K2_N48_Q3,
                                 *(heat3d_k3_n64(Q) for Q in (2, 3, 4, 5)))}
HEADLINE = heat3d_k3_n64(3)
METRIC = "stage-DoF updates/s per IRK step at 1e-10 residual"
UNIT = "stage-DoF/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def slowest_rank_ms(ms_total, dist, device):
    """Replicas: the job's timed region is the slowest rank's (max over ranks; one rank: itself)."""
    if dist is None:
        return ms_total
    import torch
    tt = torch.tensor([ms_total], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(units_per_rank, world, ms_step):
    """Whole-job stage-DoF/s: every rank advances its own replica by units_per_rank per step."""
    return world * units_per_rank / (ms_step / 1e3)


FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal, profiling recipe's table; ~2 FMA/clk/SM x 152 x 2.07 GHz x 2)
FF_CEILING_TFLOPS = 152 * 128 * 2.07e9 / 15 * 2 / 1e12  # emulation ceiling of float-float (not a hardware peak)
FP32_PEAK_TFLOPS = 152 * 128 * 2.07e9 * 2 / 1e12       # FP32 FMA: 152 SMs x 128 lanes x 2.07 GHz x 2


def recorded_traffic():
    """ncu DRAM traffic per launch recorded in profiles/, valid only while the kernel source is unchanged."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return rec if h.hexdigest() == rec["source_sha256"] else None
    except Exception:
        return None


def algorithmic_flops_per_cell(dim, k):
    """Flops the stage operator (M u and K u of one stage vector) costs per cell in the DoF-space
    Kronecker form of the tensor-product element matrices: 14 p^4 + 4 p^3 in 3D, 8 p^3 in 2D
    (p = k + 1), the per-unit figure the roofline divides by."""
    p = k + 1
    return 14.0 * p ** 4 + 4.0 * p ** 3 if dim == 3 else 8.0 * p ** 3


def smoother_alu(w, cheb_degree, avg_launch_ms, fp32=True):
    """ALU side of the finest-level smoother's roofline: per launch the level operator on all Q blocks
    in the algorithmic flops of the DoF-space Kronecker form, plus the pointwise epilogue (about 6
    flops per stage-DoF for a Chebyshev step, 1 for the residual), averaged over the launch mix of
    a smoothing: 2m - 1 Chebyshev steps and one residual."""
    m = cheb_degree
    op = algorithmic_flops_per_cell(w.dim, w.degree) * w.cells ** w.dim * w.Q
    epi = ((2 * m - 1) * 6.0 + 1.0) / (2 * m) * w.n_interior * w.Q
    flops = op + epi
    achieved = flops / (avg_launch_ms / 1e3) / 1e12
    peak = FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS
    src = ("derived: 152 SM x 128 FP32 lanes x 2.07 GHz x 2" if fp32 else "nominal FP64 rate of the profiling recipe")
    return {"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_launch": flops, "peak_source": src}


def flops_per_stage_dof(dim, k):
    """Flops the line-fused sum-factorised kernel executes per node and stage vector for M and K.

    d = 3: y contraction 2 (k+2) taps for (My u, Ky u); x contraction 3 (k+1)^2 / k per node
    (Mx g, Kx g + Mx h); z contraction 3 (k+1)^2 / k (Mz, Kz into two outputs); x2 for FMA.
    d = 2: x contraction 2 (k+1)^2 / k, y contraction 3 (k+1)^2 / k.
    """
    p = k + 1
    if dim == 3:
        return 2.0 * (2 * (k + 2) + 3.0 * p * p / k + 3.0 * p * p / k)
    return 2.0 * (2.0 * p * p / k + 3.0 * p * p / k)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"irk_bench_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        with open(self.path) as fh:
            return summarise_clocks(fh)


def summarise_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen active in the CSV lines of
    ClockSampler.FIELDS (nvidia-smi --format=csv,noheader,nounits); None without a valid sample."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for name, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


def _oracle_replica(wd, steps, warmup, barrier, out_q):
    """One host process: the oracle's problem and fast diagonalisation for workload ``wd``, ``warmup``
    untimed exact IRK steps (at least one), then (after every replica is ready) ``steps`` timed steps
    of its own replica; puts the elapsed seconds on ``out_q``."""
    from synthetic import Workload
    from oracle.irk import FastDiag, Problem, step_fastdiag
    w = Workload(**wd)
    prob = Problem(w.dim, w.cells, w.degree, w.Q, w.tau)
    fd = FastDiag(prob)
    y = prob.y0()
    nw = max(1, warmup)
    for i in range(nw):
        y = step_fastdiag(prob, y, i * w.tau, fd)
    barrier.wait()
    t0 = time.perf_counter()
    for i in range(steps):
        y = step_fastdiag(prob, y, (i + nw) * w.tau, fd)
    out_q.put(time.perf_counter() - t0)


def oracle_replicas(w, steps, nproc=None, timeout_s=900, warmup=1):
    """The oracle's exact IRK step (per-mode fast diagonalisation, numpy/scipy) on every host core:
    one single-threaded replica per process (spawned, so no GPU context is inherited), all timed
    together after a common start.  Returns (whole-host stage-DoF/s, processes, s per step)."""
    import dataclasses
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    nproc = cores if nproc is None else nproc
    try:   # bound the replicas by the host memory (about 300 bytes per node and replica, plus 0.3 GB)
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        nproc = max(1, min(nproc, int(avail // (2 * (300 * w.ndofs + 3e8)))))
    except (ValueError, OSError, AttributeError):
        pass
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    try:
        ctx = mp.get_context("spawn")
        barrier, out_q = ctx.Barrier(nproc), ctx.Queue()
        procs = [ctx.Process(target=_oracle_replica, args=(dataclasses.asdict(w), steps, warmup, barrier, out_q))
                 for _ in range(nproc)]
        for pr in procs:
            pr.start()
        times = [out_q.get(timeout=timeout_s) for _ in procs]
        for pr in procs:
            pr.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    per_step = max(times) / steps
    return nproc * w.Q * w.n_interior / per_step, nproc, per_step


def cpu_baseline(w):
    """The oracle on the host cores: one exact IRK step per replica, a replica per core."""
    value, nproc, per = oracle_replicas(w, steps=1)
    return {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"1 exact IRK step of {w.name} on each of {nproc} single-threaded replica processes "
                      f"(per-mode fast diagonalisation, numpy/scipy), timed together after one untimed step; "
                      f"setup excluded",
            "s_per_step_per_replica": per}


def cpu_baseline_one_thread(w, timeout_s=300):
    """The same oracle step on one host thread: one replica process with BLAS/OpenMP pools of one."""
    value, _, per = oracle_replicas(w, steps=1, nproc=1, timeout_s=timeout_s)
    return {"value": value, "unit": UNIT, "cores": 1, "s_per_step": per,
            "sample": "1 exact IRK step, one single-threaded replica process"}


def serving_measure(n_requests, realtime=True, **solver_opts):
    """Serve the seeded request stream (Poisson arrivals at 200/s) through irk_serve: groups of waiting
    same-shape requests share launches and idle handles are reused unless the options say otherwise."""
    import paper_2209_06700_gb300 as pkg
    from synthetic import serving_stream
    reqs = serving_stream(512)[:n_requests]
    t0 = time.perf_counter()
    st, res, _ = pkg.serve(reqs, max_active=16, realtime=realtime, **solver_opts)
    wall = time.perf_counter() - t0
    ok = [r for r in res if r.status == 0]
    lat = sorted(r.latency_ms for r in ok)
    units = sum(q.Q * (q.degree * q.cells - 1) ** q.dim for q, r in zip(reqs, res) if r.status == 0)
    pct = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
    return {"requests": n_requests, "completed": len(ok), "status": st, "p50_ms": pct(0.50), "p99_ms": pct(0.99),
            "mean_ms": sum(lat) / len(lat) if lat else None, "makespan_s": wall,
            "throughput": units / wall, "unit": UNIT,
            "mean_setup_ms": sum(r.setup_ms for r in ok) / max(1, len(ok)),
            "mean_solve_ms": sum(r.solve_ms for r in ok) / max(1, len(ok)),
            "mean_queue_ms": sum(r.queue_ms for r in ok) / max(1, len(ok)),
            "mean_iterations": sum(r.iterations for r in ok) / max(1, len(ok)),
            "mean_group_size": sum(r.group_size for r in ok) / max(1, len(ok)),
            "requests_in_shared_launches": sum(1 for r in ok if r.group_size > 1),
            "handles_reused_fraction": sum(r.handle_reused for r in ok) / max(1, len(ok)),
            "slots": 16, "arrivals": "Poisson 200/s, seed 0" if realtime else "all at t=0",
            "order": "arrival" if solver_opts.get("smallest_first", 1) == 0 else "smallest first"}


def run_reference(args, w):
    """Reference arm: the CPU oracle on the host cores (rank 0 only): one single-threaded replica
    per core, W untimed and K timed exact IRK steps each, whole-host throughput."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    value, nproc, per = oracle_replicas(w, steps=max(1, args.steps), warmup=args.warmup)
    ms = 1e3 * per
    sample = (f"{args.steps} exact IRK steps of {w.name} on each of {nproc} single-threaded replica processes "
              f"(per-mode fast diagonalisation), after {max(1, args.warmup)} untimed steps each")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "dim": w.dim, "degree": w.degree, "cells": w.cells, "Q": w.Q,
                       "tau": w.tau},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(w, steps=3, warm=2, **opts):
    """ms per irk_step of workload w with solver options opts (CUDA events on the solver's stream after
    `warm` untimed steps, inputs resident) and the FGMRES iterations of the timed steps."""
    import torch
    import paper_2209_06700_gb300 as pkg
    stream = torch.cuda.Stream()
    opts.setdefault("cheb_degree", w.cheb_degree)
    s = pkg.Solver(w.dim, w.cells, w.degree, w.Q, w.tau, stream=stream, **opts)
    try:
        y = s.vector()
        with torch.cuda.stream(stream):
            s.interpolate_initial(y, 0.0)
        for i in range(warm):
            s.step(y, i * w.tau)
        its = []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            its.append(s.step(y, (i + warm) * w.tau).iterations)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    finally:
        s.close()
    units = w.Q * w.n_interior
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "fgmres_iterations": sum(its) / len(its), "stage_dofs": units}


def other_workloads(steps=3):
    """The remaining configurations, each timed like the headline one: the 64^3 degree-3 problem for
    Q = 2..5 and in float-float outer arithmetic; the 32^3 degree-4 problem with per-stage launches
    (as its configuration states) and stage-batched; the 48^3 degree-2 Q=3 problem in the LU and the
    directly diagonalised variants; the 2D 16^2 degree-2 problem in FP64 throughout."""
    import paper_2209_06700_gb300 as pkg
    cases = [(heat3d_k3_n64(Q), "lu", {}) for Q in (2, 3, 4, 5)]
    cases += [(heat3d_k3_n64(3), "lu-float-float-outer", dict(op_ff=1))]
    cases += [(HEAT3D_K4_N32_Q3, "lu-per-stage", dict(batched=0)), (HEAT3D_K4_N32_Q3, "lu", {})]
    cases += [(HEAT3D_K2_N48_Q3, "lu", {}), (HEAT3D_K2_N48_Q3, "diag", dict(variant=pkg.IRK_VARIANT_DIAG)),
              (HEAT3D_K2_N48_Q3, "diag-gmg2x2", dict(variant=pkg.IRK_VARIANT_DIAG, pair_precond=1))]
    cases += [(HEAT2D_K2_N16_Q2, "lu-fp64-mg", dict(mg_precision=64))]
    out = {}
    for w, var, opts in cases:
        out[f"{w.name}_{var}"] = timed_steps(w, steps=steps, **opts)
    return out


def accuracy_vs_oracle(w):
    """Max relative error of one GPU step from the initial interpolant against the oracle's exact IRK
    step (per-mode fast diagonalisation), for the native FP64 and the float-float outer arithmetic."""
    import numpy as np
    import torch
    import paper_2209_06700_gb300 as pkg
    from oracle.irk import Problem, step_fastdiag
    prob = Problem(w.dim, w.cells, w.degree, w.Q, w.tau)
    ref = step_fastdiag(prob, prob.y0(), 0.0)
    out = {}
    for name, op_ff in (("fp64_outer", 0), ("float_float_outer", 1)):
        with pkg.Solver(w.dim, w.cells, w.degree, w.Q, w.tau, cheb_degree=w.cheb_degree, op_ff=op_ff) as s:
            y = s.vector()
            s.interpolate_initial(y, 0.0)
            s.step(y, 0.0)
            torch.cuda.synchronize()
            got = y.cpu().numpy()
        out[name] = float(np.abs(got - ref).max() / np.abs(ref).max())
    out["reference"] = "oracle exact IRK step (fast diagonalisation), one step from the interpolant"
    return out


def curved_mesh_workload(w, eps=0.05, steps=3, reps=10):
    """The headline problem on the curved mesh (irk_options.deform = eps): the step (FP64-accurate
    stage operator with the mapping data of every Gauss point, Cartesian preconditioner), and the stage
    operator alone as one launch over all Q stages (mapping data read once per cell) against Q
    per-stage launches (read Q times), each timed with CUDA events on the solver's stream."""
    import numpy as np
    import torch
    import paper_2209_06700_gb300 as pkg
    stream = torch.cuda.Stream()
    s = pkg.Solver(w.dim, w.cells, w.degree, w.Q, w.tau, stream=stream, cheb_degree=w.cheb_degree, deform=eps)
    try:
        Cm, Ck = np.eye(w.Q), w.tau * np.eye(w.Q)
        with torch.cuda.stream(stream):
            u = s.stage_vector()
            u.uniform_(-1.0, 1.0, generator=torch.Generator(device="cuda").manual_seed(0))
            v = torch.zeros_like(u)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        batched = timed(lambda: s.apply_op(u, v, Cm, Ck))
        per_stage = timed(lambda: [s.apply_op(u[i:i + 1], v[i:i + 1], Cm[i:i + 1, i:i + 1], Ck[i:i + 1, i:i + 1])
                                   for i in range(w.Q)])
        y = s.vector()
        with torch.cuda.stream(stream):
            s.interpolate_initial(y, 0.0)
        s.step(y, 0.0)
        its = []
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(steps):
            its.append(s.step(y, (i + 1) * w.tau).iterations)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    finally:
        s.close()
    ncell, nq, nf = w.cells ** w.dim, (w.degree + 1) ** w.dim, 1 + w.dim * (w.dim + 1) // 2
    geo = ncell * nq * nf * 8
    vec = w.n1 ** w.dim * 8
    units = w.Q * w.n_interior
    return {"workload": f"{w.name}_curved", "eps": eps, "value": units / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "fgmres_iterations": sum(its) / len(its),
            "apply": {"ms_batched": batched, "ms_per_stage": per_stage, "stages": w.Q,
                      "mapping_bytes_per_read": geo,
                      "bytes_batched": geo + 2 * w.Q * vec, "bytes_per_stage": w.Q * (geo + 2 * vec),
                      "arithmetic": "native FP64 (the default outer arithmetic), FP64 vectors and mapping "
                                    "data (FP64-pipe bound: the batched launch saves mapping-data traffic, "
                                    "little time)"}}


def fp64_per_stage_baseline(w, cheb, units, steps=3):
    """The same step on the plain GPU path: native FP64 operator and vectors, FP64 V-cycle, one launch
    per stage, no graph replay."""
    r = timed_steps(w, steps=steps, warm=1, cheb_degree=cheb, op_ff=0, mg_precision=64, batched=0, use_graph=0)
    r["path"] = "FP64 operator, FP64 multigrid, per-stage launches, no graph"
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE.name, choices=sorted(WORKLOADS))
    ap.add_argument("--cells", type=int, default=None,
                    help="override the workload's cells per axis (small cases for profiler captures)")
    ap.add_argument("--mg-precision", type=int, default=0, choices=[0, 32, 64],
                    help="multigrid precision: 0 automatic (FP32 up to Q = 5), 32 or 64")
    ap.add_argument("--per-stage", action="store_true", help="per-stage launches (batched=0)")
    ap.add_argument("--variant", default="lu", choices=["lu", "diag"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-fp64-baseline", action="store_true", help="skip the per-stage FP64 GPU step baseline")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the other configurations and the accuracy check against the oracle")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-baseline-requests", type=int, default=512)
    ap.add_argument("--op-ff", type=int, default=0, choices=[0, 1],
                    help="outer solver arithmetic: native FP64 (0, default) or float-float (1)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="time the operator launch shapes at create (1) or keep the cost model's (0)")
    ap.add_argument("--cheb-degree", type=int, default=None)
    ap.add_argument("--smoothing-range", type=float, default=None)
    ap.add_argument("--gs-reorth", type=int, default=0, choices=[0, 1],
                    help="second Gram-Schmidt pass: 0 where needed (default), 1 at every step")
    ap.add_argument("--eig-safety", type=float, default=None)
    ap.add_argument("--curved-only", action="store_true",
                    help="run only the curved-mesh measurement (profiler captures of its operator)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.cells is not None and args.cells != w.cells:
        import dataclasses
        w = dataclasses.replace(w, name=f"heat{w.dim}d_k{w.degree}_n{args.cells}_q{w.Q}", cells=args.cells)
    if args.curved_only:
        print(json.dumps({"curved_mesh": curved_mesh_workload(w)}))
        return
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2209_06700_gb300 as pkg
    from paper_2209_06700_gb300 import _capi
    PROF_NAMES = _capi.PROF_CATEGORIES

    stream = torch.cuda.Stream()
    variant = pkg.IRK_VARIANT_DIAG if args.variant == "diag" else pkg.IRK_VARIANT_LU
    extra = {}
    if args.smoothing_range is not None:
        extra["smoothing_range"] = args.smoothing_range
    if args.gs_reorth:
        extra["gs_reorth"] = 1
    if args.eig_safety is not None:
        extra["eig_safety"] = args.eig_safety
    cheb = w.cheb_degree if args.cheb_degree is None else args.cheb_degree
    mg_bits = args.mg_precision or (32 if w.Q <= 5 else 64)   # the library's automatic choice
    s = pkg.Solver(w.dim, w.cells, w.degree, w.Q, w.tau, stream=stream, cheb_degree=cheb,
                   mg_precision=args.mg_precision, batched=0 if args.per_stage else 1, variant=variant,
                   op_ff=args.op_ff, autotune=args.autotune, **extra)
    lib = _capi.lib()
    y = s.vector()
    with torch.cuda.stream(stream):
        s.interpolate_initial(y, 0.0)
    t = 0.0
    its = []
    for _ in range(args.warmup):
        st = s.step(y, t)
        its.append(st.iterations)
        t += w.tau

    # one profiled step with every category timed (eager: no graph replay while kernels are timed)
    lib.irk_profile(s.h, (1 << len(PROF_NAMES)) - 1)
    s.step(y, t)
    t += w.tau
    cat_ms = {}
    for i, name in enumerate(PROF_NAMES):
        ms, n, nt = _capi.ctypes.c_double(), _capi.ctypes.c_longlong(), _capi.ctypes.c_longlong()
        lib.irk_profile_read(s.h, i, _capi.ctypes.byref(ms), _capi.ctypes.byref(n), _capi.ctypes.byref(nt))
        cat_ms[name] = (ms.value, n.value, nt.value)
    # the dominant single kernel of the step, from the measured times of the categories that hold one
    # kernel template each: the FP64-accurate stage operator (Eq. irk:A) or the finest-level smoother
    single = ("apply64", "mg_op_fine")
    dom = PROF_NAMES.index(max(single, key=lambda c: cat_ms[c][0]))

    # timed region: only the dominant category is bracketed by events; all launches counted
    lib.irk_profile(s.h, 1 << dom)
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_window:
        torch.cuda.profiler.start()
    ev0.record(stream)
    lat = []
    reo = []
    for _ in range(args.steps):
        w0 = time.perf_counter()
        st = s.step(y, t)
        lat.append(1e3 * (time.perf_counter() - w0))
        its.append(st.iterations)
        reo.append(st.reorth_passes)
        t += w.tau
    ev1.record(stream)
    torch.cuda.synchronize()
    if args.profile_window:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms_total = ev0.elapsed_time(ev1)
    launches = 0
    for i in range(len(PROF_NAMES)):
        ms, n, nt = _capi.ctypes.c_double(), _capi.ctypes.c_longlong(), _capi.ctypes.c_longlong()
        lib.irk_profile_read(s.h, i, _capi.ctypes.byref(ms), _capi.ctypes.byref(n), _capi.ctypes.byref(nt))
        launches += n.value
        if i == dom:
            dom_ms, dom_n = ms.value, nt.value
    lib.irk_profile(s.h, 0)
    ms_total = slowest_rank_ms(ms_total, dist, "cuda")
    ms_step = ms_total / args.steps
    units = w.Q * w.n_interior
    value = job_throughput(units, world, ms_step)

    # end to end through the C ABI with host buffers: H2D of y_n, the step, D2H of y_{n+1}
    y_host = torch.empty(s.n, dtype=torch.float64, pin_memory=True)
    y_host.copy_(y.cpu())
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(max(3, args.steps // 3)):
        w0 = time.perf_counter()
        with torch.cuda.stream(stream):
            y.copy_(y_host, non_blocking=True)
        s.step(y, t)
        with torch.cuda.stream(stream):
            y_host.copy_(y, non_blocking=True)
        stream.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - w0))
        t += w.tau
    e2e_step = statistics.median(e2e_ms)

    hbm, hbm_src = peaks()
    traffic_rec = recorded_traffic()
    arith = "ff" if args.op_ff else "double"

    def rec_traffic(kname):
        if traffic_rec and w.name == traffic_rec.get("workload"):
            return traffic_rec["kernels"].get(kname, {}).get("dram_bytes_per_launch")
        return None

    def operator_roofline(avg_ms):
        """The stage operator: algorithmic flops (the DoF-space Kronecker form, (14p^4 + 4p^3) per
        cell and stage, p = k + 1) against
        the FP64 pipe (native FP64) or the float-float emulation ceiling, and its algorithmic bytes
        (16 B per stage-DoF: read u, write v) against measured HBM."""
        flops = algorithmic_flops_per_cell(w.dim, w.degree) * w.cells ** w.dim * w.Q
        executed = flops_per_stage_dof(w.dim, w.degree) * w.n_interior * w.Q
        achieved = flops / (avg_ms / 1e3) / 1e12
        kname = f"op3d_kernel<{arith},{w.degree},DUAL>"
        bytes_ = 16.0 * w.n_interior * w.Q
        r = {"bound": "alu", "achieved": achieved, "unit": "TFLOP/s", "traffic": rec_traffic(kname),
             "kernel": kname, "avg_launch_ms": avg_ms, "flops_per_launch": flops,
             "executed_flops_per_launch": executed,
             "hbm": {"achieved": bytes_ / (avg_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": bytes_ / (avg_ms / 1e3) / 1e9 / hbm, "bytes_per_launch": bytes_,
                     "peak_source": hbm_src}}
        if args.op_ff:
            r.update(peak=FP64_PEAK_TFLOPS, frac=achieved / FP64_PEAK_TFLOPS,
                     peak_source="nominal FP64 rate (the float-float kernel is compared with what native FP64 "
                                 "could reach)",
                     float_float_emulation_ceiling=FF_CEILING_TFLOPS,
                     frac_of_emulation_ceiling=achieved / FF_CEILING_TFLOPS)
        else:
            r.update(peak=FP64_PEAK_TFLOPS, frac=achieved / FP64_PEAK_TFLOPS,
                     peak_source="nominal FP64 rate of the profiling recipe (152 SM x ~2 FP64 FMA/clk x 2.07 GHz "
                                 "x 2); a DFMA probe measured 1.06 TFLOP/s on this GPU",
                     executed_frac=executed / (avg_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS)
        return r

    def smoother_roofline(avg_ms):
        """The finest-level FP32 smoother: algorithmic bytes (16 B per stage-DoF for a Chebyshev step,
        12 B for the residual) against measured HBM, with its ALU side against the FP32 peak."""
        m = cheb
        eb = 4 if mg_bits == 32 else 8
        per_node = ((2 * m - 1) * 4 * eb + 3 * eb) / (2 * m)
        bytes_ = per_node * w.n_interior * w.Q
        ach = bytes_ / (avg_ms / 1e3) / 1e9
        sname = f"op3d_kernel<{'float' if eb == 4 else 'double'},{w.degree},CHEB>"
        return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": rec_traffic(sname), "kernel": sname + " (finest level, Chebyshev steps and residual)",
                "peak_source": hbm_src, "avg_launch_ms": avg_ms, "bytes_per_launch": bytes_,
                "alu": smoother_alu(w, m, avg_ms, fp32=(eb == 4))}

    # the dominant kernel is timed in the timed region; the other single-kernel category from the
    # profiled eager step
    avg_dom = dom_ms / max(1, dom_n)
    if PROF_NAMES[dom] == "apply64":
        roof = operator_roofline(avg_dom)
        sm_ms, _, sm_nt = cat_ms["mg_op_fine"]
        roof_other = smoother_roofline(sm_ms / sm_nt) if sm_nt else None
        roof_other_key = "roofline_smoother"
    else:
        roof = smoother_roofline(avg_dom)
        op_ms, _, op_nt = cat_ms["apply64"]
        roof_other = operator_roofline(op_ms / op_nt) if op_nt else None
        roof_other_key = "roofline_operator"
    roof["timing"] = "CUDA events around each launch of this kernel on the solver stream, timed region"
    roof["selected_by"] = ("largest device time per step among the single-kernel categories "
                           f"(stage operator {cat_ms['apply64'][0]:.2f} ms, finest smoother "
                           f"{cat_ms['mg_op_fine'][0]:.2f} ms in the profiled step)")
    if roof_other:
        roof_other["timing"] = "CUDA events on the solver stream, profiled eager step"
    kry_ms, kry_n, _ = cat_ms["krylov"]
    its_prof = max(1, round(sum(its[-3:]) / 3)) if its else 1
    passes = min(its_prof, round(sum(reo[-3:]) / len(reo[-3:]))) if reo else its_prof
    # Gram-Schmidt in iteration j (j = 1..its, j basis vectors) per element: with the second pass 4j
    # multiply-adds and about 3j + 5 vector reads and writes, without it 2j and 2j + 5 (dots, then
    # the update in place, then the normalisation); the second passes fall on the last iterations,
    # where the basis's estimated loss of orthogonality has grown.  8 bytes per element in either
    # arithmetic.
    js = range(1, its_prof + 1)
    second = lambda j: j > its_prof - passes
    kry_flops = sum((8.0 if second(j) else 4.0) * j for j in js) * w.Q * w.ndofs
    kry_bytes = sum(((3 * j + 5) if second(j) else (2 * j + 5)) * 8.0 for j in js) * w.Q * w.ndofs
    roof_krylov = {"category_ms_per_step": kry_ms, "launches": kry_n, "iterations": its_prof,
                   "second_passes": passes,
                   "hbm": {"achieved": kry_bytes / (kry_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": kry_bytes / (kry_ms / 1e3) / 1e9 / hbm},
                   "alu": {"achieved": kry_flops / (kry_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                           "unit": "TFLOP/s", "frac": kry_flops / (kry_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                           "arithmetic": "float-float" if args.op_ff else "native FP64"}}
    if args.op_ff:
        dtype = "float-float outer (~48 bits) / f32 multigrid"
    else:
        dtype = "f64 outer / f32 multigrid" if mg_bits == 32 else "f64"

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype,
                "data": "synthetic (manufactured solution, seeded)",
                "config": {"workload": w.name, "dim": w.dim, "degree": w.degree, "cells": w.cells, "Q": w.Q,
                           "tau": w.tau, "cheb_degree": cheb, "rtol": 1e-10,
                           "n_interior": w.n_interior, "stage_dofs": units,
                           "launch": "per-stage" if args.per_stage else "stage-batched",
                           "outer_arithmetic": "float-float" if args.op_ff else "fp64",
                           "variant": args.variant, "mg_precision": mg_bits,
                           "parallelism": f"replicas x{world}",
                           "smoothing_range": extra.get("smoothing_range", 10.0),
                           "gs_second_pass": "every step" if args.gs_reorth else "where needed (orthogonality to 2^-16)",
                           "l2": "inputs larger than L2: Krylov basis of several GB > 129 MB; no flush"},
                "latency_ms": {"p50": statistics.median(lat),
                               "p99": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))]},
                "fgmres_iterations": {"mean": sum(its) / len(its), "min": min(its), "max": max(its),
                                      "gs_second_passes_mean": sum(reo) / max(1, len(reo))},
                "e2e": {"value": units / (e2e_step / 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * s.n,
                        "d2h_bytes_per_step": 8 * s.n, "ms_per_step": e2e_step},
                "gpu_launches": launches,
                "roofline": roof,
                roof_other_key: roof_other,
                "roofline_krylov": roof_krylov,
                "category_ms_one_step": {k: round(v[0], 4) for k, v in cat_ms.items()},
                "autotune": pkg.autotune_report().splitlines(),
                "clocks": clk}
        if world == 1 and not args.no_fp64_baseline:
            line["gpu_fp64_per_stage_baseline"] = fp64_per_stage_baseline(w, cheb, units)
        if world == 1 and not args.no_other_workloads:
            line["other_workloads"] = other_workloads()
            line["curved_mesh"] = curved_mesh_workload(HEAT3D_K4_N32_Q3)
            line["accuracy_vs_oracle"] = accuracy_vs_oracle(w)
        if world == 1 and not args.no_serve:
            line["serving"] = serving_measure(args.serve_requests)
            line["serving_arrival_order"] = serving_measure(args.serve_requests, smallest_first=0)
            # the plain per-stage FP64 GPU path (native FP64 operator, FP64 V-cycle, one launch per stage)
            line["serving_fp64_per_stage_baseline"] = serving_measure(
                args.serve_baseline_requests, op_ff=0, mg_precision=64, batched=0, max_group=1, reuse_handles=0,
                smallest_first=0)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
            line["cpu_baseline"]["one_thread"] = cpu_baseline_one_thread(w)
            line["cpu_baseline"]["machine"] = platform.machine()
            line["cpu_baseline"]["host_cores"] = os.cpu_count()
        print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
