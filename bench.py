"""Benchmark: SSP-RK3 steps of the hybrid residual on one or more GB300s.

A "step" is one three-stage SSP Runge-Kutta step, i.e. three passes of the
whole hot path (linear candidate + detector, tagging + compaction, CWENOZ,
MUSCL, Harten bound, fluxes) plus the stage updates, over the whole mesh.
Metric: cell-residual evaluations per second (3 per cell per step).

Default workload: the 2D four-state quadrant Riemann problem on the seeded
mixed triangle/quadrilateral mesh of the unit square (408 x 408 quads, half
of them cut into triangles: 249,601 cells), order 3 (r = 2), HLLC, FP32
operators with FP64 Runge-Kutta accumulation, hybrid scheme.  The JSON line
also carries hybrid vs pure CWENOZ and FP32 vs FP64 at orders 3 and 5.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank advances its own replica of the workload
(no collective on the data path); value = all ranks' cell-residuals / max
time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-residuals/s (hybrid vs CWENOZ, FP32 vs FP64) and % of HBM roofline"
UNIT = "cell-residuals/s"
L2_FLUSH_BYTES = 256 << 20


# DRAM traffic of k_linear per cell, from one ncu capture of the kernel
# (dram__bytes_read.sum + dram__bytes_write.sum of a launch / its cells; the
# kernel reads per-cell data only, so traffic scales with the cells).  A figure
# holds only while the kernel's sources (its header and what it includes) are
# those the capture ran: their hash is stored beside it, and a mismatch
# reports null.
KERNEL_SOURCES = ("k_linear.cuh", "device_common.cuh", "kernels.cuh", "tma.cuh", "physics.cuh")
TRAFFIC = {
    # the 249,601-cell quadrant mesh itself, order 3 hybrid FP32: 99,144,960 B
    # read + 8,281,856 B written per launch
    ("quadrant", 3, "fp32", "hybrid"): {"bytes_per_cell": 430.394, "sources": "a1f3e660e08e75d8"},
    # 110,592-cell turbulence mesh, order 4 hybrid FP32: 447,680,256 B read +
    # 43,790,336 B written
    ("turbulence", 4, "fp32", "hybrid"): {"bytes_per_cell": 4443.998, "sources": "a1f3e660e08e75d8"},
}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2510_25906_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(workload, order, precision, scheme, cells):
    t = TRAFFIC.get((workload, order, precision, scheme))
    if not t or t["sources"] != kernel_source_hash():
        return None
    return int(round(t["bytes_per_cell"] * cells))


def replica_rate(units_per_rank: float, seconds: float, world: int, dist=None, device=None) -> tuple[float, float]:
    """Whole-job rate of N independent replicas (one per rank, no collective
    on the data path): every rank processed `units_per_rank` in its own
    `seconds`; the job took the slowest rank's time.  Returns
    (all ranks' units / max seconds over ranks, that max)."""
    slowest = seconds
    if world > 1:
        import torch
        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        slowest = float(t.item())
    return world * units_per_rank / slowest, slowest


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alu_peaks(H):
    """FMA ceilings of the CUDA cores, measured here (hfv_fma_rate): FP64
    DFMA, FP32 FFMA and packed FFMA2, FLOP/s."""
    return {"fp64_flops": H.fma_rate("fp64", 100.0), "fp32_flops": H.fma_rate("fp32", 100.0),
            "fp32x2_flops": H.fma_rate("fp32x2", 100.0)}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def _env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def _oracle_sample(mesh, band=0.05):
    vm = mesh.vertex_means()
    return np.nonzero(np.abs(vm[:, 1] - 0.5) < band)[0].astype(np.int64)


def _oracle_block(mesh, k):
    """a k x k x k block of cells about the domain's centre (3D sample)"""
    vm = mesh.vertex_means()
    lo, hi = vm.min(axis=0), vm.max(axis=0)
    h = (hi - lo) / np.cbrt(mesh.n_cells)
    inside = np.all(np.abs(vm - 0.5 * (lo + hi)) < 0.5 * k * h, axis=1)
    return np.nonzero(inside)[0].astype(np.int64)


def _oracle_steps(mesh, U, order, flux, scheme, steps, warmup, band=0.05, sample=None):
    """Time the FP64 oracle (single thread) on a band of cells across the
    domain centre (every quadrant interface crosses it), or on the given
    sample: one 'step' = three residual evaluations of the sample, the work of
    one SSP-RK3 step there."""
    import oracle as O
    om = O.Mesh(mesh)
    s = O.Scheme(om, order=order, flux=flux, scheme=scheme)
    smp = _oracle_sample(mesh, band) if sample is None else sample
    for _ in range(max(1, warmup)):
        s.residual(U, sample=smp)          # the first call also builds the operators
    t0 = time.perf_counter()
    for _ in range(steps):
        for _ in range(3):
            s.residual(U, sample=smp)
    dt = time.perf_counter() - t0
    return 3.0 * smp.size * steps / dt, smp.size, dt


def _oracle_worker(mesh, U, order, flux, scheme, steps, smp, barrier, out):
    import oracle as O
    s = O.Scheme(O.Mesh(mesh), order=order, flux=flux, scheme=scheme)
    s.residual(U, sample=smp)              # builds this chunk's operators
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        for _ in range(3):
            s.residual(U, sample=smp)
    out.put((smp.size, time.perf_counter() - t0))


def _oracle_steps_parallel(mesh, U, order, flux, scheme, steps, band, procs):
    """The oracle on `procs` host processes at once (spawned, one per core),
    the band split into contiguous chunks: cell-residuals of all chunks over
    the longest process's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    smp = _oracle_sample(mesh, band)
    chunks = np.array_split(smp, procs)
    barrier = ctx.Barrier(procs)
    out = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(mesh, U, order, flux, scheme, steps, c, barrier, out))
          for c in chunks]
    for p in ps:
        p.start()
    try:
        res = [out.get(timeout=900) for _ in ps]
    finally:
        for p in ps:
            p.join(timeout=5)
            if p.is_alive():
                p.terminate()
    cells = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return 3.0 * cells * steps / t, cells, t


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_2510_25906_gb300 import inputs as I
    mesh, U, dflt = I.workload(args.workload, args.scale)
    v, ns, dt = _oracle_steps(mesh, U, args.order, dflt["flux"], args.scheme, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, mesh, note="FP64 CPU oracle, single thread", precision="fp64"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{ns} cells (|y - 0.5| < 0.05) of the {mesh.n_cells}-cell mesh, 3 residual "
                                   f"evaluations per step, operators built before timing"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, mesh, **extra):
    names = {"quadrant": "2D quadrant Riemann problem, seeded mixed tri/quad mesh of [0,1]^2",
             "turbulence": "3D decaying turbulence, periodic [0,2pi]^3, uniform hexahedra",
             "density_wave": "2D smooth density wave, periodic jittered triangles"}
    # the workload names the problem only; the arithmetic is the "precision" key
    # (the reference arm runs the same workload in the FP64 oracle)
    cfg = {"workload": f"{names[args.workload]}, {mesh.n_cells} cells, order {args.order} {args.scheme}, "
                       f"SSP-RK3",
           "cells": mesh.n_cells, "order": args.order, "scheme": args.scheme, "precision": args.precision,
           "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{args.gpus}"}
    cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# GPU timing
# ---------------------------------------------------------------------------

class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"hfv_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


FACES = np.array([0, 3, 4, 4, 6, 5, 5], np.int64)     # faces per cell type (index = HFV_* type)
# floating-point operations of one HLLC evaluation at a face point plus its
# weighted accumulation (counted from physics.cuh: an FMA counts 2, a divide
# or square root 1), 2D / 3D
RIEMANN_FLOP = {2: 100, 3: 125}


def path_model(mesh, s, b):
    """Algorithmic bytes and flops per cell-residual of the whole path, the
    per-class terms averaged over the mesh's cells:
      B_lin   = nv b (U_i) + 4 M (stencil) + Q M b (L) + (nf/2)(d+1) b (face
                normals and areas) + b (1/|V|) + 4 nf (face neighbours) + nv b (R)
      B_cweno = (N M (P) + N(N+1)/2 (OI) + nf d Md (directional) + Q d (Phi_lin)) b
                + nf Md (directional indices)
      B_muscl = (d Md (gradient operator) + Q d (Phi_lin)) b
    (gathers of neighbour states are L2 hits; face-state round trips are not
    counted), and the flops
      F_lin   = 2 Q M nv (candidate contraction) + Q F_riemann
      F_cweno = 2 N M nv (p_opt) + 2 nf d Md nv (directional) + nv (N(N+1) + nf d(d+1)) (indicators)
      F_muscl = 2 d Md nv."""
    d, nv, M, N, Md = mesh.dim, s.nv, s.M, s.N, s.Md
    nf = FACES[mesh.cell_type].astype(np.float64)
    Q = nf * s.nfp
    B_lin = nv * b + 4 * M + Q * M * b + (nf / 2) * (d + 1) * b + b + 4 * nf + nv * b
    B_cw = (N * M + N * (N + 1) / 2 + nf * d * Md + Q * d) * b + nf * Md
    B_mu = (d * Md + Q * d) * b
    F_lin = 2 * Q * M * nv + Q * RIEMANN_FLOP[d]
    F_cw = 2 * N * M * nv + 2 * nf * d * Md * nv + nv * (N * (N + 1) + nf * d * (d + 1))
    F_mu = np.full_like(nf, 2.0 * d * Md * nv)
    return {"B_lin": float(B_lin.mean()), "B_cweno": float(B_cw.mean()), "B_muscl": float(B_mu.mean()),
            "F_lin": float(F_lin.mean()), "F_cweno": float(F_cw.mean()), "F_muscl": float(F_mu.mean())}


def queue_fractions(torch, g, U, dev):
    """CWENOZ and MUSCL queue lengths / cells of one residual at state U (FP64 device)."""
    Ur = (U.float() if g.fp32 else U).contiguous()
    g.residual(Ur)
    torch.cuda.synchronize(dev)
    counts, _ = g.queues()
    return counts[0] / g.n_cells, counts[1] / g.n_cells


def path_roofline(mesh, g, value, fq, peaks):
    """The metric's "% of HBM roofline": B_alg x cell-residuals/s / peak, with
    B_alg = B_lin + f_cweno B_cweno + f_muscl B_muscl at the measured queue
    fractions.  FP64 paths are also held against the FP64 FMA ceiling: the
    bound is the lower of HBM / B_alg and FP64 FLOP/s / F_alg."""
    b = 4 if g.fp32 else 8
    pm = path_model(mesh, g, b)
    f_cw, f_mu = fq
    B = pm["B_lin"] + f_cw * pm["B_cweno"] + f_mu * pm["B_muscl"]
    F = pm["F_lin"] + f_cw * pm["F_cweno"] + f_mu * pm["F_muscl"]
    hbm = peaks["hbm_gbs"] * 1e9
    out = {"b_alg_per_cell_residual": B, "flop_per_cell_residual": F, "f_cweno": f_cw, "f_muscl": f_mu,
           "achieved_GBs": B * value / 1e9, "peak_GBs": peaks["hbm_gbs"], "frac_hbm": B * value / hbm,
           "hbm_ceiling": hbm / B}
    if not g.fp32 and peaks.get("fp64_flops"):
        alu = peaks["fp64_flops"] / F
        out.update({"fp64_peak_tflops": peaks["fp64_flops"] / 1e12, "fp64_alu_ceiling": alu,
                    "frac_fp64_alu": value / alu})
        out["bound"] = "fp64_alu" if alu < out["hbm_ceiling"] else "hbm"
        out["frac"] = value / min(alu, out["hbm_ceiling"])
    else:
        out["bound"] = "hbm"
        out["frac"] = out["frac_hbm"]
    return out


def _k1_bytes(mesh, s, b):
    """Algorithmic bytes of one launch of the linear-candidate + detector
    kernel: per cell U_i (nv b), stencil ids (4 M), L (Q M b), threshold (b),
    face-point states written (Q nv b), face counts + offsets + class (10).
    Stencil neighbours' states are L2 hits (U is read from DRAM once)."""
    nf = np.array([0, 3, 4, 4, 6, 5, 5], np.int64)[mesh.cell_type]     # faces per cell type
    Q = nf * s.nfp
    per = s.nv * b + 4 * s.M + Q * s.M * b + b + Q * s.nv * b + 10
    return int(per.sum())


def kernel_roofline(mesh, g, times, peak, peak_kind, traffic):
    """The candidate kernel's achieved bandwidth: the algorithmic bytes of one
    launch -- B_lin of every cell (path_model; the candidate kernel reads
    U_i, the stencil ids and L, the flux kernel the face geometry and writes
    R) -- over the launch's average duration by events.  The kernel's own
    byte count, which adds the face states it writes, is reported beside it."""
    k_ms, k_n = times["linear"]
    b = 4 if g.fp32 else 8
    blin = path_model(mesh, g, b)["B_lin"] * mesh.n_cells
    dur = k_ms / k_n * 1e-3 if k_n else None
    achieved = blin / dur / 1e9 if dur else None
    tot_ms = sum(v[0] for v in times.values())
    return {"kernel": "k_linear (gather + linear candidate + detector + Harten test)", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback",
            "algorithmic_bytes_per_launch": int(round(blin)),
            "kernel_bytes_per_launch": _k1_bytes(mesh, g, b),
            "kernel_bytes_frac": (_k1_bytes(mesh, g, b) / dur / 1e9 / peak) if dur else None,
            "avg_launch_us": 1e3 * k_ms / max(k_n, 1),
            "kernel_share": {k: round(v[0] / tot_ms, 4) for k, v in times.items() if v[1]}}


def time_steps(H, torch, g, U0, steps, warmup, cfl, dev, with_timer=False):
    """Warm up, capture one step in a CUDA graph, then time `steps` replays,
    each bracketed by CUDA events on the launching stream, with an L2 flush
    (untimed) before each."""
    st = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    U = torch.tensor(U0, dtype=torch.float64, device=dev)
    with torch.cuda.stream(st):
        for _ in range(warmup):
            g.step(U, cfl=cfl, stream=st)
        torch.cuda.synchronize(dev)
        n0 = H.launch_count()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            g.step(U, cfl=cfl)
        per_step_launches = H.launch_count() - n0
        graph.replay()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(st)
            graph.replay()
            ev[k][1].record(st)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    return ms, wall, per_step_launches * steps, U


def kernel_pass(H, torch, g, U0, steps, cfl, dev):
    """Eager steps with the library's per-kernel event timer (events recorded
    on the launch stream around every kernel), L2 flushed between steps; the
    kernels of a step are queued behind a ~2 ms sleep kernel, so they run
    back to back as in the graph-timed region.  Each kernel's time is the
    median over the steps of its per-step total, times the number of steps:
    a step whose launches waited on a slow host does not move it."""
    st = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    U = torch.tensor(U0, dtype=torch.float64, device=dev)
    g.kernel_timer(True)
    g.kernel_times(reset=True)
    per_step = []
    with torch.cuda.stream(st):
        for _ in range(steps):
            flush.zero_()
            # a bounded sleep kernel keeps the GPU busy while the host enqueues
            # the step, so no event pair spans a host launch gap
            torch.cuda._sleep(4_000_000)
            g.step(U, cfl=cfl, stream=st)
            per_step.append(g.kernel_times(reset=True))
    g.kernel_timer(False)
    return median_kernel_times(per_step)


def median_kernel_times(per_step):
    """{kernel: (ms, launches)} per step -> {kernel: (median per-step ms x
    steps, all launches)}: a kernel's steady-state total, robust to a few
    steps that waited on the host."""
    times = {}
    for k in per_step[0]:
        n = sum(t[k][1] for t in per_step)
        if n:
            times[k] = (float(np.median([t[k][0] for t in per_step])) * len(per_step), n)
        else:
            times[k] = (0.0, 0)
    return times


def e2e_pass(g, torch, U0, steps, cfl):
    """hfv_advance_host per step: pinned host state in, one step, state out."""
    Uh = torch.tensor(U0, dtype=torch.float64).pin_memory().numpy()
    g.advance_host(Uh, 1, cfl=cfl)
    t0 = time.perf_counter()
    for _ in range(steps):
        g.advance_host(Uh, 1, cfl=cfl)
    return time.perf_counter() - t0, Uh.nbytes


def turbulence_variants(H, I, torch, dev, args, peaks):
    """The 3D workload: 128^3 periodic hexahedra, order 4, HLLC.  The seeded
    initial field is first advanced `pre` steps (hybrid, FP32; untimed input
    preparation) so that compressible structures have formed; every variant
    then times `steps` steps from that same state, L2 flushed between steps,
    with its path roofline.  The FP32 hybrid also carries the candidate
    kernel's roofline, the end-to-end rate through hfv_advance_host and the
    oracle on a block of the mesh."""
    mesh, U0, d = I.workload("turbulence", args.turbulence_scale)
    gm = H.Mesh(mesh)
    cells, cfl, steps = mesh.n_cells, d["cfl"], args.turbulence_steps
    out = {"workload": f"3D decaying turbulence, periodic [0,2pi]^3, {cells} hexahedra, order 4, HLLC, SSP-RK3",
           "pre_steps": args.turbulence_pre, "steps": steps}
    g = H.Scheme(gm, order=4, flux="hllc", scheme="hybrid", precision="fp32", step_chain=1)
    U = torch.tensor(U0, device=dev)
    for _ in range(args.turbulence_pre):
        g.step(U, cfl=cfl)
    torch.cuda.synchronize(dev)
    Upre = U.cpu().numpy()
    cls = torch.empty(cells, dtype=torch.uint8, device=dev)
    g.residual(U.float().contiguous(), class_out=cls)
    out["classes_at_start"] = np.bincount(cls.cpu().numpy(), minlength=4).tolist()
    peak, peak_kind = _peaks()
    for scheme in ("hybrid", "cweno"):
        for prec in ("fp32", "fp64"):
            gv = g if (scheme, prec) == ("hybrid", "fp32") else H.Scheme(gm, order=4, flux="hllc", scheme=scheme,
                                                                           precision=prec, step_chain=1)
            ms, _, _, Ufin = time_steps(H, torch, gv, Upre, steps, 3, cfl, dev)
            value = 3.0 * cells * steps / (ms * 1e-3)
            a0 = queue_fractions(torch, gv, torch.tensor(Upre, device=dev), dev)
            a1 = queue_fractions(torch, gv, Ufin, dev)
            del Ufin
            entry = {"value": value, "ms_per_step": ms / steps,
                     "path": path_roofline(mesh, gv, value, (0.5 * (a0[0] + a1[0]), 0.5 * (a0[1] + a1[1])), peaks)}
            if (scheme, prec) == ("hybrid", "fp32"):
                times = kernel_pass(H, torch, gv, Upre, steps, cfl, dev)
                entry["k_linear"] = kernel_roofline(mesh, gv, times, peak, peak_kind,
                                                    _traffic("turbulence", 4, "fp32", "hybrid", cells))
                e2e_s, nbytes = e2e_pass(gv, torch, Upre, steps, cfl)
                entry["e2e"] = {"value": 3.0 * cells * steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                                "d2h_bytes_per_step": nbytes, "api": "hfv_advance_host"}
                if args.cpu_baseline:
                    smp = _oracle_block(mesh, 10)
                    v, ns, dt = _oracle_steps(mesh, Upre, 4, "hllc", "hybrid", 50, 1, sample=smp)
                    entry["cpu_baseline"] = {
                        "value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": _cpu_model(),
                        "sample": f"{ns} cells (a 10^3 block at the domain centre) of the {cells}-cell mesh, 50 steps x "
                                  f"3 residual evaluations, FP64, operators built before timing ({dt:.1f} s timed)"}
            out[f"{scheme}_{prec}"] = entry
            if gv is not g:
                del gv
                torch.cuda.empty_cache()
    # the viscous residual (Sec. 2; the paper's turbulence run is the viscous
    # Taylor-Green vortex at Re = 1600): mu0 = 1/1600 at the reference
    # temperature T0 = p/rho = 1/gamma of this field, hybrid, FP32
    gv = H.Scheme(gm, order=4, flux="hllc", scheme="hybrid", precision="fp32", mu0=1.0 / 1600.0, t0=1.0 / 1.4,
                  prandtl=0.71, step_chain=1)
    ms, _, _, Ufin = time_steps(H, torch, gv, Upre, steps, 3, cfl, dev)
    value = 3.0 * cells * steps / (ms * 1e-3)
    a0 = queue_fractions(torch, gv, torch.tensor(Upre, device=dev), dev)
    a1 = queue_fractions(torch, gv, Ufin, dev)
    out["hybrid_fp32_viscous"] = {"value": value, "ms_per_step": ms / steps, "mu0": 1.0 / 1600.0,
                                  "path_euler_bytes": path_roofline(mesh, gv, value,
                                                                    (0.5 * (a0[0] + a1[0]), 0.5 * (a0[1] + a1[1])), peaks)}
    del gv, Ufin
    torch.cuda.empty_cache()
    if args.order6:
        try:
            out["order6"] = order6_variants(H, torch, dev, mesh, gm, Upre, cfl, args, peaks)
        except H.HfvError as e:   # recorded, not fatal: the rest of the line stands
            out["order6"] = {"error": str(e)}
            torch.cuda.empty_cache()
    return out


def order6_variants(H, torch, dev, mesh, gm, Upre, cfl, args, peaks):
    """The paper's headline comparison (Sec. 3.6): Hybrid6 against CWENOZ6 on
    128^3 hexahedra (order 6, r = 5: M = 112 stencil cells, 55 coefficients,
    54 face points per cell), FP32, HLLC, from the same pre-advanced field;
    `order6_steps` SSP-RK3 steps each, L2 flushed between steps."""
    out = {"workload": f"{mesh.n_cells} hexahedra, order 6, HLLC, SSP-RK3, FP32", "steps": args.order6_steps}
    t0 = time.perf_counter()
    g = H.Scheme(gm, order=6, flux="hllc", scheme="hybrid", precision="fp32", step_chain=1)
    out["setup_s"] = time.perf_counter() - t0
    out["setup_ms_stencils_operators"] = g.setup_ms()
    out["device_bytes"] = g.device_bytes()
    for scheme in ("hybrid", "cweno"):
        g.set_kind(scheme)      # the same stencils and operators
        ms, _, _, Ufin = time_steps(H, torch, g, Upre, args.order6_steps, 3, cfl, dev)
        value = 3.0 * mesh.n_cells * args.order6_steps / (ms * 1e-3)
        a0 = queue_fractions(torch, g, torch.tensor(Upre, device=dev), dev)
        a1 = queue_fractions(torch, g, Ufin, dev)
        out[scheme] = {"value": value, "ms_per_step": ms / args.order6_steps,
                       "path": path_roofline(mesh, g, value, (0.5 * (a0[0] + a1[0]), 0.5 * (a0[1] + a1[1])), peaks)}
        if scheme == "hybrid":
            cls = torch.empty(mesh.n_cells, dtype=torch.uint8, device=dev)
            g.residual(torch.tensor(Upre, device=dev).float().contiguous(), class_out=cls)
            out["classes_at_start"] = np.bincount(cls.cpu().numpy(), minlength=4).tolist()
        del Ufin
    del g
    torch.cuda.empty_cache()
    out["speedup_hybrid_vs_cweno"] = out["cweno"]["ms_per_step"] and out["cweno"]["ms_per_step"] / out["hybrid"]["ms_per_step"]
    return out


def mixed_variants(H, I, torch, dev, args):
    """The 3D mixed-element workload: an open unit cube of tetrahedra, prisms,
    pyramids and hexahedra (inputs.mixed_element_mesh), order 3, HLLC, a
    Gaussian density pulse ahead of a Mach 2 shock; hybrid and pure CWENOZ
    in FP32 and the hybrid in FP64, `steps` steps each, L2 flushed between
    steps, with the candidate kernel's share of the measured HBM bandwidth
    for the FP32 hybrid."""
    t0 = time.perf_counter()
    mesh = I.mixed_element_mesh(args.mixed_n)
    U0 = I.shock_pulse_state(mesh)
    gm = H.Mesh(mesh)
    cells, steps = mesh.n_cells, args.mixed_steps
    counts = np.bincount(mesh.cell_type, minlength=7)
    out = {"workload": f"open unit cube, {cells} cells: {counts[3]} tetrahedra, {counts[5]} prisms, {counts[6]} pyramids, "
                       f"{counts[4]} hexahedra; order 3, HLLC, SSP-RK3, Mach 2 shock and density pulse",
           "cells": int(cells), "steps": steps, "mesh_s": round(time.perf_counter() - t0, 2)}
    for scheme, prec in (("hybrid", "fp32"), ("cweno", "fp32"), ("hybrid", "fp64")):
        g = H.Scheme(gm, order=3, flux="hllc", scheme=scheme, precision=prec, step_chain=1)
        ms, _, _, _ = time_steps(H, torch, g, U0, steps, 2, 0.5, dev)
        entry = {"value": 3.0 * cells * steps / (ms * 1e-3), "ms_per_step": ms / steps}
        if (scheme, prec) == ("hybrid", "fp32"):
            times = kernel_pass(H, torch, g, U0, steps, 0.5, dev)
            k_ms, k_n = times["linear"]
            kb = _k1_bytes(mesh, g, 4)
            ach = kb / (k_ms / k_n * 1e-3) / 1e9
            peak, _ = _peaks()
            entry["k_linear"] = {"achieved_GBs": ach, "frac": ach / peak, "avg_launch_us": 1e3 * k_ms / k_n,
                                 "algorithmic_bytes_per_launch": kb}
            cls = torch.empty(cells, dtype=torch.uint8, device=dev)
            g.residual(torch.tensor(U0, dtype=torch.float32, device=dev), class_out=cls)
            out["classes_at_start"] = np.bincount(cls.cpu().numpy(), minlength=4).tolist()
        out[f"{scheme}_{prec}"] = entry
        del g
        torch.cuda.empty_cache()
    return out


def batched_variants(H, I, torch, dev, args):
    """Independent open 2D problems of uneven size and order (the batched
    workload): one batched mesh and scheme per order, all advanced by one
    hfv_step_many per step (one stream per order, one CUDA graph), against
    one scheme per problem stepped one after another (also graph-captured).
    Cell-residuals/s of the whole batch, FP32, CFL 0.5, each problem with
    its own CFL step."""
    t0 = time.perf_counter()
    P = I.batched_problems(args.batched, seed=5)
    t_gen = time.perf_counter() - t0
    cells = sum(p["mesh"].n_cells for p in P)
    groups = {}
    for k, p in enumerate(P):
        groups.setdefault(p["order"], []).append(k)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.Stream(device=dev)

    def timed(step_fn, steps, warmup):
        with torch.cuda.stream(st):
            for _ in range(warmup):
                step_fn(st)
            torch.cuda.synchronize(dev)
            n0 = H.launch_count()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=st):
                step_fn(st)
            launches = H.launch_count() - n0
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(st)
                graph.replay()
                ev[k][1].record(st)
            torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in ev), launches

    t0 = time.perf_counter()
    schemes, states = [], []
    for order, ks in sorted(groups.items()):
        gm = H.Mesh.batch([P[k]["mesh"] for k in ks])
        schemes.append(H.Scheme(gm, order=order, flux="hllc", precision="fp32", step_chain=1))
        states.append(torch.tensor(np.concatenate([P[k]["U"] for k in ks], axis=1), device=dev))
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    shapes = {}
    if args.batched_autotune:
        for (order, _), g, U in zip(sorted(groups.items()), schemes, states):
            shapes[int(order)] = g.autotune(U.float().contiguous(), reps=3)
    t_tune = time.perf_counter() - t0
    ms_b, l_b = timed(lambda s: H.step_many(schemes, states, cfl=0.5, stream=s), args.batched_steps, 3)
    hist = np.zeros(4, np.int64)
    for g, U in zip(schemes, states):
        cls = torch.empty(g.n_cells, dtype=torch.uint8, device=dev)
        g.residual(U.float().contiguous(), class_out=cls)
        hist += np.bincount(cls.cpu().numpy(), minlength=4)
    del schemes, states
    torch.cuda.empty_cache()

    t0 = time.perf_counter()
    single = []
    for p in P:
        g = H.Scheme(H.Mesh(p["mesh"]), order=p["order"], flux="hllc", precision="fp32", step_chain=1)
        single.append((g, torch.tensor(p["U"], device=dev)))
    t_setup1 = time.perf_counter() - t0

    def each(s):
        for g, U in single:
            g.step(U, cfl=0.5, stream=s)
    ms_1, l_1 = timed(each, args.batched_steps, 3)
    del single
    torch.cuda.empty_cache()
    K = args.batched_steps
    return {"workload": f"{len(P)} independent open 2D problems, jittered triangle meshes of 1k-200k cells "
                        f"(log-uniform), orders {sorted(groups)} uniform, sine waves and rotated Sod tubes, HLLC, FP32",
            "problems": len(P), "cells": int(cells), "per_order": {int(o): len(ks) for o, ks in sorted(groups.items())},
            "classes": hist.tolist(), "steps": K,
            "batched": {"value": 3.0 * cells * K / (ms_b * 1e-3), "ms_per_step": ms_b / K,
                        "launches_per_step": l_b, "form": "one batched mesh per order, hfv_step_many, one graph"},
            "per_problem": {"value": 3.0 * cells * K / (ms_1 * 1e-3), "ms_per_step": ms_1 / K,
                            "launches_per_step": l_1, "form": "one scheme per problem, hfv_step each, one graph"},
            "speedup": ms_1 / ms_b, "autotuned_shapes": shapes,
            "setup_s": {"inputs": t_gen, "batched": t_setup, "autotune": t_tune, "per_problem": t_setup1}}


def adjoint_variants(H, I, torch, dev, args):
    """The adjoint workload: dJ/dU0 of J = sum |V| rho^2 after K checkpointed
    SSP-RK3 steps (FP64, order 3 hybrid, HLLC, Venkatakrishnan's limiter with
    K = 5, classes frozen along the forward trajectory) on an open unit cube
    of 6 n^3 jittered tetrahedra with a Gaussian density pulse ahead of a
    planar Mach 2 shock.  Reports the time of the forward sweep and of the
    backward sweep (stage recomputation and three residual VJPs per step), the
    VJP rate, and the gradient against central differences of the whole
    K-step trajectory (classes and step sizes frozen) along two directions:
    a seeded random one and the density pulse."""
    from paper_2510_25906_gb300 import adjoint as A
    n = args.adjoint_n
    m, U0 = I.adjoint_problem(n)
    gm = H.Mesh(m)
    g = H.Scheme(gm, order=3, flux="hllc", precision="fp64", limiter="venkatakrishnan", venkat_k=5.0)
    U = torch.tensor(U0, device=dev)
    J = A.density_square_integral(gm.volumes())
    # one warm call of each kernel family
    A.rk3_gradient(g, U, 1, J, cfl=0.5)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    Jv, dJ, UN, dts = A.rk3_gradient(g, U, args.adjoint_steps, J, cfl=0.5)
    torch.cuda.synchronize(dev)
    total = time.perf_counter() - t0
    # the backward sweep alone: forward once more, then time a VJP burst
    cls = torch.empty(m.n_cells, dtype=torch.uint8, device=dev)
    g.residual(U, class_out=cls)
    lam = torch.ones_like(U)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        g.residual_vjp(U, cls, lam)
    e1.record()
    torch.cuda.synchronize(dev)
    vjp_ms = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        g.residual(U, forced=cls)
    e1.record()
    torch.cuda.synchronize(dev)
    res_ms = e0.elapsed_time(e1) / reps
    # one VJP with the per-kernel timer (events around every launch): the
    # forward residual it re-evaluates and the three VJP kernel families
    g.kernel_timer(True)
    g.kernel_times(reset=True)
    g.residual_vjp(U, cls, lam)
    torch.cuda.synchronize(dev)
    kt = {k: v[0] for k, v in g.kernel_times(reset=True).items() if v[1]}
    g.kernel_timer(False)
    vjp_kernels = {k: round(v, 4) for k, v in kt.items() if k.startswith("vjp_")}
    vjp_kernels["forward_residual"] = round(sum(v for k, v in kt.items() if not k.startswith("vjp_")), 4)
    # the stencil gather of the VJP reads, per cell, its own contribution
    # S0 (nv doubles), its inverse-map range (8 bytes) and M (index, nv
    # doubles) contributions, and writes nv doubles of the gradient
    nv, M = U.shape[0], g.M
    b_gather = (2 * nv * 8 + 8 + M * (4 + nv * 8)) * m.n_cells
    peak, _ = _peaks()
    gather = None
    if "vjp_gather" in kt:
        gbs = b_gather / (kt["vjp_gather"] * 1e-3) / 1e9
        gather = {"bound": "hbm", "algorithmic_bytes": int(b_gather), "achieved": gbs, "peak": peak, "unit": "GB/s",
                  "frac": gbs / peak}
    hist = np.bincount(cls.cpu().numpy(), minlength=4).tolist()
    # central differences of the same trajectory (h = 1e-6)
    ccls, W = [], U.clone()
    for h_ in dts:
        _, _, W3, cc = A._stages(g, W, h_)
        ccls.append(cc)
        W = W3.contiguous()

    def traj(Ux):
        W = Ux.clone()
        for cc, h_ in zip(ccls, dts):
            W = A._stages(g, W, h_, classes=cc)[2].contiguous()
        return J(W)[0]
    rng = np.random.default_rng(1)
    cen = torch.tensor(m.vertex_means(), device=dev)
    dirs = {"random": torch.tensor(rng.standard_normal(U.shape), device=dev) * U.abs().mean(dim=1, keepdim=True),
            "pulse": torch.zeros_like(U)}
    dirs["pulse"][0] = torch.exp(-((cen - torch.tensor([0.75, 0.5, 0.5], device=dev)) ** 2).sum(1) / (2 * 0.08 ** 2))
    fd_check = {}
    for name, d in dirs.items():
        fd = (traj(U + 1e-6 * d) - traj(U - 1e-6 * d)) / 2e-6
        an = float((dJ * d).sum().item())
        fd_check[name] = {"central_difference": fd, "adjoint": an, "rel": abs(fd - an) / abs(fd)}
    return {"workload": f"open unit cube, {n}^3 hexahedra cut into {m.n_cells} jittered tetrahedra, Gaussian density pulse ahead "
                        f"of a planar Mach 2 shock, order 3 hybrid, HLLC, Venkatakrishnan K = 5, FP64, classes frozen",
            "fd_check": fd_check,
            "cells": int(m.n_cells), "steps": args.adjoint_steps, "objective": "sum |V| rho^2 after the steps",
            "J": Jv, "grad_norm": float(dJ.norm().item()), "classes_at_start": hist,
            "forward_plus_backward_s": total, "vjp_ms": vjp_ms, "residual_ms": res_ms, "vjp_over_residual": vjp_ms / res_ms,
            "vjp_kernels_ms": vjp_kernels, "vjp_gather_roofline": gather,
            "flux_vjp_ns_per_face_point": (kt["vjp_flux"] * 1e6 / (m.n_cells * 4 * g.nfp)) if "vjp_flux" in kt else None,
            "vjp_cells_per_s": m.n_cells / (vjp_ms * 1e-3), "checkpoint_bytes": int(args.adjoint_steps * U.numel() * 8)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="quadrant", choices=["quadrant", "turbulence", "density_wave"])
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--scheme", default="hybrid", choices=["hybrid", "cweno", "linear", "muscl"])
    ap.add_argument("--variants", type=int, default=1, help="also time hybrid/CWENOZ x FP32/FP64 at orders 3, 5")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--scale", type=int, default=None, help="mesh size parameter (small cases for profiling)")
    ap.add_argument("--turbulence", type=int, default=1, help="also time the 3D workload (rank 0)")
    ap.add_argument("--turbulence-scale", type=int, default=None)
    ap.add_argument("--turbulence-pre", type=int, default=100)
    ap.add_argument("--turbulence-steps", type=int, default=10)
    ap.add_argument("--order6", type=int, default=1, help="also time order 6 hybrid vs CWENOZ on the 3D workload")
    ap.add_argument("--order6-steps", type=int, default=3)
    ap.add_argument("--batched", type=int, default=256, help="problems of the batched workload (0: skip)")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--batched-autotune", type=int, default=1)
    ap.add_argument("--autotune", type=int, default=0, help="tune the main scheme's launch shape before timing")
    ap.add_argument("--adjoint", type=int, default=1, help="also time the checkpointed adjoint (rank 0)")
    ap.add_argument("--mixed", type=int, default=1, help="also time the 3D mixed-element workload (rank 0)")
    ap.add_argument("--mixed-n", type=int, default=48)
    ap.add_argument("--mixed-steps", type=int, default=10)
    ap.add_argument("--adjoint-n", type=int, default=55)
    ap.add_argument("--adjoint-steps", type=int, default=50)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = _env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    import torch.distributed as dist

    import paper_2510_25906_gb300.hfv as H
    from paper_2510_25906_gb300 import build as B
    from paper_2510_25906_gb300 import inputs as I

    if not os.path.exists(H.LIB_PATH):
        B.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    mesh, U0, dflt = I.workload(args.workload, args.scale)
    cfl = dflt["cfl"]
    gm = H.Mesh(mesh)

    def make(order, scheme, precision):
        return H.Scheme(gm, order=order, flux=dflt["flux"], scheme=scheme, precision=precision, step_chain=1)

    g = make(args.order, args.scheme, args.precision)
    tuned = None
    if args.autotune:
        # hfv_autotune on the initial state (outside the timed region)
        Ut = torch.tensor(U0, device=dev, dtype=torch.float32 if g.fp32 else torch.float64)
        tuned = list(g.autotune(Ut, reps=5))
    peak, peak_kind = _peaks()
    peaks = {"hbm_gbs": peak}
    peaks.update(alu_peaks(H))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with Clocks(local) as clk:
        ms, wall, launches, Ufin = time_steps(H, torch, g, U0, args.steps, args.warmup, cfl, dev)
    cells = mesh.n_cells
    value, s_max = replica_rate(3.0 * cells * args.steps, ms * 1e-3, world, dist, dev)
    if world > 1:
        dist.barrier()
    ms_max = 1e3 * s_max

    # class histogram of the final state
    cls = torch.empty(cells, dtype=torch.uint8, device=dev)
    Uf = Ufin.float() if g.fp32 else Ufin
    g.residual(Uf.contiguous(), class_out=cls)
    hist = np.bincount(cls.cpu().numpy(), minlength=4).tolist()

    # the metric's path roofline at the measured class queues (start and end of the timed steps)
    fq0 = queue_fractions(torch, g, torch.tensor(U0, device=dev), dev)
    fq1 = queue_fractions(torch, g, Ufin, dev)
    fq = (0.5 * (fq0[0] + fq1[0]), 0.5 * (fq0[1] + fq1[1]))
    # dominant kernel: linear candidate + detector
    times = kernel_pass(H, torch, g, U0, args.steps, cfl, dev)
    roofline = kernel_roofline(mesh, g, times, peak, peak_kind,
                               _traffic(args.workload, args.order, args.precision, args.scheme, cells))
    roofline["path"] = path_roofline(mesh, g, value / world, fq, peaks)
    roofline["alu_peaks_tflops"] = {k: v / 1e12 for k, v in peaks.items() if k.endswith("flops")}

    # end to end through the C ABI with host buffers
    e2e_s, nbytes = e2e_pass(g, torch, U0, args.steps, cfl)
    e2e_value, _ = replica_rate(3.0 * cells * args.steps, e2e_s, world, dist, dev)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "api": "hfv_advance_host"}

    variants = {}
    if args.variants and rank == 0 and args.workload == "quadrant":
        for order in (3, 5):
            for scheme in ("hybrid", "cweno"):
                for prec in ("fp32", "fp64"):
                    key = f"order{order}_{scheme}_{prec}"
                    if (order, scheme, prec) == (args.order, args.scheme, args.precision):
                        variants[key] = {"value": value / world, "ms_per_step": ms_max / args.steps,
                                         "path": roofline["path"]}
                        continue
                    gv = make(order, scheme, prec)
                    msv, _, _, Uv = time_steps(H, torch, gv, U0, args.steps, args.warmup, cfl, dev)
                    vv = 3.0 * cells * args.steps / (msv * 1e-3)
                    a0 = queue_fractions(torch, gv, torch.tensor(U0, device=dev), dev)
                    a1 = queue_fractions(torch, gv, Uv, dev)
                    variants[key] = {"value": vv, "ms_per_step": msv / args.steps,
                                     "path": path_roofline(mesh, gv, vv, (0.5 * (a0[0] + a1[0]), 0.5 * (a0[1] + a1[1])),
                                                           peaks)}
                    del gv
    turbulence = None
    if args.turbulence and rank == 0:
        turbulence = turbulence_variants(H, I, torch, dev, args, peaks)
    batched = None
    if args.batched and rank == 0:
        batched = batched_variants(H, I, torch, dev, args)
    mixed = None
    if args.mixed and rank == 0:
        mixed = mixed_variants(H, I, torch, dev, args)
    adjoint = None
    if args.adjoint and rank == 0:
        adjoint = adjoint_variants(H, I, torch, dev, args)

    cpu = None
    if args.cpu_baseline and rank == 0 and world == 1:
        v, ns, dt = _oracle_steps(mesh, U0, args.order, dflt["flux"], args.scheme, 50, 1, band=0.2)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": _cpu_model(),
               "sample": f"{ns} cells (|y - 0.5| < 0.2) of the {cells}-cell mesh, 50 steps x 3 residual "
                         f"evaluations, FP64, operators built before timing ({dt:.1f} s timed)"}
        procs = min(16, os.cpu_count() or 1)
        if procs > 1:
            vp, nsp, dtp = _oracle_steps_parallel(mesh, U0, args.order, dflt["flux"], args.scheme, 200, 0.45, procs)
            cpu["all_cores"] = {"value": vp, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{nsp} cells (|y - 0.5| < 0.45) split into {procs} contiguous chunks, one "
                                          f"spawned process each, 200 steps x 3 residual evaluations, FP64 "
                                          f"({dtp:.1f} s for the slowest process)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if g.fp32 else "f64", "data": "synthetic",
                "config": _config(args, mesh, **({"launch_shape": tuned} if tuned else {})), "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(), "classes_final": hist,
                "wall_s_timed": wall, "variants": variants, "turbulence": turbulence, "mixed": mixed, "batched": batched,
                "adjoint": adjoint}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
