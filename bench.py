"""Benchmark: implicit-integrator steps/s on the paper-scale cloth (about 1.65M triangles).

One step = the whole hot path through the C ABI (pc_step): dynamic pattern of the step's
contacts, element evaluation and value assembly, mixed-precision Jacobi-PCG to a
relative residual of 1e-6, state update. Inputs (rest mesh, state, every step's
contact pairs) are resident on the device before timing starts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. With N > 1 (torchrun) every rank runs an independent replica of
the workload ("replicas only": the path does not shard) and rank 0 reports the
aggregate over ranks with the slowest rank's time.

Two further forms of the integrator have their own lines (one GPU):
  --form batched    64 garments (log-uniform 2k..200k triangles) stepped together: one
                    CUDA graph per step with one persistent batched PCG launch
  --form warmstart  learned warm start: train on 2,000 integrator steps of 256 x 256
                    cloths, then step a 708 x 708 cloth with the zero, previous-step and
                    learned initial guesses (and plain FP32 PCG for comparison)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

METRIC = "steps/s at 1.65M tris (assemble+PCG to 1e-6); BSR SpMV GB/s vs 8 TB/s"
FALLBACK_HBM_GBS = 6800.0
# shared-memory bandwidth per SM and clock (bytes), the peak of the cluster solve, which
# works out of the shared memory of the 16 SMs of one thread-block cluster
SMEM_BYTES_PER_CLK = 128
CLUSTER_SMS = 16
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the PCG SpMV,
# from one ncu capture of the current kernel on that workload (mean of 3 launches).
# ncu DRAM read + write bytes per launch of the PCG product, by (workload, storage)
SPMV_DRAM_BYTES = {("stack3x526", "offdiag"): 408.4e6 + 8.7e6}  # steady state (ncu --cache-control none)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stack3x526")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=20000, help="PCG iteration cap per step (short profiling runs)")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "block"])
    ap.add_argument("--storage", default="offdiag", choices=["full", "sym", "sell", "offdiag"],
                    help="matrix layout of the PCG products")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--form", default="step", choices=["step", "batched", "warmstart"])
    ap.add_argument("--no-sequential", action="store_true", help="batched form: skip the one-garment-at-a-time comparison")
    ap.add_argument("--train-steps", type=int, default=2000, help="warmstart form: Adam steps")
    ap.add_argument("--garments", type=int, default=64, help="batched form: number of garments")
    ap.add_argument("--no-fuse", action="store_true", help="two-kernel PCG update (no fused direction step)")
    ap.add_argument("--schedule", default="auto", choices=["auto", "grid", "cluster"],
                    help="PCG schedule: whole solve in one thread-block cluster when the system fits (auto), "
                         "grid-wide kernels, or the cluster only")
    ap.add_argument("--damp-mass", type=float, default=0.0, help="Rayleigh damping alpha (1/s)")
    ap.add_argument("--damp-stiff", type=float, default=0.0, help="Rayleigh damping beta (s)")
    return ap.parse_args()


def make_workload(name: str, damp_mass: float = 0.0, damp_stiff: float = 0.0):
    import dataclasses

    from paper_2008_00409_gb300 import workloads as wk
    wl = wk.WORKLOADS[name]()
    if damp_mass or damp_stiff:
        wl = dataclasses.replace(wl, material=dataclasses.replace(wl.material, damp_mass=damp_mass,
                                                                  damp_stiff=damp_stiff))
    return wl


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
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
            except Exception:
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_hbm():
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------------- CPU oracle sample


PROXIMITY_SAMPLE = 100  # vertices whose oracle query is timed (proximity workloads)


def oracle_step(wl, step: int, tol: float = 1e-6, max_iter: int | None = None):
    """Time the FP64 oracle on one step of the same workload: pattern + assembly, then
    Jacobi-PCG to `tol` (or `max_iter` iterations when given). Returns (t_setup, t_solve,
    iterations, converged). With the proximity query the oracle's brute-force query is
    timed on PROXIMITY_SAMPLE vertices and scaled to all vertices, and the assembly is
    timed without contact elements (a full brute-force query does not fit a bounded
    sample)."""
    import oracle
    om = oracle.Mesh.from_workload(wl)
    t_query = 0.0
    if wl.contact_kind == "proximity":
        from oracle import proximity as px
        rings = px.one_rings(wl.V, wl.tris)
        sample = np.linspace(0, wl.V - 1, PROXIMITY_SAMPLE).astype(np.int64)
        tq = time.perf_counter()
        px.query(wl.x0, wl.tris, wl.material.contact_thickness, vertices=sample, rings=rings)
        t_query = (time.perf_counter() - tq) * wl.V / PROXIMITY_SAMPLE
        pairs, w = np.zeros((0, 4), np.int32), np.zeros((0, 3))
    else:
        pairs, w = wl.contacts(step)
    t0 = time.perf_counter()
    rp, ci, vals, b = om.assemble(wl.x0, wl.v0, pairs, w, wl.h)
    t1 = time.perf_counter()
    if max_iter is None:
        _, iters, rel = oracle.pcg(rp, ci, vals, b, tol=tol, max_iter=200000, check=False)
    else:
        _, iters, rel = oracle.pcg(rp, ci, vals, b, tol=1e-30, max_iter=int(max_iter), check=False)
    t2 = time.perf_counter()
    return t1 - t0 + t_query, t2 - t1, iters, rel <= tol


def cpu_baseline(wl, tol: float):
    """One full step of the FP64 oracle on every host core: measured, not extrapolated."""
    import oracle
    t_setup, t_solve, iters, ok = oracle_step(wl, 1, tol)
    per_step = t_setup + t_solve
    extra = (f" (the brute-force FP32 proximity query timed on {PROXIMITY_SAMPLE} vertices and scaled to "
             f"all; assembly without contact elements)") if wl.contact_kind == "proximity" else ""
    return {"value": 1.0 / per_step, "unit": "steps/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"FP64 C oracle (OpenMP, {oracle.num_threads()} threads), one whole step of {wl.name} "
                       f"(step 1): pattern+assembly {t_setup:.1f} s{extra}, then Jacobi-PCG to {tol:g} in "
                       f"{iters} iterations, {t_solve:.1f} s{'' if ok else ' (not converged)'}; measured, "
                       f"not extrapolated")}


# --------------------------------------------------------------------------- reference arm

REF_SAMPLE_ITERS = 500  # PCG iterations timed per reference step after the first


def run_reference(args):
    """The oracle as the reference arm, on this arm's workload and metric. Its first step
    runs whole (pattern, assembly, FP64 PCG to the tolerance) and gives the oracle's own
    iteration count; each further step times pattern + assembly + REF_SAMPLE_ITERS PCG
    iterations and scales the iterations to that count."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args.workload, args.damp_mass, args.damp_stiff)
    times, n_iter, wall = [], None, time.perf_counter()
    for k in range(args.warmup + args.steps):
        step = k % max(wl.steps, 1)
        if n_iter is None:
            t_setup, t_solve, n_iter, _ = oracle_step(wl, step, args.tol)
            dt = t_setup + t_solve
        else:
            t_setup, t_solve, it, _ = oracle_step(wl, step, args.tol, max_iter=REF_SAMPLE_ITERS)
            dt = t_setup + n_iter * t_solve / max(it, 1)
        if k >= args.warmup:
            times.append(dt)
    wall = time.perf_counter() - wall
    per_step = float(np.mean(times))
    value = 1.0 / per_step
    sample = (f"FP64 C oracle (OpenMP, {oracle.num_threads()} threads): the first step whole (pattern, assembly, "
              f"PCG to {args.tol:g} in {n_iter} iterations); later steps pattern + assembly + "
              f"{REF_SAMPLE_ITERS} PCG iterations, scaled to {n_iter}; {wall:.0f} s of wall time in all")
    out = {"metric": METRIC, "value": value, "unit": "steps/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "V": wl.V, "T": wl.T, "contacts_per_step": wl.n_contacts, "tol": args.tol},
           "cpu_baseline": {"value": value, "unit": "steps/s", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------- ranks


def max_over_ranks(seconds: float, world: int) -> float:
    """The slowest rank's time (every rank gets it); a barrier follows the reduction."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def aggregate_steps_per_s(world: int, steps: int, slowest_seconds: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' steps over the slowest time."""
    return world * steps / slowest_seconds


# --------------------------------------------------------------------------- our arm


def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2008_00409_gb300 import build as cuda_build
    if local == 0:
        cuda_build.build()
    if world > 1:
        dist.barrier()
    from paper_2008_00409_gb300 import pcloth as pc

    wl = make_workload(args.workload, args.damp_mass, args.damp_stiff)
    cl = pc.Cloth(wl)
    prec = pc.PC_PREC_MIXED if args.precision == "mixed" else pc.PC_PREC_FP32
    precond = pc.PC_PRECOND_BLOCK if args.precond == "block" else pc.PC_PRECOND_JACOBI
    storage = {"sym": pc.PC_STORAGE_SYM, "sell": pc.PC_STORAGE_SELL,
               "offdiag": pc.PC_STORAGE_OFFDIAG}.get(args.storage, pc.PC_STORAGE_FULL)
    schedule = {"grid": pc.PC_SCHED_GRID, "cluster": pc.PC_SCHED_CLUSTER}.get(args.schedule, pc.PC_SCHED_AUTO)
    nsteps = args.warmup + args.steps
    proximity = wl.contact_kind == "proximity"
    # random contact sets are inputs (generated before timing); proximity contacts are
    # found by the GPU query at each step's positions, inside the timed step
    contacts = None if proximity else [cl.contacts_device(k % max(wl.steps, 1)) for k in range(nsteps)]
    n_pairs, query_s = [], []
    torch.cuda.synchronize()

    def one_step(k):
        if proximity:
            tq = time.perf_counter()  # the query synchronizes (it returns the pair count)
            pd, wd = cl.proximity()
            query_s.append(time.perf_counter() - tq)
            n_pairs.append(0 if pd is None else int(pd.shape[0]))
        else:
            pd, wd = contacts[k]
        info, st = cl.step(pd, wd, tol=args.tol, precision=prec, warm_start=pc.PC_WARM_PREV,
                           max_iter=args.max_iter, precond=precond, storage=storage, fuse=not args.no_fuse,
                           schedule=schedule, allow_not_converged=True)
        return info

    for k in range(args.warmup):
        one_step(k)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = pc.pc_launch_count(cl.ctx)
    pc.pc_spmv_stats(cl.ctx)  # reset
    pc.pc_assembly_stats(cl.ctx)
    pc.pc_cluster_stats(cl.ctx)
    pc.pc_set_profiling(cl.ctx, True)
    iters, rels, nnzbs = [], [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for k in range(args.warmup, nsteps):
            info = one_step(k)
            iters.append(info.solve.iters)
            rels.append(info.solve.rel_res)
            nnzbs.append(info.nnzb)
        ev1.record(stream)
        torch.cuda.synchronize()
    pc.pc_set_profiling(cl.ctx, False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = pc.pc_launch_count(cl.ctx) - launches0
    n_spmv, spmv_ms, spmv_blocks = pc.pc_spmv_stats(cl.ctx)
    nnzb = int(nnzbs[-1]) if nnzbs else 0
    n_asm, asm_ms = pc.pc_assembly_stats(cl.ctx)
    n_cl, cl_iters, cl_ms = pc.pc_cluster_stats(cl.ctx)
    elapsed = max_over_ranks(elapsed, world)
    value = aggregate_steps_per_s(world, args.steps, elapsed)

    # roofline of the dominant kernel: the PCG SpMV q = A p in the difference form.
    # Algorithmic bytes per launch: the blocks the product reads and their column indices
    # (40 per block: the off-diagonal blocks with the default storage, whose diagonal
    # blocks would multiply p_i - p_i = 0; all blocks with the full matrix), row pointers
    # (4 (V+1)), the difference diagonal (4 V: one scalar per row, m_i I; the few rows next
    # to pins read 36 more bytes, not counted), p read once and q written (float4, 16 V each)
    V = wl.V
    diag_bytes = 4 * V if args.storage in ("offdiag", "full") else 36 * V
    spmv_bytes = 40 * spmv_blocks + 4 * (V + 1) + diag_bytes + 16 * V + 16 * V
    avg_spmv_s = (spmv_ms / 1e3) / max(n_spmv, 1)
    achieved = spmv_bytes / avg_spmv_s / 1e9 if n_spmv else None
    peak, peak_src = measured_hbm()
    clocks = clk.summary()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": SPMV_DRAM_BYTES.get((wl.name, args.storage)),
                "kernel": {"sell": "spmv_sell_kernel<true>", "sym": "spmv_sym_kernel<true>"}.get(
                    args.storage, "spmv_kernel<true,true,CAPR>") + " (q = A p, difference form, with p.q; "
                    + args.storage + " storage; CAPR = 14 or 18 blocks per row per stage, chosen per "
                    "solve from the largest tile)",
                "blocks_per_launch": int(spmv_blocks),
                "bytes_per_launch": spmv_bytes, "peak_source": peak_src,
                "avg_launch_us": avg_spmv_s * 1e6, "timed_launches": n_spmv,
                "sampling": "CUDA events around the first and the middle product of each 32-iteration chunk; "
                            "the middle one stands for the chunk's other products"}
    if n_cl and cl_iters:
        # the whole solve ran in one thread-block cluster: its roofline is the shared memory
        # of the cluster's SMs. Algorithmic shared-memory bytes per iteration: per stored
        # block (off-diagonal blocks in the difference form) 40 (nine values and the
        # column index) + 16 (the gathered u); per row 192 (the update: p, u, s, w, x, r and
        # the Jacobi inverse read, p, s, x, r, u written) + 100 (the product's own row: u,
        # p, s read, w written, and the 36-byte difference diagonal)
        stored = max(nnzb - V, 0)
        it_bytes = 56 * stored + 292 * V
        us_per_it = 1e3 * cl_ms / cl_iters
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2032.0
        smem_peak = SMEM_BYTES_PER_CLK * CLUSTER_SMS * mhz * 1e6 / 1e9
        ach = it_bytes / (us_per_it * 1e-6) / 1e9
        roofline = {"bound": "smem", "achieved": ach, "peak": smem_peak, "unit": "GB/s", "frac": ach / smem_peak,
                    "traffic": None,
                    "kernel": "cluster_pcg_kernel<true,false> (whole Chronopoulos-Gear PCG solve in one 16-CTA "
                              "cluster; unit: one iteration)",
                    "bytes_per_iteration": it_bytes,
                    "peak_source": f"derived: {SMEM_BYTES_PER_CLK} B/clk/SM x {CLUSTER_SMS} SMs x "
                                   f"{mhz:.0f} MHz (median SM clock under load)",
                    "us_per_iteration": us_per_it, "timed_launches": int(n_cl), "timed_iterations": int(cl_iters)}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e and proximity:
        # host state in pinned memory; per step: state to the device, query, step, state back
        xh = torch.from_numpy(wl.x0.copy()).pin_memory()
        vh = torch.from_numpy(wl.v0.copy()).pin_memory()
        cl_e = pc.Cloth(wl)

        def e2e_step():
            cl_e.x.copy_(xh, non_blocking=True)
            cl_e.v.copy_(vh, non_blocking=True)
            pd, wd = cl_e.proximity()
            cl_e.step(pd, wd, tol=args.tol, precision=prec, warm_start=pc.PC_WARM_PREV, max_iter=args.max_iter,
                      precond=precond, storage=storage, fuse=not args.no_fuse, schedule=schedule,
                      allow_not_converged=True)
            xh.copy_(cl_e.x)
            vh.copy_(cl_e.v)

        for k in range(args.warmup):
            e2e_step()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.warmup, nsteps):
            e2e_step()
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": aggregate_steps_per_s(world, args.steps, te), "unit": "steps/s",
               "h2d_bytes_per_step": 24 * V, "d2h_bytes_per_step": 24 * V}
        cl_e.close()
    elif not args.no_e2e:
        xh = torch.from_numpy(wl.x0.copy()).pin_memory().numpy()
        vh = torch.from_numpy(wl.v0.copy()).pin_memory().numpy()
        host_contacts = [wl.contacts(k % max(wl.steps, 1)) for k in range(nsteps)]
        host_contacts = [(torch.from_numpy(p).pin_memory().numpy(), torch.from_numpy(w).pin_memory().numpy())
                         for p, w in host_contacts]
        cl_e = pc.Cloth(wl)
        o = pc.pc_step_opts()
        o.h = wl.h
        o.solve = pc.solve_opts(tol=args.tol, precision=prec, max_iter=args.max_iter, precond=precond,
                                storage=storage, fuse=not args.no_fuse, schedule=schedule)
        o.warm_start = pc.PC_WARM_PREV
        for k in range(args.warmup):
            pc.pc_step_host(cl_e.ctx, xh, vh, host_contacts[k][0], host_contacts[k][1], o, allow_not_converged=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.warmup, nsteps):
            pc.pc_step_host(cl_e.ctx, xh, vh, host_contacts[k][0], host_contacts[k][1], o, allow_not_converged=True)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        P = wl.n_contacts
        e2e = {"value": aggregate_steps_per_s(world, args.steps, te), "unit": "steps/s",
               "h2d_bytes_per_step": 24 * V + 28 * P,
               "d2h_bytes_per_step": 24 * V}
        cl_e.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.tol)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "V": V, "T": wl.T, "H": cl.H, "nnzb": int(nnzb), "storage": args.storage, "fused_update": not args.no_fuse, "schedule": args.schedule,
                       "contacts_per_step": (float(np.mean(n_pairs[-args.steps:])) if proximity else wl.n_contacts),
                       "contact_model": (f"one-sided thickness {wl.material.contact_thickness * 1e3:.2f} mm, "
                                         "pairs from the GPU proximity query each step") if proximity
                       else "hold penalty, seeded random pairs",
                       "query_ms_per_step": (1e3 * float(np.mean(query_s[-args.steps:])) if proximity else None),
                       "precision": args.precision, "tol": args.tol,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": (f"inputs larger than L2 (about {spmv_bytes / 1e6:.0f} MB per SpMV)" if not n_cl else
                              f"the system ({spmv_bytes / 1e6:.1f} MB) fits L2; the solve runs from the shared "
                              "memory of one cluster, filled from global memory at each solve's start"),
                       "pcg_iters_per_step": float(np.mean(iters)), "max_rel_res": float(np.max(rels)),
                       "assembly_ms_per_step": asm_ms / max(n_asm, 1),
                       "rayleigh_damping": [wl.material.damp_mass, wl.material.damp_stiff]},
            "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    cl.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- other forms


def _setup_single():
    import torch
    torch.cuda.set_device(0)
    from paper_2008_00409_gb300 import build as cuda_build
    cuda_build.build()
    from paper_2008_00409_gb300 import pcloth as pc
    return torch, pc


def run_batched(args):
    """Batched form: every step advances all garments (pc_step_batched)."""
    torch, pc = _setup_single()
    from paper_2008_00409_gb300 import workloads as wk
    u = wk.garment_batch_union(args.garments)
    cl = pc.Cloth(u)
    o = pc.pc_step_opts()
    o.h = u.h
    o.solve = pc.solve_opts(tol=args.tol, max_iter=args.max_iter)
    o.warm_start = pc.PC_WARM_PREV
    nsteps = args.warmup + args.steps
    contacts = [cl.contacts_device(k) for k in range(nsteps)]
    for k in range(args.warmup):
        pc.pc_step_batched(cl.ctx, cl.x, cl.v, *contacts[k], u.inst_rows, o, allow_not_converged=True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = pc.pc_launch_count(cl.ctx)
    its, rels = [], []
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for k in range(args.warmup, nsteps):
            infos, _ = pc.pc_step_batched(cl.ctx, cl.x, cl.v, *contacts[k], u.inst_rows, o, allow_not_converged=True)
            its.append([i.iters for i in infos])
            rels.append(max(i.rel_res for i in infos))
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = pc.pc_launch_count(cl.ctx) - launches0
    grid, order, width, grid_sizes, tune_ms = pc.pc_batched_config(cl.ctx)
    its = np.array(its)
    seq = None
    if not args.no_sequential:
        parts = [pc.Cloth(p) for p in u.parts]
        pcont = [[pp.contacts_device(k) for k in range(3)] for pp in parts]
        for pp, cc in zip(parts, pcont):
            pp.step(*cc[0], tol=args.tol, precision=pc.PC_PREC_MIXED, warm_start=pc.PC_WARM_PREV,
                    allow_not_converged=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in (1, 2):
            for pp, cc in zip(parts, pcont):
                pp.step(*cc[k], tol=args.tol, precision=pc.PC_PREC_MIXED, warm_start=pc.PC_WARM_PREV,
                        allow_not_converged=True)
        torch.cuda.synchronize()
        seq = 2 / (time.perf_counter() - t0)
        for pp in parts:
            pp.close()
    out = {"metric": f"batched steps/s: {len(u.parts)} garments ({u.T / 1e6:.2f}M tris), one persistent PCG launch "
                     "per step, 1e-6 per garment",
           "value": args.steps / elapsed, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": u.name, "garments": len(u.parts), "V": u.V, "T": u.T,
                      "contacts_per_step": u.n_contacts, "tol": args.tol,
                      "l2": f"matrix {len(u.tris) * 13 * 40 / 1e6 / 2:.0f} MB (L2 is 129 MB)",
                      "iters_per_garment_min": int(its.min()), "iters_per_garment_mean": float(its.mean()),
                      "iters_per_garment_max": int(its.max()), "max_rel_res": float(max(rels)),
                      "autotuned_grid_ctas": grid, "autotuned_spmv_order": ["strided", "chunked"][order],
                      "autotuned_stage_blocks_per_row": width, "autotune_grids": grid_sizes,
                      "autotune_ms": {f"{w_} blocks/row {o_}": tune_ms[w_][i_] for w_ in (14, 18)
                                      for i_, o_ in enumerate(("strided", "chunked"))}},
           "sequential_steps_per_s": seq, "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_warmstart(args):
    """Learned warm start: train, then compare initial guesses on the 708 x 708 cloth."""
    torch, pc = _setup_single()
    from paper_2008_00409_gb300 import warmstart as ws
    from paper_2008_00409_gb300 import workloads as wk
    t0 = time.perf_counter()
    feat, dv = ws.collect(wk.warm_start_training(), tol=args.tol)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, stats, losses = ws.train(feat, dv, steps=args.train_steps, batch=65536, lr=1e-3, seed=0,
                                     log_every=max(1, args.train_steps // 4))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    rows = int(feat.shape[0])
    del feat, dv
    wl = wk.warm_start_eval()
    nsteps = args.warmup + args.steps
    with ClockSampler(0) as clk:
        res = ws.evaluate(wl, params, stats, steps=nsteps, tol=args.tol)
        fp32 = ws.evaluate(wl, params, stats, steps=nsteps, tol=args.tol, precision=pc.PC_PREC_FP32,
                           modes=(pc.PC_WARM_ZERO,))[pc.PC_WARM_ZERO]
    names = {pc.PC_WARM_ZERO: "zero", pc.PC_WARM_PREV: "prev", pc.PC_WARM_MLP: "mlp"}

    def summary(rec):
        w = slice(args.warmup, nsteps)
        return {"steps_per_s": len(rec["sec"][w]) / sum(rec["sec"][w]), "iters_mean": float(np.mean(rec["iters"][w])),
                "max_rel_res": float(np.max(rec["rel_res"][w]))}

    modes = {names[m]: summary(r) for m, r in res.items()}
    mlp = res[pc.PC_WARM_MLP]
    modes["mlp"]["guess_used"] = [int(g) for g in mlp["guess"][args.warmup:]]
    modes["mlp"]["guess_coef"] = [list(c) for c in mlp["guess_coef"][args.warmup:]]
    # CG energies of the guesses per timed step: zero (0), previous, learned, and the one used
    modes["mlp"]["energies"] = [list(e[1:]) + [u] for e, u in zip(mlp["guess_energy"][args.warmup:],
                                                                  mlp["combo_energy"][args.warmup:])]
    modes["fp32_zero"] = summary(fp32)
    out = {"metric": "steps/s at 1M tris (708^2 cloth, 2% contacts) to 1e-6 with the learned warm start",
           "value": modes["mlp"]["steps_per_s"], "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 / modes["mlp"]["steps_per_s"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
           "config": {"workload": wl.name, "V": wl.V, "T": wl.T, "contacts_per_step": wl.n_contacts, "tol": args.tol,
                      "precision": "mixed", "train_rows": rows, "train_steps": args.train_steps,
                      "train_batch": 65536, "data_seconds": t_gen, "train_seconds": t_train,
                      "loss_curve": losses},
           "modes": modes, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "batched":
        run_batched(args)
    elif args.form == "warmstart":
        run_warmstart(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
