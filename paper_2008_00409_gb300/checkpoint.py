"""Checkpoint and resume of an integrator run, and a per-step metrics log.

A checkpoint holds what the next step depends on: positions, velocities, the previous
step's dv (the PC_WARM_PREV guess and an input of the learned guess), the step index
(contact sets and other seeded inputs are generated from (seed, step), so they are
reproduced, not stored) and, when training, the network's parameters, statistics and
Adam state. Resuming from it gives the same steps, bit for bit, as running on.
"""
import json
import os
import time

import numpy as np
import torch

from . import pcloth as pc

FORMAT = 1


def save(path, cloth, step: int, mlp=None, params=None, stats=None):
    """Write the state of `cloth` (a pcloth.Cloth) after `step` steps to an .npz file;
    `mlp` (a pc_mlp handle), `params` and `stats` (device tensors) are optional."""
    V = cloth.V
    dv = torch.zeros(V * 3, dtype=torch.float32, device=cloth.device)
    has_prev = pc.pc_get_prev_dv(cloth.ctx, dv)
    out = {
        "format": np.int64(FORMAT),
        "workload": np.array(cloth.wl.name),
        "V": np.int64(V),
        "T": np.int64(cloth.T),
        "step": np.int64(step),
        "x": cloth.x.detach().cpu().numpy(),
        "v": cloth.v.detach().cpu().numpy(),
        "dv_prev": dv.cpu().numpy().reshape(V, 3),
        "has_prev": np.int64(has_prev),
    }
    if params is not None:
        out["mlp_params"] = params.detach().cpu().numpy()
    if stats is not None:
        out["mlp_stats"] = stats.detach().cpu().numpy()
    if mlp is not None:
        m1 = torch.zeros(pc.PC_MLP_NPARAMS, dtype=torch.float32, device=cloth.device)
        m2 = torch.zeros_like(m1)
        out["adam_t"] = np.int64(pc.pc_mlp_get_state(mlp, m1, m2))
        out["adam_m"] = m1.cpu().numpy()
        out["adam_v"] = m2.cpu().numpy()
    tmp = str(path) + ".tmp.npz"
    np.savez(tmp, **out)
    os.replace(tmp, path)


def load(path, cloth, mlp=None):
    """Restore a checkpoint into `cloth` (created for the same workload) and, when given,
    the Adam state into `mlp`. Returns (step, params, stats); the last two are device
    tensors or None."""
    with np.load(path, allow_pickle=False) as f:
        if int(f["format"]) != FORMAT:
            raise ValueError(f"unknown checkpoint format {int(f['format'])}")
        if int(f["V"]) != cloth.V or int(f["T"]) != cloth.T:
            raise ValueError("checkpoint is for another mesh")
        cloth.x.copy_(torch.from_numpy(f["x"]))
        cloth.v.copy_(torch.from_numpy(f["v"]))
        if int(f["has_prev"]):
            pc.pc_set_prev_dv(cloth.ctx, torch.from_numpy(f["dv_prev"].reshape(-1)).to(cloth.device))
        else:
            pc.pc_set_prev_dv(cloth.ctx, None)
        params = torch.from_numpy(f["mlp_params"]).to(cloth.device) if "mlp_params" in f else None
        stats = torch.from_numpy(f["mlp_stats"]).to(cloth.device) if "mlp_stats" in f else None
        if mlp is not None and "adam_m" in f:
            pc.pc_mlp_set_state(mlp, torch.from_numpy(f["adam_m"]).to(cloth.device),
                                torch.from_numpy(f["adam_v"]).to(cloth.device), int(f["adam_t"]))
        return int(f["step"]), params, stats


class StepLog:
    """Appends one JSON line per step: nnzb, PCG iterations, outer refinements, FP64
    relative residual, the guess the step started from, wall time, and (when the
    context's profiling is on) assembly ms and, since the previous line, SpMV GB/s of the
    grid schedule or microseconds per iteration of the cluster schedule (whichever ran)."""

    def __init__(self, path, cloth):
        self.path = path
        self.cloth = cloth
        self.t = time.perf_counter()
        self.asm = pc.pc_assembly_stats(cloth.ctx)
        self.spmv = pc.pc_spmv_stats(cloth.ctx)
        self.cluster = pc.pc_cluster_stats(cloth.ctx)

    def record(self, step: int, info, status: int):
        now = time.perf_counter()
        asm = pc.pc_assembly_stats(self.cloth.ctx)
        spmv = pc.pc_spmv_stats(self.cloth.ctx)
        cluster = pc.pc_cluster_stats(self.cloth.ctx)
        line = {"step": step, "status": int(status), "nnzb": int(info.nnzb), "iters": int(info.solve.iters),
                "outer": int(info.solve.outer), "rel_res": float(info.solve.rel_res), "guess": int(info.guess),
                "wall_ms": 1e3 * (now - self.t)}
        if asm[0] > 0:
            line["assembly_ms"] = asm[1] / asm[0]
        if spmv[0] > 0 and spmv[1] > 0:
            V = self.cloth.V
            nbytes = 40 * spmv[2] + 4 * (V + 1) + 36 * V + 32 * V
            line["spmv_us"] = 1e3 * spmv[1] / spmv[0]
            line["spmv_gbs"] = nbytes / (spmv[1] / spmv[0] / 1e3) / 1e9
        if cluster[0] > 0 and cluster[1] > 0:
            line["cluster_us_per_iter"] = 1e3 * cluster[2] / cluster[1]
        with open(self.path, "a") as fh:
            fh.write(json.dumps(line) + "\n")
        self.t = now
        return line
