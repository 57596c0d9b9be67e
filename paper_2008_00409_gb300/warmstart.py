"""Learned warm start: training data from the integrator, training, and evaluation.

Buffer management and calls into the library only (pc_step, pc_mlp_*): every arithmetic
step -- the time steps that generate the data, the features, the statistics, the
forward and backward passes, Adam, and the choice of the initial guess -- runs in the
CUDA library.

Training rows are (features, dv) pairs that pc_step itself writes for each vertex of
each step (feat_out, dv_out); the network learns dv - dv_prev.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import pcloth as pc

N_IN, N_HID, N_OUT = pc.PC_MLP_IN, pc.PC_MLP_HIDDEN, pc.PC_MLP_OUT


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-uniform weights and zero biases, flat float32 in the library's layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((N_HID, N_IN), (N_HID, N_HID), (N_OUT, N_HID)):
        bound = np.sqrt(6.0 / fan_in)
        parts += [rng.uniform(-bound, bound, size=fan_out * fan_in), np.zeros(fan_out)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == pc.PC_MLP_NPARAMS
    return torch.from_numpy(p).to(device)


def collect(workloads, steps: int | None = None, tol: float = 1e-6, precision: int = pc.PC_PREC_MIXED,
            device="cuda"):
    """Run each workload for `steps` steps (previous-step guess) and keep every vertex's
    features and solution. Returns (feat float[N][12], dv float[N][3]) on the device."""
    counts = [wl.V * (steps if steps is not None else wl.steps) for wl in workloads]
    total = int(sum(counts))
    feat = torch.empty(total, N_IN, device=device)
    dv = torch.empty(total, 3, device=device)
    off = 0
    for wl in workloads:
        n_steps = steps if steps is not None else wl.steps
        cl = pc.Cloth(wl, device=device)
        for t in range(n_steps):
            pairs, w = cl.contacts_device(t)
            cl.step(pairs, w, tol=tol, precision=precision, warm_start=pc.PC_WARM_PREV,
                    dv_out=dv[off:off + wl.V], feat_out=feat[off:off + wl.V], allow_not_converged=True)
            off += wl.V
        cl.close()
    assert off == total
    return feat, dv


def train(feat: torch.Tensor, dv: torch.Tensor, steps: int = 2000, batch: int = 65536, lr: float = 1e-3,
          seed: int = 0, log_every: int = 0):
    """Adam on random mini-batches (with replacement). Returns (params, stats, losses)."""
    n = int(feat.shape[0])
    dev = feat.device
    m = pc.pc_mlp_create()
    try:
        stats = torch.empty(pc.PC_MLP_NSTATS, device=dev)
        pc.pc_mlp_stats(m, n, feat, dv, stats)
        params = init_params(seed, dev)
        rng = np.random.default_rng(seed + 1)
        idx = torch.from_numpy(rng.integers(0, n, size=(steps, batch), dtype=np.int64).astype(np.int32)).to(dev)
        opts = pc.adam_opts(lr)
        losses = []
        for s in range(steps):
            want = log_every > 0 and (s % log_every == 0 or s == steps - 1)
            loss = pc.pc_mlp_train_step(m, batch, idx[s], params, stats, feat, dv, opts, with_loss=want)
            if want:
                losses.append((s, loss))
        torch.cuda.synchronize(dev)
    finally:
        pc.pc_mlp_destroy(m)
    return params, stats, losses


def dataset_loss(params, stats, feat, dv) -> float:
    """Loss of the network over a whole dataset (no update)."""
    m = pc.pc_mlp_create()
    try:
        grad = torch.empty(pc.PC_MLP_NPARAMS, device=feat.device)
        return pc.pc_mlp_grad(m, int(feat.shape[0]), None, params, stats, feat, dv, grad)
    finally:
        pc.pc_mlp_destroy(m)


def evaluate(wl, params, stats, steps: int, tol: float = 1e-6, precision: int = pc.PC_PREC_MIXED,
             modes=(pc.PC_WARM_ZERO, pc.PC_WARM_PREV, pc.PC_WARM_MLP), device="cuda"):
    """Run the same trajectory once per warm-start mode. Per mode: PCG iterations, the
    guess used and the guesses' relative residuals per step, and seconds per step."""
    out = {}
    contacts = None
    for mode in modes:
        cl = pc.Cloth(wl, device=device)
        if contacts is None:
            contacts = [cl.contacts_device(t) for t in range(steps)]
        if mode == pc.PC_WARM_MLP:
            pc.pc_set_warm_mlp(cl.ctx, params, stats)
        rec = {"iters": [], "guess": [], "guess_res": [], "guess_energy": [], "guess_coef": [], "combo_energy": [],
               "rel_res": [], "sec": []}
        for t in range(steps):
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            info, _ = cl.step(*contacts[t], tol=tol, precision=precision, warm_start=mode, allow_not_converged=True)
            torch.cuda.synchronize(device)
            rec["sec"].append(time.perf_counter() - t0)
            rec["iters"].append(info.solve.iters)
            rec["rel_res"].append(info.solve.rel_res)
            rec["guess"].append(info.guess)
            rec["guess_res"].append(list(info.guess_res))
            rec["guess_energy"].append(list(info.guess_energy))
            rec["guess_coef"].append(list(info.guess_coef))
            rec["combo_energy"].append(info.combo_energy)
        if mode == pc.PC_WARM_MLP:
            pc.pc_set_warm_mlp(cl.ctx, None, None)
        cl.close()
        out[mode] = rec
    return out
