"""Shared helpers for the GPU parity tests (no test functions here)."""
from __future__ import annotations

import numpy as np

from paper_2008_00409_gb300 import workloads as wk

# Tolerances. Values: per block |A_gpu - A_ref|_F <= 1e-5 |A_ref|_F + 1e-7 |A_ref,ii|_F
# (the floor, relative to the row's diagonal block, covers zero and cancelling blocks).
# dv: relative L2 error 1e-5 against the oracle solved to 1e-12.
BLOCK_RTOL = 1e-5
BLOCK_FLOOR = 1e-7
DV_RTOL = 1e-5


def block_errors(rp, ci, vals_gpu, vals_ref):
    """Per-block excess over the tolerance (<= 0 means within)."""
    vg = np.asarray(vals_gpu, np.float64).reshape(-1, 3, 3)
    vr = np.asarray(vals_ref, np.float64).reshape(-1, 3, 3)
    V = len(rp) - 1
    rows = np.repeat(np.arange(V), np.diff(rp))
    diag_slot = np.zeros(V, np.int64)
    is_diag = ci == rows
    diag_slot[rows[is_diag]] = np.nonzero(is_diag)[0]
    dnorm = np.linalg.norm(vr[diag_slot].reshape(V, 9), axis=1)
    err = np.linalg.norm((vg - vr).reshape(-1, 9), axis=1)
    ref = np.linalg.norm(vr.reshape(-1, 9), axis=1)
    return err - (BLOCK_RTOL * ref + BLOCK_FLOOR * dnorm[rows])


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def small_contact_cloth(nx=37, ny=29, frac=0.05, seed=11, flip=0.1, jitter=0.2, z_jitter=1e-4):
    """Ragged jittered grid with edge flips, two pins and per-step random contacts."""
    rest, tris, flipm = wk.grid_piece(nx, ny, 1.0 * (nx - 1) / 63, 1.0 * (ny - 1) / 63, jitter=jitter,
                                      flip_prob=flip, seed=seed)
    rest, tris, sheets = wk._assemble_pieces([(nx, ny, rest, tris, flipm)])
    x0 = rest.astype(np.float64).copy()
    x0[:, 2] += z_jitter * wk.normal(seed, 1, rest.shape[0])
    return wk.Workload(f"ragged{nx}x{ny}", rest, tris, wk._corner_pins(sheets), x0.astype(np.float32),
                       np.zeros_like(rest), 1.0 / 200.0, wk.Material(), sheets, seed, contact_kind="grid",
                       contact_frac=frac, contact_radius=4)


def small_stack(n=21, layers=3, seed=5):
    return wk.stacked_sheets(n, layers, seed=seed, contact_frac=0.05, steps=3, name=f"stack{layers}x{n}")
