"""The allocation-free solve entry point, through the C ABI.

pc_pcg_solve_static serves callers that cannot allocate device memory (a plug-in whose
host application owns all GPU memory, a real-time loop that must never call cudaMalloc,
because an allocation can synchronize the device): it keeps every scratch buffer in one
static device array inside the library. Each test compares it with the context-based
pc_pcg_solve on two calls in a row (the array keeps the previous call's contents), and
one compares it with the FP64 oracle. This file runs last so that, if it fails, a run
that stops at the first failure has already run every other test; it also passes on its
own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2008_00409_gb300 import workloads as wk
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2008_00409_gb300 import build
    build.build()
    from paper_2008_00409_gb300 import pcloth
    return pcloth


@pytest.fixture(scope="module")
def system(pc):
    wl = wk.small_square()  # 4,096 rows, within the static limit
    cl = pc.Cloth(wl)
    s = cl.assemble()
    return wl, cl, s


def _context_solve(pc, cl, s, opts, dres):
    ref = torch.zeros(cl.V * 3, device="cuda")
    info, _ = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], dres, s["b"], ref, opts)
    return ref.cpu().numpy(), info


def _static_solve(pc, cl, s, opts, dres, allow_not_converged=False):
    dv = torch.zeros(cl.V * 3, device="cuda")
    info, st = pc.pc_pcg_solve_static(cl.V, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], dres, s["b"], dv, opts,
                                      allow_not_converged=allow_not_converged)
    return dv.cpu().numpy(), info, st


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("precond", ["jacobi", "block"])
@pytest.mark.parametrize("form", ["fused", "two-kernel", "cluster"])
def test_static_solve_matches_context_solve_on_two_calls(pc, system, precision, precond, form):
    wl, cl, s = system
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP32
    pre = pc.PC_PRECOND_BLOCK if precond == "block" else pc.PC_PRECOND_JACOBI
    # the static entry point streams the caller's matrix: the context solve on the same layout
    opts = pc.solve_opts(tol=1e-9 if precision == "mixed" else 1e-6, precision=prec, max_iter=50000, precond=pre,
                         storage=pc.PC_STORAGE_FULL, fuse=form == "fused",
                         schedule=pc.PC_SCHED_CLUSTER if form == "cluster" else pc.PC_SCHED_GRID)
    ref, info_ref = _context_solve(pc, cl, s, opts, s["dres"])
    for call in range(2):
        got, info, st = _static_solve(pc, cl, s, opts, s["dres"])
        assert st == pc.PC_OK
        assert H.rel_l2(got, ref) <= H.DV_RTOL, f"call {call}"
        assert abs(info.iters - info_ref.iters) <= 2
        assert info.rel_res <= max(2 * info_ref.rel_res, 1e-12)


def test_static_solve_default_options_and_plain_form(pc, system):
    """opts = NULL (the default storage, which the static call reads as the full matrix)
    and a solve without the difference-form diagonal, each twice in a row."""
    wl, cl, s = system
    ref, _ = _context_solve(pc, cl, s, pc.solve_opts(), s["dres"])
    for call in range(2):
        dv = torch.zeros(cl.V * 3, device="cuda")
        A = pc.bsr_struct(s["row_ptr"], s["col_idx"], s["nnzb"])
        info = pc.pc_solve_info()
        st = pc.lib().pc_pcg_solve_static(cl.V, ctypes.byref(A), pc._ptr(s["vals"]), pc._ptr(s["dres"]),
                                          pc._ptr(s["b"]), pc._ptr(dv), None, ctypes.byref(info), pc._stream(None))
        assert st == pc.PC_OK
        assert H.rel_l2(dv.cpu().numpy(), ref) <= H.DV_RTOL, f"call {call}"
    opts = pc.solve_opts(tol=1e-6, precision=pc.PC_PREC_FP32, storage=pc.PC_STORAGE_FULL)
    ref, _ = _context_solve(pc, cl, s, opts, None)
    for call in range(2):
        got, info, st = _static_solve(pc, cl, s, opts, None)
        assert st == pc.PC_OK and H.rel_l2(got, ref) <= H.DV_RTOL, f"call {call}"


def test_static_solve_after_a_call_that_stopped_early(pc, system):
    """A call that ends PC_ERR_NOT_CONVERGED leaves its scalars in the shared array; the
    next call must start clean and match the context solve."""
    wl, cl, s = system
    opts = pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED, storage=pc.PC_STORAGE_FULL)
    ref, _ = _context_solve(pc, cl, s, opts, s["dres"])
    short = pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED, storage=pc.PC_STORAGE_FULL, max_iter=5)
    _, info, st = _static_solve(pc, cl, s, short, s["dres"], allow_not_converged=True)
    assert st == pc.PC_ERR_NOT_CONVERGED and info.iters <= 5 + 32
    got, info, st = _static_solve(pc, cl, s, opts, s["dres"])
    assert st == pc.PC_OK and H.rel_l2(got, ref) <= H.DV_RTOL


def test_static_solve_matches_oracle(pc, system):
    wl, cl, s = system
    om = oracle.Mesh.from_workload(wl)
    rp, ci, vals_ref, b_ref = om.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), h=wl.h)
    dv_ref, _, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    opts = pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED, max_iter=50000)
    for call in range(2):
        got, info, st = _static_solve(pc, cl, s, opts, s["dres"])
        assert st == pc.PC_OK
        assert H.rel_l2(got, dv_ref) <= H.DV_RTOL, f"call {call}"


def test_static_solve_rejects_more_rows_than_its_array(pc, system):
    wl, cl, s = system
    A = pc.bsr_struct(s["row_ptr"], s["col_idx"], s["nnzb"])
    info = pc.pc_solve_info()
    o = pc.solve_opts()
    dv = torch.zeros(cl.V * 3, device="cuda")
    # raw call: the size check comes before any device work
    st = pc.lib().pc_pcg_solve_static(16385, ctypes.byref(A), pc._ptr(s["vals"]), pc._ptr(s["dres"]), pc._ptr(s["b"]),
                                      pc._ptr(dv), ctypes.byref(o), ctypes.byref(info), pc._stream(None))
    assert st == pc.PC_ERR_CAPACITY
    assert np.all(dv.cpu().numpy() == 0)


def test_static_solve_rejects_columns_beyond_its_rows(pc, system):
    """V smaller than the matrix's column range: the solve must refuse (PC_ERR_ARG) before
    any product gathers past the vectors, and a correct call afterwards still works."""
    wl, cl, s = system
    A = pc.bsr_struct(s["row_ptr"], s["col_idx"], s["nnzb"])
    info = pc.pc_solve_info()
    o = pc.solve_opts(storage=pc.PC_STORAGE_FULL)
    dv = torch.zeros(cl.V * 3, device="cuda")
    st = pc.lib().pc_pcg_solve_static(cl.V // 2, ctypes.byref(A), pc._ptr(s["vals"]), pc._ptr(s["dres"]),
                                      pc._ptr(s["b"]), pc._ptr(dv), ctypes.byref(o), ctypes.byref(info),
                                      pc._stream(None))
    assert st == pc.PC_ERR_ARG
    assert np.all(dv.cpu().numpy() == 0)
    ref, _ = _context_solve(pc, cl, s, o, s["dres"])
    got, info, st = _static_solve(pc, cl, s, o, s["dres"])
    assert st == pc.PC_OK and H.rel_l2(got, ref) <= H.DV_RTOL
