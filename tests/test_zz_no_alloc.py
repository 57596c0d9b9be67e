"""The allocation-free solve entry point, through the C ABI.

pc_pcg_solve_static serves callers that cannot allocate device memory (a plug-in whose
host application owns all GPU memory, a real-time loop that must never call cudaMalloc):
it keeps every scratch buffer in one static device array inside the library. This file
runs last so that, if it fails, a run that stops at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2008_00409_gb300 import workloads as wk
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2008_00409_gb300 import build
    build.build()
    from paper_2008_00409_gb300 import pcloth
    return pcloth


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_static_solve_matches_context_solve_on_two_calls(pc, precision):
    wl = wk.small_square()  # 4,096 rows, within the static limit
    cl = pc.Cloth(wl)
    s = cl.assemble()
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP32
    # the static entry point reads the full matrix; compare with the context solve on the same layout
    opts = pc.solve_opts(tol=1e-9 if precision == "mixed" else 1e-6, precision=prec, max_iter=50000,
                         storage=pc.PC_STORAGE_FULL)
    ref = torch.zeros(cl.V * 3, device="cuda")
    info_ref, _ = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], ref,
                                  opts)
    ref_np = ref.cpu().numpy()
    for call in range(2):
        dv = torch.zeros(cl.V * 3, device="cuda")
        info, st = pc.pc_pcg_solve_static(cl.V, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"],
                                          s["b"], dv, opts)
        assert st == pc.PC_OK
        got = dv.cpu().numpy()
        assert H.rel_l2(got, ref_np) <= H.DV_RTOL, f"call {call}"
        assert abs(info.iters - info_ref.iters) <= 2
        assert info.rel_res <= max(2 * info_ref.rel_res, 1e-12)


def test_static_solve_rejects_more_rows_than_its_array(pc):
    wl = wk.small_square()
    cl = pc.Cloth(wl)
    s = cl.assemble()
    too_many = pc.lib().pc_pcg_solve_static  # raw call: the size check comes before any device work
    from paper_2008_00409_gb300.pcloth import bsr_struct, pc_solve_info, solve_opts, _ptr, _stream
    import ctypes
    A = bsr_struct(s["row_ptr"], s["col_idx"], s["nnzb"])
    info = pc_solve_info()
    o = solve_opts()
    dv = torch.zeros(cl.V * 3, device="cuda")
    st = too_many(16385, ctypes.byref(A), _ptr(s["vals"]), _ptr(s["dres"]), _ptr(s["b"]), _ptr(dv), ctypes.byref(o),
                  ctypes.byref(info), _stream(None))
    assert st == pc.PC_ERR_CAPACITY
    assert np.all(dv.cpu().numpy() == 0)
