"""The row-partitioned solve (Sec. 3.1, Eq. 4-5) through the C ABI: two and three ranks
(processes) on one GPU, exchanging the halo and the scalars through gloo on the host (so
no kernel ever waits on another process's kernels). Every rank's rows of dv are compared
with the single-GPU solve of the whole system and with the FP64 oracle."""
import datetime
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2008_00409_gb300 import build
    build.build()
    from paper_2008_00409_gb300 import dist as ds
    from paper_2008_00409_gb300 import pcloth as pc
    from paper_2008_00409_gb300 import workloads as wk
    from tests import _helpers as H

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=300))
    wl = H.small_contact_cloth() if case == "contacts" else wk.small_square()
    cl = pc.Cloth(wl)
    pairs, w = wl.contacts(1)
    pd, wd = cl.contacts_device(1)
    s = cl.assemble(pd, wd)
    nnzb = s["nnzb"]
    rp = s["row_ptr"].cpu().numpy()
    rs = ds.partition(wl.V, world, rp)
    r0, r1 = int(rs[rank]), int(rs[rank + 1])
    comm = ds.HostComm()
    solver = ds.DistSolver(comm, rs, max_blocks=nnzb)
    solver.plan(s["row_ptr"], s["col_idx"], nnzb)
    sizes = solver.sizes()
    om = oracle.Mesh.from_workload(wl)
    rpo, cio, vals_ref, b_ref = om.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), pairs, w, wl.h)
    dv_ref, _, _ = oracle.pcg(rpo, cio, vals_ref, b_ref, tol=1e-12)
    res = {"sizes": sizes, "rows": (r0, r1)}
    b_rows = s["b"].view(-1, 3)[r0:r1]
    for label, prec, tol, diff in (("mixed", pc.PC_PREC_MIXED, 1e-9, True), ("fp32", pc.PC_PREC_FP32, 1e-6, True),
                                   ("mixed-plain", pc.PC_PREC_MIXED, 1e-9, False)):
        dres = s["dres"] if diff else None
        opts = pc.solve_opts(tol=tol, precision=prec, max_iter=50000, storage=pc.PC_STORAGE_FULL)
        dv_rows = torch.zeros(r1 - r0, 3, device="cuda")
        info, st = solver.solve(s["vals"], dres.view(-1, 9)[r0:r1] if diff else None, b_rows, dv_rows, opts)
        single = torch.zeros(wl.V * 3, device="cuda")
        info1, _ = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"], dres, s["b"], single, opts)
        # the two-kernel form takes its direction step the way the partitioned solve does
        opts2 = pc.solve_opts(tol=tol, precision=prec, max_iter=50000, storage=pc.PC_STORAGE_FULL, fuse=False)
        info2, _ = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"], dres, s["b"],
                                   torch.zeros(wl.V * 3, device="cuda"), opts2)
        got = dv_rows.cpu().numpy().astype(np.float64)
        res[label] = {
            "iters": info.iters, "iters_single": info1.iters, "iters_two_kernel": info2.iters, "rel_res": info.rel_res,
            "err_single": H.rel_l2(got, single.view(-1, 3)[r0:r1].cpu().numpy()),
            "err_oracle": H.rel_l2(got, dv_ref[r0:r1]), "pins_zero": bool(np.all(got[np.isin(np.arange(r0, r1),
                                                                                             wl.pins)] == 0.0)),
        }
    res["calls"] = dict(comm.calls)
    out[rank] = res
    solver.close()
    cl.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", ["contacts", "square64"])
def test_row_partitioned_solve_matches_single_gpu_and_oracle(world, case):
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), case, out), nprocs=world, join=True)
    for r in range(world):
        res = out[r]
        print(r, res)
        # every rank exchanges a halo (the partition cuts the mesh)
        assert res["sizes"]["n_halo"] > 0 and res["sizes"]["n_send"] > 0
        for label in ("mixed", "fp32", "mixed-plain"):
            rec = res[label]
            # the same global scalars on every rank: the same iteration count
            assert rec["iters"] == out[0][label]["iters"]
            # the partitioned solve needs no more iterations than the single-GPU one
            assert rec["iters"] <= 1.05 * rec["iters_two_kernel"] + 5, (label, rec)
            assert rec["err_single"] <= 1e-5, (label, rec)
            assert rec["pins_zero"]
            if label != "fp32":
                assert rec["rel_res"] <= 1e-9 * 1.01
            # the difference form reaches the oracle within 1e-5; the plain form stores the
            # diagonal blocks in FP32, whose rounding (6e-8 of the stiffness) is a visible
            # share of the mass term they contain, and FP32 PCG stops on its recurrence
            # residual: both are held to 1e-4, as in the single-GPU parity tests
            assert rec["err_oracle"] <= (1e-5 if label == "mixed" else 1e-4), (label, rec)
    # all ranks made the same collective calls
    assert len({tuple(sorted(out[r]["calls"].items())) for r in range(world)}) == 1
