"""Failure paths of the solvers on the GPU, made on the host (no fault, trap or hang):
a grid-barrier wait that runs out (a budget of one cycle), an indefinite system (a
positive diagonal but p.Ap < 0) and a non-finite garment inside a batch. Each must
come back as a status, leave the failed part's state untouched and keep the context
usable."""
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


def _np(t):
    return t.detach().cpu().numpy()


def small_batch():
    parts = [wk.garment(s, seed=91, stream=300 + 16 * k, contact_frac=0.03) for k, s in enumerate([9, 14, 11, 20])]
    return wk.batch_union(parts, name="batch4")


def _step_opts(pc, u, tol=1e-9):
    o = pc.pc_step_opts()
    o.h = u.h
    o.solve = pc.solve_opts(tol=tol, max_iter=50000)
    o.warm_start = pc.PC_WARM_ZERO
    return o


def test_barrier_timeout_is_reported_and_the_context_recovers(pc):
    u = small_batch()
    cl = pc.Cloth(u)
    s = cl.assemble(*cl.contacts_device(0))
    args = (cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"])
    opts = pc.solve_opts(tol=1e-9, max_iter=50000)
    ref = torch.zeros(cl.V * 3, device="cuda")
    pc.pc_pcg_solve_batched(*args, ref, u.inst_rows, opts)
    # one cycle: no wait at a grid barrier can succeed, the launch unwinds
    pc.pc_set_barrier_wait(cl.ctx, 1)
    dv = torch.full((cl.V * 3,), 0.25, device="cuda")
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve_batched(*args, dv, u.inst_rows, opts)
    assert e.value.status == pc.PC_ERR_TIMEOUT
    assert torch.all(dv == 0.25)  # no result written back
    # default budget again: the same schedule gives the identical solve
    pc.pc_set_barrier_wait(cl.ctx, 0)
    dv.zero_()
    infos, st = pc.pc_pcg_solve_batched(*args, dv, u.inst_rows, opts)
    assert st == pc.PC_OK and all(i.rel_res <= 2e-9 for i in infos)
    assert torch.equal(dv, ref)


def test_batched_step_timeout_leaves_the_state_and_recovers(pc):
    u = small_batch()
    cl = pc.Cloth(u)
    pd, wd = cl.contacts_device(0)
    x0, v0 = cl.x.clone(), cl.v.clone()
    # set before the first step: the autotuner's own runs time out too
    pc.pc_set_barrier_wait(cl.ctx, 1)
    with pytest.raises(pc.PcError) as e:
        pc.pc_step_batched(cl.ctx, cl.x, cl.v, pd, wd, u.inst_rows, _step_opts(pc, u))
    assert e.value.status == pc.PC_ERR_TIMEOUT
    assert torch.equal(cl.x, x0) and torch.equal(cl.v, v0)
    pc.pc_set_barrier_wait(cl.ctx, -5)  # <= 0: default
    infos, st = pc.pc_step_batched(cl.ctx, cl.x, cl.v, pd, wd, u.inst_rows, _step_opts(pc, u))
    assert st == pc.PC_OK and all(i.rel_res <= 2e-9 for i in infos)
    fresh = pc.Cloth(u)
    pc.pc_step_batched(fresh.ctx, fresh.x, fresh.v, pd, wd, u.inst_rows, _step_opts(pc, u))
    assert H.rel_l2(_np(cl.v - v0), _np(fresh.v - v0)) <= H.DV_RTOL


def _two_instance_matrix(V):
    """Rows [0, V/2): SPD (4 I on the diagonal, -I to the row neighbours). Rows [V/2, V):
    I on the diagonal and 2 I between rows i and i + V/4, so the pair matrix
    [[1, 2], [2, 1]] has eigenvalues 3 and -1; b = +1 on the first quarter and -1 on the
    second makes the first Jacobi direction p = b with p.Ap = -2 per pair and component."""
    h = V // 2
    q = h // 2
    rows = []
    for i in range(V):
        cols = {i: 4.0 if i < h else 1.0}
        if i < h:
            if i > 0:
                cols[i - 1] = -1.0
            if i + 1 < h:
                cols[i + 1] = -1.0
        else:
            k = i - h
            cols[h + (k + q) % h] = 2.0
        rows.append(sorted(cols.items()))
    rp = np.zeros(V + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    nnzb = int(rp[-1])
    cap = (nnzb + 3) // 4 * 4
    ci = np.zeros(cap, np.int32)
    vals = np.zeros((cap, 3, 3), np.float32)
    dense = np.zeros((3 * V, 3 * V))
    for i, r in enumerate(rows):
        for n, (j, a) in enumerate(r):
            ci[rp[i] + n] = j
            vals[rp[i] + n] = a * np.eye(3)
            dense[3 * i:3 * i + 3, 3 * j:3 * j + 3] = a * np.eye(3)
    rng = np.random.default_rng(5)
    b = np.zeros((V, 3))
    b[:h] = rng.normal(size=(h, 3))
    b[h:h + q] = 1.0
    b[h + q:] = -1.0
    return rp, ci, nnzb, vals, b.astype(np.float32), dense, h


def test_indefinite_system_is_reported_and_isolated(pc):
    wl = wk.garment(8, seed=91, stream=400)
    assert wl.V == 64
    cl = pc.Cloth(wl)
    rp, ci, nnzb, vals, b, dense, h = _two_instance_matrix(wl.V)
    t = [torch.from_numpy(a).cuda() for a in (rp, ci, vals.reshape(-1), b.reshape(-1))]
    opts = pc.solve_opts(tol=1e-10, max_iter=1000, precision=pc.PC_PREC_MIXED)
    # the single-system solver on the whole matrix, on both schedules
    dv = torch.zeros(wl.V * 3, device="cuda")
    for sched in (pc.PC_SCHED_GRID, pc.PC_SCHED_CLUSTER):
        with pytest.raises(pc.PcError) as e:
            pc.pc_pcg_solve(cl.ctx, t[0], t[1], nnzb, t[2], None, t[3], dv,
                            pc.solve_opts(tol=1e-10, max_iter=1000, precision=pc.PC_PREC_MIXED, schedule=sched))
        assert e.value.status == pc.PC_ERR_NONFINITE
    # batched: the indefinite instance stops, the SPD one converges to the exact solution
    dv.zero_()
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve_batched(cl.ctx, t[0], t[1], nnzb, t[2], None, t[3], dv, [0, h, wl.V], opts)
    assert e.value.status == pc.PC_ERR_NONFINITE
    want = np.linalg.solve(dense[:3 * h, :3 * h], b[:h].reshape(-1).astype(np.float64)).reshape(-1, 3)
    got = _np(dv).reshape(-1, 3)[:h].astype(np.float64)
    assert H.rel_l2(got, want) <= 1e-6


def test_nonfinite_garment_keeps_its_state_while_the_others_step(pc):
    u = small_batch()
    bad, good = pc.Cloth(u), pc.Cloth(u)
    pd, wd = bad.contacts_device(0)
    k = 2
    r0, r1 = int(u.inst_rows[k]), int(u.inst_rows[k + 1])
    bad.x[r0 + 5, 1] = float("nan")
    x0, v0 = bad.x.clone(), bad.v.clone()
    with pytest.raises(pc.PcError) as e:
        pc.pc_step_batched(bad.ctx, bad.x, bad.v, pd, wd, u.inst_rows, _step_opts(pc, u))
    assert e.value.status == pc.PC_ERR_NONFINITE
    pc.pc_step_batched(good.ctx, good.x, good.v, pd, wd, u.inst_rows, _step_opts(pc, u))
    # the failed garment did not move
    assert torch.equal(bad.v[r0:r1], v0[r0:r1])
    assert np.array_equal(_np(bad.x[r0:r1]), _np(x0[r0:r1]), equal_nan=True)
    # every other garment advanced as in the clean batch
    dv_bad = _np(bad.v - v0)
    dv_good = _np(good.v - v0)
    for j in range(len(u.parts)):
        if j == k:
            continue
        a, c = int(u.inst_rows[j]), int(u.inst_rows[j + 1])
        assert np.isfinite(dv_bad[a:c]).all()
        assert H.rel_l2(dv_bad[a:c], dv_good[a:c]) <= H.DV_RTOL, j


def test_fused_update_barrier_timeout_and_recovery(pc):
    """The single-system solve's fused update meets at a grid barrier once per iteration:
    with a one-cycle budget the solve reports PC_ERR_TIMEOUT, and with the default budget
    the same context gives the identical solve."""
    wl = H.small_contact_cloth()
    cl = pc.Cloth(wl)
    s = cl.assemble(*cl.contacts_device(0))
    args = (cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"])
    opts = pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED, max_iter=50000, schedule=pc.PC_SCHED_GRID)
    ref = torch.zeros(cl.V * 3, device="cuda")
    info_ref, _ = pc.pc_pcg_solve(*args, ref, opts)
    pc.pc_set_barrier_wait(cl.ctx, 1)
    dv = torch.zeros(cl.V * 3, device="cuda")
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve(*args, dv, opts)
    assert e.value.status == pc.PC_ERR_TIMEOUT
    pc.pc_set_barrier_wait(cl.ctx, 0)
    dv.zero_()
    info, st = pc.pc_pcg_solve(*args, dv, opts)
    assert st == pc.PC_OK and info.iters == info_ref.iters
    assert torch.equal(dv, ref)
