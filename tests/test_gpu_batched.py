"""Batched solver (one persistent PCG launch over many garments) against the oracle and
against per-garment solves, through the C ABI."""
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


def small_batch():
    sides = [8, 13, 21, 9, 30, 17]  # uneven sizes, each >= 32 rows
    parts = [wk.garment(s, seed=77, stream=100 + 16 * k, contact_frac=0.03) for k, s in enumerate(sides)]
    return wk.batch_union(parts, name="batch6")


def _np(t):
    return t.detach().cpu().numpy()


def test_batched_solve_matches_oracle_and_single_solves(pc):
    u = small_batch()
    cl = pc.Cloth(u)
    pd, wd = cl.contacts_device(0)
    pairs, w = u.contacts(0)
    s = cl.assemble(pd, wd)
    dv = torch.zeros(cl.V * 3, device="cuda")
    opts = pc.solve_opts(tol=1e-9, max_iter=50000)
    infos, st = pc.pc_pcg_solve_batched(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"],
                                        dv, u.inst_rows, opts)
    assert st == pc.PC_OK
    got = _np(dv).reshape(-1, 3)
    grid, order, width, sizes, ms = pc.pc_batched_config(cl.ctx)
    assert grid in sizes and order in (0, 1) and width in (14, 18)
    gi = sizes.index(grid)
    assert ms[width][order][gi] > 0
    # the autotuner timed both stage widths (tile shapes), both entry orders and several
    # grids, and kept the fastest candidate
    for w_ in (14, 18):
        assert all(sum(t > 0 for t in ms[w_][o]) >= 2 for o in (0, 1)), w_
    tried = [t for w_ in (14, 18) for row in ms[w_] for t in row if t > 0]
    assert len(tried) >= 8 and ms[width][order][gi] == min(tried)
    for k, part in enumerate(u.parts):
        r0, r1 = u.inst_rows[k], u.inst_rows[k + 1]
        # oracle on the garment alone, at the same state
        om = oracle.Mesh.from_workload(part)
        sel = (pairs[:, 0] >= r0) & (pairs[:, 0] < r1)
        rp, ci, vals, b = om.assemble(part.x0.astype(np.float64), part.v0.astype(np.float64), pairs[sel] - r0,
                                      w[sel], part.h)
        ref, _, _ = oracle.pcg(rp, ci, vals, b, tol=1e-12)
        assert H.rel_l2(got[r0:r1], ref) <= H.DV_RTOL, f"instance {k}"
        assert infos[k].rel_res <= 2e-9 and infos[k].iters > 0
    # the same systems solved one at a time with the single-instance solver
    single = torch.zeros_like(dv)
    pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], single,
                    pc.solve_opts(tol=1e-11, precision=pc.PC_PREC_MIXED, max_iter=50000))
    assert H.rel_l2(got, _np(single)) <= H.DV_RTOL


def test_batched_steps_follow_the_oracle(pc):
    u = small_batch()
    cl = pc.Cloth(u)
    opts = pc.pc_step_opts()
    opts.h = u.h
    opts.solve = pc.solve_opts(tol=1e-9, max_iter=50000)
    opts.warm_start = pc.PC_WARM_PREV
    meshes = [oracle.Mesh.from_workload(p) for p in u.parts]
    for step in range(3):
        x = _np(cl.x).astype(np.float64)
        v = _np(cl.v).astype(np.float64)
        pairs, w = u.contacts(step)
        pd, wd = cl.contacts_device(step)
        infos, st = pc.pc_step_batched(cl.ctx, cl.x, cl.v, pd, wd, u.inst_rows, opts)
        assert st == pc.PC_OK
        v1 = _np(cl.v).astype(np.float64)
        for k, (part, om) in enumerate(zip(u.parts, meshes)):
            r0, r1 = u.inst_rows[k], u.inst_rows[k + 1]
            sel = (pairs[:, 0] >= r0) & (pairs[:, 0] < r1)
            dv_ref, _, _, _ = om.step(x[r0:r1], v[r0:r1], pairs[sel] - r0, w[sel], h=u.h, tol=1e-12)
            err = H.rel_l2(v1[r0:r1] - v[r0:r1], dv_ref)
            print(f"batched step {step} garment {k}: dv rel err {err:.3e}")
            assert err <= H.DV_RTOL, f"step {step} instance {k}"


def test_batched_rejects_coupled_or_tiny_instances(pc):
    u = small_batch()
    cl = pc.Cloth(u)
    s = cl.assemble()
    dv = torch.zeros(cl.V * 3, device="cuda")
    cut = list(u.inst_rows)
    cut[1] += 10  # splits garment 0 / 1 across a mesh: blocks couple two instances
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve_batched(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], dv, cut)
    assert e.value.status == pc.PC_ERR_ARG
    tiny = [0, 16] + list(u.inst_rows[1:])
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve_batched(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], dv, tiny)
    assert e.value.status == pc.PC_ERR_ARG


def test_batched_not_converged_reports_per_instance(pc):
    u = small_batch()
    cl = pc.Cloth(u)
    s = cl.assemble()
    dv = torch.zeros(cl.V * 3, device="cuda")
    infos, st = pc.pc_pcg_solve_batched(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"],
                                        dv, u.inst_rows, pc.solve_opts(tol=1e-12, max_iter=5),
                                        allow_not_converged=True)
    assert st == pc.PC_ERR_NOT_CONVERGED
    assert all(i.iters == 5 for i in infos)
    assert np.isfinite(_np(dv)).all()


def test_batched_solve_is_deterministic_and_plain_form_agrees(pc):
    """Each garment's sums are taken in a fixed order (its CTA slots in order, the same in
    every CTA that needs them), so two solves of the same systems on the tuned launch shape
    give bit-identical dv and iteration counts. The plain form (no difference diagonal: the
    product streams A itself, the kernel's other instantiation) solves the same systems."""
    u = small_batch()
    cl = pc.Cloth(u)
    s = cl.assemble(*cl.contacts_device(0))
    opts = pc.solve_opts(tol=1e-9, max_iter=50000)
    args = (cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"])
    runs = []
    for _ in range(2):
        dv = torch.zeros(cl.V * 3, device="cuda")
        infos, st = pc.pc_pcg_solve_batched(*args, s["dres"], s["b"], dv, u.inst_rows, opts)
        assert st == pc.PC_OK
        runs.append((dv.clone(), [i.iters for i in infos]))
    assert torch.equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]
    plain = torch.zeros(cl.V * 3, device="cuda")
    infos, st = pc.pc_pcg_solve_batched(*args, None, s["b"], plain, u.inst_rows, opts)
    assert st == pc.PC_OK and all(i.rel_res <= 2e-9 for i in infos)
    got, ref = _np(plain).reshape(-1, 3), _np(runs[0][0]).reshape(-1, 3)
    for k in range(len(u.parts)):
        r0, r1 = u.inst_rows[k], u.inst_rows[k + 1]
        assert H.rel_l2(got[r0:r1], ref[r0:r1]) <= H.DV_RTOL, f"instance {k}"
