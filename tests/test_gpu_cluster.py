"""The cluster schedule (PC_SCHED_CLUSTER): the whole PCG solve of a small system in one
launch of one thread-block cluster, through the C ABI.

Checked against the FP64 oracle and against the grid-wide schedule: both preconditioners,
both precisions, the difference and the plain form, ragged and tiny systems (row counts
that leave CTAs with a partial row range or none), a warm start, the stop statuses, the
capacity refusal (on the host before the launch, and by the CTAs' own vote inside it,
with the automatic schedule then falling back to the grid), the FP64 solution it leaves
for pc_get_solution64, its timing counters, and a step that goes through it by default.
"""
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


def _np(t):
    return t.detach().cpu().numpy()


CASES = {
    "square64": lambda: wk.small_square(),
    "ragged37x29-contacts": lambda: H.small_contact_cloth(),
    "square45": lambda: wk.square_cloth(45, seed=77, steps=1, name="square45"),  # 2,025 rows: 127 per CTA, ragged
}


def _system(pc, wl):
    cl = pc.Cloth(wl)
    pairs, w = wl.contacts(0)
    s = cl.assemble(*cl.contacts_device(0))
    om = oracle.Mesh.from_workload(wl)
    rp, ci, vals_ref, b_ref = om.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), pairs, w, wl.h)
    return cl, s, (rp, ci, vals_ref, b_ref)


def _solve(pc, cl, s, dres, dv=None, **kw):
    dv = torch.zeros(cl.V * 3, device="cuda") if dv is None else dv
    info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], dres, s["b"], dv,
                               pc.solve_opts(**kw), allow_not_converged=True)
    return dv, info, st


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precond", ["jacobi", "block"])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_cluster_solve_matches_oracle_and_grid(pc, case, precond, precision):
    wl = CASES[case]()
    cl, s, (rp, ci, vals_ref, b_ref) = _system(pc, wl)
    dv_ref, _, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    pre = pc.PC_PRECOND_BLOCK if precond == "block" else pc.PC_PRECOND_JACOBI
    prec = pc.PC_PREC_MIXED if precision == "mixed" else pc.PC_PREC_FP32
    tol = 1e-9 if precision == "mixed" else 1e-6
    kw = dict(tol=tol, precision=prec, precond=pre, max_iter=50000)
    dv_c, info_c, st_c = _solve(pc, cl, s, s["dres"], schedule=pc.PC_SCHED_CLUSTER, **kw)
    dv_g, info_g, st_g = _solve(pc, cl, s, s["dres"], schedule=pc.PC_SCHED_GRID, **kw)
    err = H.rel_l2(_np(dv_c), dv_ref)
    print(f"{case} {precond} {precision}: cluster {info_c.iters} it (outer {info_c.outer}), grid {info_g.iters} it; "
          f"dv err vs oracle {err:.3e}, vs grid {H.rel_l2(_np(dv_c), _np(dv_g)):.3e}")
    assert st_c == pc.PC_OK and st_g == pc.PC_OK
    if precision == "mixed":
        assert info_c.rel_res <= 2 * tol and info_c.outer >= 1
        assert err <= H.DV_RTOL
    else:
        # as for the grid schedule: FP32 PCG stops on its recurrence residual
        assert info_c.rel_res <= 1e-4 and err <= 1e-4 and info_c.outer == 0
    # the cluster schedule runs the single-reduction (Chronopoulos-Gear) form of the same
    # method: the same count in FP32 and at moderate tolerances; near FP32's attainable
    # accuracy (the mixed form at 1e-9) its residual recurrence, which goes through the
    # recurrence for A p, needs up to about a third more iterations
    slack = 0.35 if precision == "mixed" else 0.05
    assert info_c.iters <= (1 + slack) * info_g.iters + 5 and info_c.iters >= 0.9 * info_g.iters - 5
    assert (_np(dv_c).reshape(-1, 3)[wl.pins] == 0).all()


@pytest.mark.parametrize("case", list(CASES))
def test_cluster_iterations_at_the_benchmark_tolerance(pc, case):
    """At a relative residual of 1e-6 (the benchmark's) the single-reduction form takes the
    iterations of the grid schedule's two-reduction form, within a few."""
    wl = CASES[case]()
    cl, s, _ = _system(pc, wl)
    kw = dict(tol=1e-6, precision=pc.PC_PREC_MIXED, max_iter=50000)
    _, info_c, st_c = _solve(pc, cl, s, s["dres"], schedule=pc.PC_SCHED_CLUSTER, **kw)
    _, info_g, st_g = _solve(pc, cl, s, s["dres"], schedule=pc.PC_SCHED_GRID, **kw)
    print(f"{case}: cluster {info_c.iters}, grid {info_g.iters} iterations at 1e-6")
    assert st_c == pc.PC_OK and st_g == pc.PC_OK and info_c.rel_res <= 1e-6
    assert abs(info_c.iters - info_g.iters) <= 0.03 * info_g.iters + 3


def test_cluster_plain_form_matches_grid(pc):
    """Without the difference-form diagonal the product reads every block, the diagonal
    block included; the same FP32 matrix solved on both schedules."""
    wl = H.small_contact_cloth()
    cl, s, _ = _system(pc, wl)
    kw = dict(tol=1e-11, precision=pc.PC_PREC_MIXED, max_iter=50000)
    dv_c, info_c, st_c = _solve(pc, cl, s, None, schedule=pc.PC_SCHED_CLUSTER, **kw)
    dv_g, info_g, st_g = _solve(pc, cl, s, None, schedule=pc.PC_SCHED_GRID, storage=pc.PC_STORAGE_FULL, **kw)
    assert st_c == pc.PC_OK and st_g == pc.PC_OK and info_c.rel_res <= 2e-11
    assert H.rel_l2(_np(dv_c), _np(dv_g)) <= 1e-6


@pytest.mark.parametrize("n", [2, 3, 5])
def test_cluster_tiny_systems(pc, n):
    """n x n sheets (4, 9 and 25 rows): most CTAs own no row. An unpinned sheet in free
    fall has dv = h g exactly."""
    rest, tris, _ = wk.grid_piece(n, n, 0.1, 0.1, jitter=0.0, flip_prob=0.0, seed=3)
    wl = wk.Workload("tiny", rest, tris, np.zeros(0, np.int32), rest.copy(), np.zeros_like(rest), 1 / 200,
                     wk.Material(), [], 0)
    cl = pc.Cloth(wl, max_contacts=0)
    s = cl.assemble()
    for prec in (pc.PC_PREC_MIXED, pc.PC_PREC_FP32):
        dv, info, st = _solve(pc, cl, s, s["dres"], tol=1e-10, precision=prec, schedule=pc.PC_SCHED_CLUSTER)
        assert st == pc.PC_OK
        np.testing.assert_allclose(_np(dv).reshape(-1, 3), np.tile([0, 0, -9.81 / 200], (cl.V, 1)), atol=1e-7)


def test_cluster_warm_start_and_stop_statuses(pc):
    wl = wk.small_square()
    cl, s, (rp, ci, vals_ref, b_ref) = _system(pc, wl)
    dv_ref, _, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    kw = dict(precision=pc.PC_PREC_MIXED, schedule=pc.PC_SCHED_CLUSTER)
    _, cold, _ = _solve(pc, cl, s, s["dres"], tol=1e-9, max_iter=50000, **kw)
    # a warm start near the answer needs fewer iterations and reaches the same solution
    guess = torch.from_numpy((dv_ref * (1 + 1e-3 * np.sin(np.arange(dv_ref.size)).reshape(dv_ref.shape)))
                             .astype(np.float32).reshape(-1)).cuda()
    dv, warm, st = _solve(pc, cl, s, s["dres"], dv=guess, tol=1e-9, max_iter=50000, **kw)
    assert st == pc.PC_OK and warm.iters < cold.iters
    assert H.rel_l2(_np(dv), dv_ref) <= H.DV_RTOL
    # the iteration limit: the status, exactly max_iter iterations, a finite iterate
    dv, info, st = _solve(pc, cl, s, s["dres"], tol=1e-12, max_iter=5, **kw)
    assert st == pc.PC_ERR_NOT_CONVERGED and info.iters == 5 and info.rel_res > 1e-12
    assert np.isfinite(_np(dv)).all()
    dv, info, st = _solve(pc, cl, s, s["dres"], tol=1e-12, max_iter=0, **kw)
    assert st == pc.PC_ERR_NOT_CONVERGED and info.iters == 0 and np.all(_np(dv) == 0)
    # a non-finite right-hand side
    b = s["b"].clone()
    b[7] = float("nan")
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], b,
                        torch.zeros(cl.V * 3, device="cuda"), pc.solve_opts(tol=1e-9, **kw))
    assert e.value.status == pc.PC_ERR_NONFINITE
    # the context still solves afterwards
    dv, info, st = _solve(pc, cl, s, s["dres"], tol=1e-9, max_iter=50000, **kw)
    assert st == pc.PC_OK and info.iters == cold.iters


def test_cluster_refuses_large_systems_and_auto_falls_back(pc):
    """128 x 128 (16,384 rows, 1,024 per CTA) leaves no shared memory for the blocks: the
    host refuses it before any launch."""
    wl = wk.square_cloth(128, seed=5, steps=1, name="square128")
    cl = pc.Cloth(wl)
    s = cl.assemble()
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"],
                        torch.zeros(cl.V * 3, device="cuda"), pc.solve_opts(schedule=pc.PC_SCHED_CLUSTER))
    assert e.value.status == pc.PC_ERR_CAPACITY
    kw = dict(tol=1e-8, precision=pc.PC_PREC_MIXED, max_iter=50000)
    dv_a, info_a, st_a = _solve(pc, cl, s, s["dres"], schedule=pc.PC_SCHED_AUTO, **kw)
    dv_g, info_g, st_g = _solve(pc, cl, s, s["dres"], schedule=pc.PC_SCHED_GRID, **kw)
    assert st_a == pc.PC_OK and info_a.iters == info_g.iters and torch.equal(dv_a, dv_g)


def _lopsided_spd(V):
    """Rows [0, 256) couple to rows r + 256 q (q = 1..15) and r + 256 q + 128 (q = 1..14),
    mirrored: 30 blocks each; every other row has its diagonal block and at most two
    mirrors. Off-diagonal blocks 0.1 x random symmetric, diagonal blocks (sum of the row's
    off-diagonal norms + 1) I: block diagonally dominant, so SPD."""
    rng = np.random.default_rng(21)
    cols = [{i} for i in range(V)]
    for r in range(256):
        for c in [r + 256 * q for q in range(1, 16)] + [r + 256 * q + 128 for q in range(1, 15)]:
            cols[r].add(c)
            cols[c].add(r)
    blocks = {}
    for i in range(V):
        for j in cols[i]:
            if j > i:
                m = rng.uniform(-1.0, 1.0, size=(3, 3))
                blocks[(i, j)] = 0.1 * (m + m.T)
                blocks[(j, i)] = blocks[(i, j)].T
    rp = np.zeros(V + 1, np.int32)
    rp[1:] = np.cumsum([len(c) for c in cols])
    nnzb = int(rp[-1])
    cap = (nnzb + 3) // 4 * 4
    ci = np.zeros(cap, np.int32)
    vals = np.zeros((cap, 3, 3), np.float32)
    for i in range(V):
        row = sorted(cols[i])
        off = sum(np.linalg.norm(blocks[(i, j)]) for j in row if j != i)
        for n, j in enumerate(row):
            ci[rp[i] + n] = j
            vals[rp[i] + n] = (off + 1.0) * np.eye(3) if j == i else blocks[(i, j)]
    return rp, ci, nnzb, vals


def test_cluster_vote_when_one_cta_overflows(pc):
    """4,096 rows (256 per CTA) where the first CTA's rows carry 30 blocks each (7,680,
    beyond one CTA's shared memory) and the average CTA's fit: the host lets the launch go,
    the CTAs vote inside it and none runs. The forced schedule reports PC_ERR_CAPACITY;
    the automatic one then solves on the grid (bitwise the grid schedule's solve)."""
    wl = wk.small_square()
    cl = pc.Cloth(wl)
    assert cl.V == 4096
    rp, ci, nnzb, vals = _lopsided_spd(cl.V)
    assert rp[256] - rp[0] == 256 * 30 and nnzb // 16 < 2000
    b = np.random.default_rng(4).normal(size=cl.V * 3).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (rp, ci, vals.reshape(-1), b)]
    with pytest.raises(pc.PcError) as e:
        pc.pc_pcg_solve(cl.ctx, t[0], t[1], nnzb, t[2], None, t[3], torch.zeros(cl.V * 3, device="cuda"),
                        pc.solve_opts(schedule=pc.PC_SCHED_CLUSTER))
    assert e.value.status == pc.PC_ERR_CAPACITY
    out = {}
    for sched in (pc.PC_SCHED_AUTO, pc.PC_SCHED_GRID):
        dv = torch.zeros(cl.V * 3, device="cuda")
        info, st = pc.pc_pcg_solve(cl.ctx, t[0], t[1], nnzb, t[2], None, t[3], dv,
                                   pc.solve_opts(tol=1e-10, precision=pc.PC_PREC_MIXED, max_iter=5000,
                                                 schedule=sched))
        assert st == pc.PC_OK
        out[sched] = (info.iters, _np(dv))
    assert out[pc.PC_SCHED_AUTO][0] == out[pc.PC_SCHED_GRID][0]
    assert np.array_equal(out[pc.PC_SCHED_AUTO][1], out[pc.PC_SCHED_GRID][1])
    # the FP64 residual of the FP32 solution (a well-conditioned matrix: near FP32 rounding)
    x = out[pc.PC_SCHED_GRID][1].astype(np.float64).reshape(-1, 3)
    r = b.astype(np.float64).reshape(-1, 3) - oracle.spmv(rp, ci[:nnzb], vals[:nnzb], x)
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(b)


def test_cluster_fp64_solution_and_counters(pc):
    wl = H.small_contact_cloth()
    cl, s, _ = _system(pc, wl)
    pc.pc_set_profiling(cl.ctx, True)
    pc.pc_cluster_stats(cl.ctx)  # reset
    dv, info, st = _solve(pc, cl, s, s["dres"], tol=1e-9, precision=pc.PC_PREC_MIXED, max_iter=50000,
                          schedule=pc.PC_SCHED_CLUSTER)
    assert st == pc.PC_OK
    solves, iters, ms = pc.pc_cluster_stats(cl.ctx)
    assert solves == 1 and iters == info.iters and ms > 0.0
    print(f"ragged37x29 cluster solve: {iters} iterations in {ms:.3f} ms ({1e3 * ms / iters:.2f} us/iteration)")
    pc.pc_set_profiling(cl.ctx, False)
    # the FP64 iterate the solve ended with; dv is its rounding
    dv64 = torch.zeros(cl.V * 3, dtype=torch.float64, device="cuda")
    pc.pc_get_solution64(cl.ctx, dv64)
    assert torch.equal(dv64.float(), dv)


def test_default_step_runs_on_the_cluster(pc):
    """pc_step with the default (automatic) schedule on the 64 x 64 cloth takes the
    cluster schedule and matches the grid schedule's step."""
    wl = wk.small_square()
    a, b = pc.Cloth(wl), pc.Cloth(wl)
    pc.pc_set_profiling(a.ctx, True)
    pc.pc_cluster_stats(a.ctx)
    da = torch.zeros(a.V * 3, device="cuda")
    db = torch.zeros(b.V * 3, device="cuda")
    a.step(tol=1e-8, precision=pc.PC_PREC_MIXED, dv_out=da)
    b.step(tol=1e-8, precision=pc.PC_PREC_MIXED, dv_out=db, schedule=pc.PC_SCHED_GRID)
    solves, _, _ = pc.pc_cluster_stats(a.ctx)
    assert solves == 1
    assert H.rel_l2(_np(da), _np(db)) <= H.DV_RTOL
