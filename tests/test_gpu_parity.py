"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Pattern (row_ptr, col_idx): bit-exact. Block values: within the per-block tolerance of
_helpers. dv: within 1e-5 relative L2 of the oracle solved to 1e-12. The oracle is fed
the GPU's own FP32 state cast exactly to FP64 (Sec. 2.5 Eq. 3 at the same x_t, v_t).
"""
import dataclasses

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


def _setup(pc, wl, step=0):
    cl = pc.Cloth(wl)
    om = oracle.Mesh.from_workload(wl)
    pairs, w = wl.contacts(step)
    pd, wd = cl.contacts_device(step)
    return cl, om, pairs, w, pd, wd


def _damped(wl):
    """The same workload with Rayleigh damping (alpha = 2 / s, beta = 0.01 s)."""
    return dataclasses.replace(wl, material=dataclasses.replace(wl.material, damp_mass=2.0, damp_stiff=0.01))


CASES = {
    "square64": lambda: wk.small_square(),
    "ragged37x29-contacts": lambda: H.small_contact_cloth(),
    "stack3x21-interlayer": lambda: H.small_stack(),
    "ragged37x29-contacts-damped": lambda: _damped(H.small_contact_cloth()),
}


@pytest.mark.parametrize("case", list(CASES))
def test_rest_state_matches_oracle(pc, case):
    wl = CASES[case]()
    cl, om, *_ = _setup(pc, wl)
    assert cl.H == om.H
    hinges = torch.zeros((max(cl.H, 1), 4), dtype=torch.int32, device="cuda")
    mass = torch.zeros(cl.V, dtype=torch.float32, device="cuda")
    pc.pc_get_rest(cl.ctx, hinges, mass)
    np.testing.assert_array_equal(_np(hinges)[: cl.H], om.hinges)
    np.testing.assert_allclose(_np(mass), om.mass, rtol=2e-7)
    assert cl.static_nnzb == len(om.pattern()[1])


@pytest.mark.parametrize("case", list(CASES))
def test_pattern_bit_exact(pc, case):
    wl = CASES[case]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    for step in range(2):
        pairs, w = wl.contacts(step)
        pd, wd = cl.contacts_device(step)
        s = cl.alloc_system()
        nnzb = pc.pc_assemble_pattern(cl.ctx, pd, wd, s["row_ptr"], s["col_idx"])
        rp, ci = om.pattern(pairs)
        assert nnzb == len(ci)
        np.testing.assert_array_equal(_np(s["row_ptr"]), rp)
        np.testing.assert_array_equal(_np(s["col_idx"])[:nnzb], ci)


@pytest.mark.parametrize("case", list(CASES))
def test_values_and_rhs_match_oracle(pc, case):
    wl = CASES[case]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    # a non-trivial state: perturbed positions and velocities
    rng = np.random.default_rng(3)
    x = wl.x0 + (2e-4 * rng.normal(size=wl.x0.shape)).astype(np.float32)
    v = (0.05 * rng.normal(size=wl.x0.shape)).astype(np.float32)
    cl.x.copy_(torch.from_numpy(x))
    cl.v.copy_(torch.from_numpy(v))
    s = cl.assemble(pd, wd)
    nnzb = s["nnzb"]
    rp, ci, vals_ref, b_ref = om.assemble(x.astype(np.float64), v.astype(np.float64), pairs, w, wl.h)
    vals = _np(s["vals"])[: 9 * nnzb].reshape(-1, 3, 3)
    excess = H.block_errors(rp, ci, vals, vals_ref)
    assert excess.max() <= 0, f"worst block excess {excess.max():.3e}"
    b = _np(s["b"]).reshape(-1, 3)
    assert H.rel_l2(b, b_ref) <= 1e-5
    # bitwise symmetry: block (i, j) is the transpose of block (j, i)
    rows = np.repeat(np.arange(cl.V), np.diff(rp))
    key = rows.astype(np.int64) * cl.V + ci
    tkey = ci.astype(np.int64) * cl.V + rows
    order = np.argsort(key)
    tpos = order[np.searchsorted(key[order], tkey)]
    np.testing.assert_array_equal(vals, vals[tpos].transpose(0, 2, 1))


@pytest.mark.parametrize("case", list(CASES))
def test_difference_diagonal_and_spmv(pc, case):
    wl = CASES[case]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    s = cl.assemble(pd, wd)
    nnzb = s["nnzb"]
    x = wl.x0.astype(np.float64)
    v = wl.v0.astype(np.float64)
    rp, ci, vals_ref, _ = om.assemble(x, v, pairs, w, wl.h)
    _, _, vals_nopin, _ = om.assemble(x, v, pairs, w, wl.h, pins=False)
    # D_i = (1 + h alpha) m_i I - sum over pinned neighbours j of the unzeroed block A_ij
    # (alpha the Rayleigh mass damping; a pinned row keeps m_i I)
    md = np.where(om.pinned, 1.0, 1.0 + wl.h * wl.material.damp_mass)
    D_ref = np.tile(np.eye(3), (cl.V, 1, 1)) * (md * om.mass)[:, None, None]
    rows = np.repeat(np.arange(cl.V), np.diff(rp))
    for sl in np.nonzero(om.pinned[ci] & (ci != rows) & ~om.pinned[rows])[0]:
        D_ref[rows[sl]] -= vals_nopin[sl]
    D = _np(s["dres"]).reshape(-1, 3, 3)
    np.testing.assert_allclose(D, D_ref, rtol=1e-5, atol=1e-7 * np.abs(D_ref).max())
    rng = np.random.default_rng(5)
    for trial in range(2):
        p = rng.normal(size=(cl.V, 3)).astype(np.float32)
        if trial == 1:  # a smooth vector: translation plus a small ripple
            p = (np.array([0.3, -0.2, 1.0]) + 1e-3 * p).astype(np.float32)
        y_ref = oracle.spmv(rp, ci, vals_ref, p.astype(np.float64))
        scale = oracle.spmv(rp, ci, np.abs(vals_ref), np.abs(p.astype(np.float64)))
        pt = torch.from_numpy(p.reshape(-1)).cuda()
        for dres in (None, s["dres"]):
            y = torch.zeros_like(pt)
            pc.pc_bsr_spmv(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"], dres, pt, y)
            err = np.abs(_np(y).reshape(-1, 3) - y_ref)
            assert (err <= 1e-5 * scale + 1e-30).all()
        # the difference form is exact on translations: y = M t
        if trial == 1:
            t = torch.from_numpy(np.tile(np.array([0.3, -0.2, 1.0], np.float32), cl.V)).cuda()
            y = torch.zeros_like(t)
            pc.pc_bsr_spmv(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"], s["dres"], t, y)
            yt = oracle.spmv(rp, ci, vals_ref, _np(t).reshape(-1, 3).astype(np.float64))
            assert H.rel_l2(_np(y), yt) <= 1e-5


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed-bench"])
@pytest.mark.parametrize("schedule", ["grid", "cluster"])
def test_pcg_solution_matches_oracle(pc, case, precision, schedule):
    """dv against the oracle solved to 1e-12, on both schedules (grid-wide kernels, and the
    whole solve inside one thread-block cluster). "mixed-bench" is the configuration the
    benchmark times (mixed precision, tol 1e-6): on these small systems a 1e-6 residual
    already bounds the dv error by 1e-5."""
    wl = CASES[case]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    s = cl.assemble(pd, wd)
    x = wl.x0.astype(np.float64)
    rp, ci, vals_ref, b_ref = om.assemble(x, wl.v0.astype(np.float64), pairs, w, wl.h)
    dv_ref, it_ref, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    prec = pc.PC_PREC_FP32 if precision == "fp32" else pc.PC_PREC_MIXED
    tol = 1e-9 if precision == "mixed" else 1e-6
    dv = torch.zeros(cl.V * 3, device="cuda")
    sched = pc.PC_SCHED_GRID if schedule == "grid" else pc.PC_SCHED_CLUSTER
    info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], dv,
                               pc.solve_opts(tol=tol, precision=prec, max_iter=50000, schedule=sched))
    err = H.rel_l2(_np(dv), dv_ref)
    print(f"{case} {precision} {schedule} tol {tol:g}: {info.iters} iterations, dv rel err {err:.3e}")
    if precision != "fp32":
        assert info.rel_res <= 2 * tol
        assert err <= H.DV_RTOL, f"dv rel err {err:.3e}"
    else:
        # FP32 PCG stops on its FP32 recurrence residual; the FP64 residual of an FP32
        # iterate of these stiff systems stalls near 1e-5, so the FP32 form is held to
        # the accuracy its own residual allows
        assert info.rel_res <= 1e-4
        assert err <= 1e-4, f"dv rel err {err:.3e} (true residual {info.rel_res:.2e})"
    assert (_np(dv).reshape(-1, 3)[wl.pins] == 0).all()


@pytest.mark.parametrize("tol", [1e-9, 1e-6])
def test_twenty_step_trajectory_small_square(pc, tol):
    """64 x 64 cloth, 20 steps: per-step dv parity with the oracle fed the same state, at
    a tight tolerance and at the benchmark's 1e-6."""
    wl = wk.small_square()
    cl = pc.Cloth(wl)
    om = oracle.Mesh.from_workload(wl)
    dv = torch.zeros(cl.V * 3, device="cuda")
    worst = 0.0
    for step in range(wl.steps):
        x = _np(cl.x).astype(np.float64)
        v = _np(cl.v).astype(np.float64)
        info, st = cl.step(tol=tol, precision=pc.PC_PREC_MIXED, dv_out=dv)
        dv_ref, _, _, oinfo = om.step(x, v, h=wl.h, tol=1e-12)
        err = H.rel_l2(_np(dv), dv_ref)
        worst = max(worst, err)
        assert err <= H.DV_RTOL, f"step {step}: rel err {err:.3e}"
    print(f"square64 trajectory tol {tol:g}: worst dv rel err over {wl.steps} steps {worst:.3e}")
    # the state really moved and stayed finite
    assert np.isfinite(_np(cl.x)).all() and np.abs(_np(cl.x) - wl.x0).max() > 1e-3


def test_benchmark_tolerance_both_precisions(pc):
    """At tol 1e-6 the mixed form meets the FP64 residual; plain FP32 converges on its
    recurrence residual and reports a true residual within two decades of it."""
    wl = wk.small_square()
    cl = pc.Cloth(wl)
    info, st = cl.step(tol=1e-6, precision=pc.PC_PREC_FP32)
    assert st == pc.PC_OK and info.solve.rel_res <= 1e-4
    info, st = cl.step(tol=1e-6, precision=pc.PC_PREC_MIXED)
    assert st == pc.PC_OK and info.solve.rel_res <= 1e-6


# ------------------------------------------------------------------------- edge cases


def test_isolated_vertices_are_reported(pc):
    # vertices in no triangle have zero lumped mass, so A is singular there: the solve
    # must report it instead of producing NaNs
    rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [2, 2, 2], [3, 3, 3]], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    wl = wk.Workload("tiny", rest, tris, np.zeros(0, np.int32), rest.copy(), np.zeros_like(rest), 1 / 200,
                     wk.Material(), [], 0)
    cl = pc.Cloth(wl, max_contacts=0)
    with pytest.raises(pc.PcError) as e:
        cl.step(tol=1e-10, precision=pc.PC_PREC_MIXED)
    assert e.value.status == pc.PC_ERR_NONFINITE


def test_single_triangle_free_fall(pc):
    rest = np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0]], np.float32)
    wl = wk.Workload("one", rest, np.array([[0, 1, 2]], np.int32), np.zeros(0, np.int32), rest.copy(),
                     np.zeros_like(rest), 1 / 200, wk.Material(), [], 0)
    cl = pc.Cloth(wl, max_contacts=0)
    assert cl.H == 0 and cl.static_nnzb == 9
    dv = torch.zeros(9, device="cuda")
    cl.step(tol=1e-10, precision=pc.PC_PREC_MIXED, dv_out=dv)
    np.testing.assert_allclose(_np(dv).reshape(-1, 3), np.tile([0, 0, -9.81 / 200], (3, 1)), atol=1e-7)


def test_free_fall_unpinned_sheet(pc):
    rest, tris, _ = wk.grid_piece(9, 7, 0.2, 0.15, jitter=0.2, flip_prob=0.2, seed=9)
    wl = wk.Workload("ff", rest, tris, np.zeros(0, np.int32), rest.copy(), np.zeros_like(rest), 1 / 200,
                     wk.Material(), [], 0)
    cl = pc.Cloth(wl, max_contacts=0)
    dv = torch.zeros(cl.V * 3, device="cuda")
    cl.step(tol=1e-10, precision=pc.PC_PREC_MIXED, dv_out=dv)
    np.testing.assert_allclose(_np(dv).reshape(-1, 3), np.tile([0, 0, -9.81 / 200], (cl.V, 1)), atol=1e-7)


def test_capacity_error_reports_required(pc):
    wl = H.small_contact_cloth()
    cl = pc.Cloth(wl)
    pd, wd = cl.contacts_device(0)
    s = cl.alloc_system()
    need = pc.pc_assemble_pattern(cl.ctx, pd, wd, s["row_ptr"], s["col_idx"])
    small = torch.zeros((need // 4) * 4 - 4, dtype=torch.int32, device="cuda")
    with pytest.raises(pc.PcError) as e:
        pc.pc_assemble_pattern(cl.ctx, pd, wd, s["row_ptr"], small)
    assert e.value.status == pc.PC_ERR_CAPACITY and e.value.required == need


def test_invalid_contact_rejected(pc):
    wl = H.small_contact_cloth()
    cl = pc.Cloth(wl)
    pairs, w = wl.contacts(0)
    bad = pairs.copy()
    bad[0, 1] = bad[0, 0]  # p repeated in its own triangle
    s = cl.alloc_system()
    with pytest.raises(pc.PcError) as e:
        pc.pc_assemble_pattern(cl.ctx, torch.from_numpy(bad).cuda(), torch.from_numpy(w).cuda(), s["row_ptr"],
                               s["col_idx"])
    assert e.value.status == pc.PC_ERR_ARG
    bad = pairs.copy()
    bad[1, 2] = cl.V + 5
    with pytest.raises(pc.PcError) as e:
        pc.pc_assemble_pattern(cl.ctx, torch.from_numpy(bad).cuda(), torch.from_numpy(w).cuda(), s["row_ptr"],
                               s["col_idx"])
    assert e.value.status == pc.PC_ERR_ARG


def test_invalid_mesh_rejected(pc):
    rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [2, 0, 0]], np.float32)
    for tris in ([[0, 1, 7]], [[0, 1, 1]], [[0, 1, 2], [1, 0, 3], [0, 1, 4]]):
        t = torch.tensor(tris, dtype=torch.int32, device="cuda")
        with pytest.raises(pc.PcError):
            pc.pc_create(5, len(tris), t, torch.from_numpy(rest).cuda(), None, wk.Material(), 0)


def test_nonfinite_state_and_not_converged(pc):
    wl = wk.small_square()
    cl = pc.Cloth(wl)
    info, st = cl.step(tol=1e-12, max_iter=3, allow_not_converged=True)
    assert st == pc.PC_ERR_NOT_CONVERGED and info.solve.iters == 3 and info.solve.rel_res > 1e-12
    cl2 = pc.Cloth(wl)
    cl2.x[10, 2] = float("nan")
    with pytest.raises(pc.PcError) as e:
        cl2.step(tol=1e-6)
    assert e.value.status == pc.PC_ERR_NONFINITE


def test_host_buffer_step_matches_device_step(pc):
    wl = H.small_contact_cloth()
    a = pc.Cloth(wl)
    b = pc.Cloth(wl)
    pairs, w = wl.contacts(0)
    pd, wd = a.contacts_device(0)
    a.step(pd, wd, tol=1e-8, precision=pc.PC_PREC_MIXED)
    xh = wl.x0.copy()
    vh = wl.v0.copy()
    o = pc.pc_step_opts()
    o.h = wl.h
    o.solve = pc.solve_opts(tol=1e-8, precision=pc.PC_PREC_MIXED)
    o.warm_start = pc.PC_WARM_ZERO
    pc.pc_step_host(b.ctx, xh, vh, pairs, w, o)
    np.testing.assert_array_equal(xh, _np(a.x))
    np.testing.assert_array_equal(vh, _np(a.v))


@pytest.mark.parametrize("schedule", ["grid", "cluster"])
def test_deterministic_repeat(pc, schedule):
    wl = H.small_contact_cloth()
    sched = pc.PC_SCHED_GRID if schedule == "grid" else pc.PC_SCHED_CLUSTER
    outs = []
    for _ in range(2):
        cl = pc.Cloth(wl)
        pd, wd = cl.contacts_device(0)
        s = cl.assemble(pd, wd)
        dv = torch.zeros(cl.V * 3, device="cuda")
        pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], dv,
                        pc.solve_opts(schedule=sched))
        outs.append((_np(s["vals"]).copy(), _np(s["b"]).copy(), _np(dv).copy()))
    for u, v in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("form", ["difference", "plain"])
def test_all_storages_agree_with_oracle(pc, case, form):
    """Full BSR, symmetric upper storage, sliced ELL and the BSR copy without diagonal
    blocks. Difference form: each against
    the oracle's exact solve. Plain form (A's FP32 blocks without the exact row sums, so
    the near-rigid modes carry the blocks' rounding: not within 1e-5 of the FP64 system
    on these stiff cloths): the three layouts solve the same FP32 matrix and must agree
    with each other."""
    wl = CASES[case]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    s = cl.assemble(pd, wd)
    dres = s["dres"] if form == "difference" else None
    rp, ci, vals_ref, b_ref = om.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), pairs, w, wl.h)
    dv_ref, _, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    tol = 1e-9 if form == "difference" else 1e-11
    out = {}
    for storage in (pc.PC_STORAGE_FULL, pc.PC_STORAGE_SYM, pc.PC_STORAGE_SELL, pc.PC_STORAGE_OFFDIAG, "cluster"):
        dv = torch.zeros(cl.V * 3, device="cuda")
        o = (pc.solve_opts(tol=tol, precision=pc.PC_PREC_MIXED, max_iter=50000, schedule=pc.PC_SCHED_CLUSTER)
             if storage == "cluster" else
             pc.solve_opts(tol=tol, precision=pc.PC_PREC_MIXED, max_iter=50000, storage=storage,
                           schedule=pc.PC_SCHED_GRID))
        info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], dres, s["b"], dv, o)
        assert st == pc.PC_OK and info.rel_res <= 2 * tol
        if form == "difference":
            assert H.rel_l2(_np(dv), dv_ref) <= H.DV_RTOL
        else:
            assert H.rel_l2(_np(dv), out[pc.PC_STORAGE_FULL][1] if out else _np(dv)) <= 1e-6
        out[storage] = (info.iters, _np(dv))
    # same method, products summed in another order: nearly the same iteration count. Near
    # 1e-9 the FP32 inner iterations stagnate between FP64 replacements and the count
    # depends on summation order (measured: 809..931 on the 64^2 cloth for the four
    # layouts, fused or not; within 1% at 1e-6); the plain form at 1e-11 more so
    slack = 0.12 if form == "difference" else 0.15
    for storage in (pc.PC_STORAGE_SYM, pc.PC_STORAGE_SELL, pc.PC_STORAGE_OFFDIAG):
        assert abs(out[storage][0] - out[pc.PC_STORAGE_FULL][0]) <= slack * out[pc.PC_STORAGE_FULL][0] + 5
    # the cluster schedule's single-reduction form needs up to about a third more
    # iterations this close to FP32's attainable accuracy (tests/test_gpu_cluster.py)
    assert out["cluster"][0] <= 1.35 * out[pc.PC_STORAGE_FULL][0] + 5
    if form == "plain":  # the copy without diagonal blocks is for the difference form only
        assert out[pc.PC_STORAGE_OFFDIAG][0] == out[pc.PC_STORAGE_FULL][0]
        assert np.array_equal(out[pc.PC_STORAGE_OFFDIAG][1], out[pc.PC_STORAGE_FULL][1])


def test_sliced_ell_product_and_fallback(pc):
    """One PCG iteration from a zero guess gives x = alpha D^-1 b with alpha = r.z / z.Az,
    so z.Az of the sliced-ELL product is checked against an FP64 product of the same
    matrix; a matrix denser than the context's capacity falls back to the full matrix
    (bitwise the same solve)."""
    wl = wk.garment(8, seed=91, stream=400)
    cl = pc.Cloth(wl)
    V = cl.V
    # dense coupling: every pair of rows shares a block (I), diagonal (V + 1) I: SPD
    rp = np.arange(V + 1, dtype=np.int32) * V
    ci = np.tile(np.arange(V, dtype=np.int32), V)
    vals = np.tile(np.eye(3, dtype=np.float32), (V * V, 1, 1))
    vals[np.arange(V) * V + np.arange(V)] *= V + 1
    rng = np.random.default_rng(8)
    b = rng.normal(size=V * 3).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (rp, ci, vals.reshape(-1), b)]
    res = {}
    for storage in (pc.PC_STORAGE_FULL, pc.PC_STORAGE_SELL):
        dv = torch.zeros(V * 3, device="cuda")
        info, st = pc.pc_pcg_solve(cl.ctx, t[0], t[1], V * V, t[2], None, t[3], dv,
                                   pc.solve_opts(tol=1e-7, precision=pc.PC_PREC_MIXED, max_iter=500, storage=storage,
                                                 schedule=pc.PC_SCHED_GRID))
        res[storage] = (st, info.iters, _np(dv))
    assert res[pc.PC_STORAGE_FULL][0] == pc.PC_OK
    assert res[pc.PC_STORAGE_SELL][1] == res[pc.PC_STORAGE_FULL][1]
    assert np.array_equal(res[pc.PC_STORAGE_SELL][2], res[pc.PC_STORAGE_FULL][2])
    # a single iteration on the step system in sliced ELL
    s = cl.assemble(*cl.contacts_device(0))
    nnzb = s["nnzb"]
    A = oracle.dense(_np(s["row_ptr"]), _np(s["col_idx"])[:nnzb],
                     _np(s["vals"])[: 9 * nnzb].astype(np.float64).reshape(-1, 3, 3))
    bb = _np(s["b"]).astype(np.float64)
    z = bb / np.diag(A)
    alpha = (bb @ z) / (z @ A @ z)
    for form in ("difference", "plain"):
        dv = torch.zeros(V * 3, device="cuda")
        pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"],
                        s["dres"] if form == "difference" else None, s["b"], dv,
                        pc.solve_opts(tol=1e-12, precision=pc.PC_PREC_FP32, max_iter=1, storage=pc.PC_STORAGE_SELL,
                                      schedule=pc.PC_SCHED_GRID),
                        allow_not_converged=True)
        np.testing.assert_allclose(_np(dv).astype(np.float64), alpha * z, rtol=2e-5, atol=1e-7 * np.abs(alpha * z).max())


def test_asymmetric_pattern_falls_back_to_full_storage(pc):
    wl = CASES["ragged37x29-contacts"]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    s = cl.assemble(pd, wd)
    nnzb = s["nnzb"]
    rp = _np(s["row_ptr"]).astype(np.int64)
    ci = _np(s["col_idx"])[:nnzb]
    vals = _np(s["vals"])[: 9 * nnzb].reshape(-1, 9)
    # add an explicit zero block (i, j) to row i only: the matrix is unchanged, the
    # pattern is no longer symmetric
    i, j = 100, cl.V - 1
    assert j not in ci[rp[i]:rp[i + 1]]
    k = rp[i] + int(np.searchsorted(ci[rp[i]:rp[i + 1]], j))
    ci2 = np.insert(ci, k, j).astype(np.int32)
    v2 = np.insert(vals, k, np.zeros(9, np.float32), axis=0)
    rp2 = rp.copy()
    rp2[i + 1:] += 1
    n2 = nnzb + 1
    cap = (n2 + 3) // 4 * 4
    ci_p = np.zeros(cap, np.int32)
    ci_p[:n2] = ci2
    v_p = np.zeros((cap, 9), np.float32)
    v_p[:n2] = v2
    args = [torch.from_numpy(rp2.astype(np.int32)).cuda(), torch.from_numpy(ci_p).cuda(), n2,
            torch.from_numpy(v_p.reshape(-1)).cuda(), s["dres"], s["b"]]
    res = {}
    for storage in (pc.PC_STORAGE_SYM, pc.PC_STORAGE_FULL):
        dv = torch.zeros(cl.V * 3, device="cuda")
        info, st = pc.pc_pcg_solve(cl.ctx, *args, dv, pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED,
                                                                      max_iter=50000, storage=storage,
                                                                      schedule=pc.PC_SCHED_GRID))
        res[storage] = (st, info.iters, _np(dv))
    assert res[pc.PC_STORAGE_FULL][0] == pc.PC_OK
    # the symmetric layout is refused and the full matrix gives the identical solve
    assert res[pc.PC_STORAGE_SYM][1] == res[pc.PC_STORAGE_FULL][1]
    assert np.array_equal(res[pc.PC_STORAGE_SYM][2], res[pc.PC_STORAGE_FULL][2])


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precond", ["jacobi", "block"])
def test_fused_and_two_kernel_updates_agree(pc, case, precond):
    """The fused update + direction kernel (one grid-wide barrier per iteration), the
    two-kernel form and the cluster schedule are the same method: all meet the tolerance
    and match the oracle, with nearly the same iteration count (summation order
    differs)."""
    wl = CASES[case]()
    cl, om, pairs, w, pd, wd = _setup(pc, wl)
    s = cl.assemble(pd, wd)
    rp, ci, vals_ref, b_ref = om.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), pairs, w, wl.h)
    dv_ref, _, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    pre = pc.PC_PRECOND_BLOCK if precond == "block" else pc.PC_PRECOND_JACOBI
    out = {}
    for form in (True, False, "cluster"):
        dv = torch.zeros(cl.V * 3, device="cuda")
        sched = pc.PC_SCHED_CLUSTER if form == "cluster" else pc.PC_SCHED_GRID
        info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], dv,
                                   pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED, max_iter=50000, precond=pre,
                                                 fuse=form is True, schedule=sched))
        assert st == pc.PC_OK and info.rel_res <= 2e-9
        assert H.rel_l2(_np(dv), dv_ref) <= H.DV_RTOL
        out[form] = info.iters
    assert abs(out[True] - out[False]) <= 0.12 * out[False] + 5  # see the storage test
    assert out["cluster"] <= 1.35 * out[False] + 5  # the single-reduction form, see the storage test


def _banded_spd(V, extra_rows, n_extra, seed):
    """Symmetric block pattern: a band of +-6 neighbours (13 blocks a row), plus, for the
    rows in `extra_rows`, `n_extra` couplings to rows 160 q further on (q = 1..n_extra),
    mirrored; off-diagonal blocks 0.1 x random symmetric 3x3, diagonal blocks the sum of
    the row's off-diagonal Frobenius norms + 1 times I (block diagonally dominant: SPD)."""
    rng = np.random.default_rng(seed)
    cols = [set(range(max(0, i - 6), min(V, i + 7))) for i in range(V)]
    for r in extra_rows:
        for q in range(1, n_extra + 1):
            c = r + 160 * q
            assert c < V
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
    ci = np.zeros(int(rp[-1]), np.int32)
    vals = np.zeros((int(rp[-1]), 3, 3))
    for i in range(V):
        row = sorted(cols[i])
        off = sum(np.linalg.norm(blocks[(i, j)]) for j in row if j != i)
        for n, j in enumerate(row):
            ci[rp[i] + n] = j
            vals[rp[i] + n] = (off + 1.0) * np.eye(3) if j == i else blocks[(i, j)]
    return rp, ci, vals


@pytest.mark.parametrize("shape", ["narrow", "wide", "direct"])
def test_product_stage_widths(pc, shape):
    """The solve streams the matrix in stages of 14 blocks per row (five CTAs per SM) when
    every 32-row tile fits, else of 18 (four CTAs per SM); a tile beyond that is read from
    global memory. One matrix per case, its largest tile checked here on the CPU; the
    mixed solve to 1e-10 against FP64 dense LU of the same FP32 blocks."""
    V = 32 * 40
    extra = {"narrow": 0, "wide": 3, "direct": 7}[shape]
    rp, ci, vals = _banded_spd(V, range(32, 64) if extra else [], extra, seed=17)
    tiles = rp[np.minimum(np.arange(V // 32 + 1) * 32, V)]
    tmax = int(np.diff(tiles).max())
    assert {"narrow": tmax <= 32 * 14, "wide": 32 * 14 < tmax <= 32 * 18, "direct": tmax > 32 * 18}[shape]
    wl = wk.garment(36, seed=91, stream=400)
    cl = pc.Cloth(wl)
    assert cl.V >= V
    # the context's V rows: the matrix above, then identity rows
    n_id = cl.V - V
    rp_full = np.concatenate([rp, rp[-1] + np.arange(1, n_id + 1, dtype=np.int32)])
    ci_full = np.concatenate([ci, np.arange(V, cl.V, dtype=np.int32)])
    vals_full = np.concatenate([vals, np.tile(np.eye(3), (n_id, 1, 1))])
    nnzb = int(rp_full[-1])
    cap = (nnzb + 3) // 4 * 4
    ci_pad = np.zeros(cap, np.int32)
    ci_pad[:nnzb] = ci_full
    vals_pad = np.zeros((cap, 3, 3), np.float32)
    vals_pad[:nnzb] = vals_full
    b = np.random.default_rng(3).normal(size=cl.V * 3).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (rp_full, ci_pad, vals_pad.reshape(-1), b)]
    dv = torch.zeros(cl.V * 3, device="cuda")
    info, st = pc.pc_pcg_solve(cl.ctx, t[0], t[1], nnzb, t[2], None, t[3], dv,
                               pc.solve_opts(tol=1e-10, precision=pc.PC_PREC_MIXED, max_iter=5000,
                                             storage=pc.PC_STORAGE_FULL, schedule=pc.PC_SCHED_GRID))
    assert st == pc.PC_OK and info.rel_res <= 2e-10
    # the solve's matrix is the FP32 rounding of these blocks: solve that one in FP64
    A = oracle.dense(rp, ci, vals.astype(np.float32).astype(np.float64))
    want = np.linalg.solve(A, b[: 3 * V].astype(np.float64))
    # dv is FP32: its rounding alone is up to the unit roundoff 2^-24 relative (measured
    # 2.5e-8 for these solutions); the solve's own error is about cond x 1e-10 = 2.5e-10
    assert H.rel_l2(_np(dv)[: 3 * V].astype(np.float64), want) <= 2.0 ** -24 + 1e-9
    np.testing.assert_allclose(_np(dv)[3 * V:], b[3 * V:], rtol=1e-6)
