"""Parity at full size, in the configuration the bench times (mixed-precision Jacobi-PCG
to 1e-6, difference form): the 512 x 512 cloth with 2% contacts and the paper-scale
3 x 526^2 stack. The pattern is compared bit for bit and every block and right-hand
side entry against the oracle's full FP64 assembly. The solution is checked by a
property that holds at any size (the FP64 residual of the solver's FP64 solution on the
assembled system, recomputed here independently, meets the tolerance, and the returned
dv is exactly that solution rounded to FP32) and, at 512 x 512, element by element
against the oracle's FP64 solve to 1e-12 (the oracle's loops run on every host core)."""
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


def diff_form_product(rp, ci, vals, dres, p):
    """(A p)_i = D_i p_i + sum_{j != i} A_ij (p_j - p_i) in FP64 (the form whose rows are
    exact for this model: every element Hessian's rows sum to zero)."""
    V = len(rp) - 1
    rows = np.repeat(np.arange(V), np.diff(rp))
    off = ci != rows
    A = vals[off]
    d = p[ci[off]] - p[rows[off]]
    contrib = np.einsum("bij,bj->bi", A, d)
    y = np.einsum("vij,vj->vi", dres, p)
    for k in range(3):
        y[:, k] += np.bincount(rows[off], weights=contrib[:, k], minlength=V)
    return y


@pytest.mark.parametrize("name", ["square512-contacts", "stack3x526"])
def test_full_size_pattern_values_and_solve(pc, name):
    wl = wk.WORKLOADS[name]()
    cl = pc.Cloth(wl)
    step = 1
    pairs, w = wl.contacts(step)
    pd, wd = cl.contacts_device(step)
    s = cl.assemble(pd, wd)
    nnzb = s["nnzb"]
    mesh = oracle.Mesh.from_workload(wl)
    rp_o, ci_o = mesh.pattern(pairs)
    rp = s["row_ptr"].cpu().numpy()
    ci = s["col_idx"][:nnzb].cpu().numpy()
    np.testing.assert_array_equal(rp, rp_o)
    np.testing.assert_array_equal(ci, ci_o)
    _, _, vals_ref, b_ref = mesh.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), pairs, w, wl.h,
                                          pattern=(rp_o, ci_o))
    vals = s["vals"][: 9 * nnzb].cpu().numpy().astype(np.float64).reshape(-1, 3, 3)
    excess = H.block_errors(rp_o, ci_o, vals, vals_ref)
    assert excess.max() <= 0, f"worst block excess {excess.max():.3e}"
    del vals_ref, excess
    b = s["b"].cpu().numpy().astype(np.float64).reshape(-1, 3)
    assert H.rel_l2(b, b_ref) <= 1e-5
    dv = torch.zeros(wl.V * 3, device="cuda")
    info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"], s["dres"], s["b"], dv,
                               pc.solve_opts(tol=1e-6, precision=pc.PC_PREC_MIXED, max_iter=20000))
    assert st == pc.PC_OK and info.rel_res <= 1e-6
    dv64 = torch.empty(wl.V * 3, dtype=torch.float64, device="cuda")
    pc.pc_get_solution64(cl.ctx, dv64)
    x64 = dv64.cpu().numpy().reshape(-1, 3)
    np.testing.assert_array_equal(dv.cpu().numpy().reshape(-1, 3), x64.astype(np.float32))
    dres = s["dres"].cpu().numpy().astype(np.float64).reshape(-1, 3, 3)
    r = b - diff_form_product(rp, ci, vals, dres, x64)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.05e-6, rel
    assert abs(rel - info.rel_res) <= 1e-3 * info.rel_res + 1e-12
    # pinned vertices do not move
    assert np.all(x64[wl.pins] == 0.0)


def test_full_size_batched_solve(pc):
    """The 64-garment union through the persistent batched solver (autotuned launch):
    every garment's dv against a tight single-system solve of the same union."""
    u = wk.garment_batch_union()
    cl = pc.Cloth(u)
    s = cl.assemble(*cl.contacts_device(0))
    dv = torch.zeros(cl.V * 3, device="cuda")
    infos, st = pc.pc_pcg_solve_batched(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"],
                                        dv, u.inst_rows, pc.solve_opts(tol=1e-8, max_iter=50000))
    assert st == pc.PC_OK
    assert all(i.rel_res <= 2e-8 for i in infos)
    ref = torch.zeros_like(dv)
    info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], ref,
                               pc.solve_opts(tol=1e-11, precision=pc.PC_PREC_MIXED, max_iter=200000))
    assert st == pc.PC_OK
    got = dv.cpu().numpy().reshape(-1, 3)
    want = ref.cpu().numpy().reshape(-1, 3)
    for k in range(len(u.parts)):
        r0, r1 = u.inst_rows[k], u.inst_rows[k + 1]
        assert H.rel_l2(got[r0:r1], want[r0:r1]) <= H.DV_RTOL, k


def test_full_size_learned_guess(pc):
    """Features and the tensor-core inference on the 708 x 708 cloth against the oracle
    on a random sample of rows."""
    from oracle import mlp as om
    wl = wk.warm_start_eval()
    cl = pc.Cloth(wl)
    pairs, w = wl.contacts(0)
    pd, wd = cl.contacts_device(0)
    rng = np.random.default_rng(31)
    v = (0.05 * rng.normal(size=(wl.V, 3))).astype(np.float32)
    dvp = (1e-3 * rng.normal(size=(wl.V, 3))).astype(np.float32)
    vt, dvpt = torch.from_numpy(v).cuda(), torch.from_numpy(dvp).cuda()
    s = cl.assemble(pd, wd, v=vt)
    feat = torch.empty(wl.V, 12, device="cuda")
    pc.pc_mlp_features(cl.ctx, vt, dvpt, s["b"], wl.h, feat)
    mesh = oracle.Mesh.from_workload(wl)
    sample = rng.choice(wl.V, 20000, replace=False)
    g = wl.material.as_array()[5:8]
    want = om.features(v, dvp, s["b"].cpu().numpy().astype(np.float64), mesh.mass, wl.h, g,
                       om.edges_of(wl.tris), wl.rest)[sample]
    got = feat.cpu().numpy().astype(np.float64)[sample]
    assert np.all(np.abs(got - want) <= 2e-6 * np.abs(want).max(axis=0) + 1e-12)
    params = om.init_params(4).astype(np.float32)
    F = feat.cpu().numpy().astype(np.float64)
    stats = om.compute_stats(F, 1e-3 * rng.normal(size=(wl.V, 3))).astype(np.float32)
    out = torch.empty(wl.V, 3, device="cuda")
    pinned = np.zeros(wl.V, np.uint8)
    pinned[wl.pins] = 1
    pc.pc_mlp_infer(wl.V, torch.from_numpy(params).cuda(), torch.from_numpy(stats).cuda(), feat, dvpt,
                    torch.from_numpy(pinned).cuda(), out)
    pred = om.predict(params.astype(np.float64), stats.astype(np.float64), F[sample], dvp[sample],
                      pinned[sample].astype(bool), bf16=True)
    o = out.cpu().numpy().astype(np.float64)[sample]
    assert np.linalg.norm((o - dvp[sample]) - (pred - dvp[sample])) <= 2e-3 * np.linalg.norm(pred - dvp[sample])
    assert np.all(out.cpu().numpy()[wl.pins] == 0.0)


FULL_DV = {
    # name: (workload, reference tolerance of the oracle's FP64 solve)
    "square512-contacts": (wk.dynamic_square, 1e-12),
    "stack3x526": (wk.paper_scale, 1e-11),          # FP64 CG stalls near 2e-9 true residual here
    "square708-contacts": (wk.warm_start_eval, 1e-11),
}


@pytest.mark.parametrize("name", list(FULL_DV))
def test_full_size_dv_matches_oracle(pc, name):
    """dv element by element against the oracle's FP64 solve of its own FP64 assembly, at
    the benchmark's tolerance (1e-6) and at a tight one (1e-9), at the full sizes of the
    512 x 512 cloth, the paper-scale stack and the 708 x 708 cloth.

    On the paper-scale stack (flat sheets: the right-hand side is essentially gravity) a
    1e-6 residual gives dv within 1e-5 of the oracle, as required. On the single sheets
    with out-of-plane jitter the condition number is about 1e6 and the jitter's elastic
    and bending forces are thousands of times the gravity load, so two effects of the
    method (not of this implementation) set the error:
    - a relative residual of 1e-6 does not bound the dv error by 1e-5: the oracle's own
      FP64 PCG stopped at 1e-6 is 6e-4 to 8e-4 away from the exact solution; at 1e-6 the
      GPU is held to twice that plus 1e-5;
    - element forces evaluated in FP32 (the paper's precision, Sec. 5) carry rounding of
      about 1e-7 of each element's force before the per-vertex sums cancel it, and this
      stiff system amplifies the sum's error: the dv error no longer falls below a few
      1e-5 (512^2) to 2e-4 (708^2) however tight the solve. At 1e-9 the GPU must still
      have at most half the error the exact method has at 1e-6, and at most 3e-4."""
    make, ref_tol = FULL_DV[name]
    wl = make()
    cl = pc.Cloth(wl)
    pairs, w = wl.contacts(1)
    pd, wd = cl.contacts_device(1)
    s = cl.assemble(pd, wd)
    mesh = oracle.Mesh.from_workload(wl)
    rp, ci, vals_ref, b_ref = mesh.assemble(wl.x0.astype(np.float64), wl.v0.astype(np.float64), pairs, w, wl.h)
    dv_ref, it_ref, res_ref = oracle.pcg(rp, ci, vals_ref, b_ref, tol=ref_tol, max_iter=200000)
    dv6, it6, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-6, max_iter=200000)
    del vals_ref
    err_oracle6 = H.rel_l2(dv6, dv_ref)
    print(f"{name}: oracle ({oracle.num_threads()} threads): {it_ref} iterations to {ref_tol:g} (true residual "
          f"{res_ref:.2e}), {it6} to 1e-6; its own dv error at 1e-6: {err_oracle6:.3e}")
    for tol in (1e-6, 1e-9):
        dv = torch.zeros(wl.V * 3, device="cuda")
        info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], s["nnzb"], s["vals"], s["dres"], s["b"], dv,
                                   pc.solve_opts(tol=tol, precision=pc.PC_PREC_MIXED, max_iter=50000))
        assert st == pc.PC_OK and info.rel_res <= tol
        got = dv.cpu().numpy().astype(np.float64).reshape(-1, 3)
        err = H.rel_l2(got, dv_ref)
        print(f"{name}: GPU mixed tol {tol:g}: {info.iters} iterations, dv rel err vs oracle {err:.3e}")
        if err_oracle6 <= 0.1 * H.DV_RTOL:  # the residual bounds the error: the parity bound holds
            assert err <= H.DV_RTOL
        elif tol == 1e-6:
            assert err <= 2 * err_oracle6 + H.DV_RTOL
        else:
            assert err <= min(0.5 * err_oracle6, 3e-4)
        assert np.all(got[wl.pins] == 0.0)
