"""One-sided thickness contact with pairs from the GPU proximity query, against the
oracle through the C ABI.

The query's pairs and weights are compared bit for bit (both sides decide regions and
d^2 < delta^2 in FP32 with the same operations); assembly with the thickness model
within the per-block tolerance; solves and steps within 1e-5 of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import proximity as px
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


def _crumpled(n=24, seed=3):
    """A square cloth folded onto itself along x = 0.5 (the folded half a third of a
    spacing above the other, shifted and jittered in the plane, with vertical noise): the
    query meets every closest-point region (vertex, edge, face)."""
    wl = wk.square_cloth(n, seed=seed, contact_frac=0.0, steps=1, name=f"crumpled{n}")
    rng = np.random.default_rng(seed)
    spacing = 1.0 / (n - 1)
    x = wl.rest.astype(np.float64).copy()
    top = x[:, 0] > 0.5
    x[top, 0] = 1.0 - x[top, 0] + 0.37 * spacing
    x[top, 1] += 0.21 * spacing
    x[top, 2] += spacing / 3
    x[:, :2] += 0.15 * spacing * rng.normal(size=(wl.V, 2))
    x[:, 2] += 0.1 * spacing * rng.normal(size=wl.V)
    wl.x0 = x.astype(np.float32)
    return wl, 0.8 * spacing


def _query_both(pc, cl, wl, delta, x=None):
    xg = cl.x if x is None else x
    pd, wd = cl.proximity(delta, xg)
    got_p = np.zeros((0, 4), np.int32) if pd is None else _np(pd)
    got_w = np.zeros((0, 3), np.float32) if wd is None else _np(wd)
    want_p, want_w = px.query(_np(xg), wl.tris, delta)
    return got_p, got_w, want_p, want_w


@pytest.mark.parametrize("case", ["stack3x21", "crumpled24"])
def test_query_bit_exact(pc, case):
    if case == "stack3x21":
        wl = wk.proximity_stack(21, 3, steps=3)
        delta = wl.material.contact_thickness
    else:
        wl, delta = _crumpled()
        wl.contact_kind, wl.contact_frac = "proximity", 40.0
    cl = pc.Cloth(wl)
    got_p, got_w, want_p, want_w = _query_both(pc, cl, wl, delta)
    assert len(want_p) > 0
    np.testing.assert_array_equal(got_p, want_p)
    np.testing.assert_array_equal(got_w, want_w)
    if case == "crumpled24":
        # every region of the closest point occurs: vertex (one weight 1), edge (one
        # weight 0), face (all weights positive)
        ones = np.any(want_w == 1.0, axis=1)
        zeros = np.any(want_w == 0.0, axis=1) & ~ones
        face = np.all(want_w > 0.0, axis=1)
        assert ones.any() and zeros.any() and face.any()


def test_query_capacity_and_arguments(pc):
    wl = wk.proximity_stack(21, 3, steps=3)
    cl = pc.Cloth(wl)
    d = wl.material.contact_thickness
    big_p = torch.zeros((cl.max_contacts, 4), dtype=torch.int32, device="cuda")
    big_w = torch.zeros((cl.max_contacts, 3), device="cuda")
    n = pc.pc_proximity_query(cl.ctx, cl.x, d, big_p, big_w)
    assert n > 1
    with pytest.raises(pc.PcError) as e:
        pc.pc_proximity_query(cl.ctx, cl.x, d, big_p[: n - 1], big_w[: n - 1])
    assert e.value.status == pc.PC_ERR_CAPACITY and e.value.required == n
    with pytest.raises(pc.PcError) as e:
        pc.pc_proximity_query(cl.ctx, cl.x, 0.0, big_p, big_w)
    assert e.value.status == pc.PC_ERR_ARG
    # a non-finite position has no cell: reported, nothing faults
    bad = cl.x.clone()
    bad[0, 0] = float("nan")
    with pytest.raises(pc.PcError) as e:
        pc.pc_proximity_query(cl.ctx, bad, d, big_p, big_w)
    assert e.value.status == pc.PC_ERR_ARG


def test_thickness_assembly_and_solve_match_oracle(pc):
    wl = wk.proximity_stack(21, 3, steps=3)
    cl = pc.Cloth(wl)
    om = oracle.Mesh.from_workload(wl)
    pd, wd = cl.proximity()
    pairs, w = _np(pd), _np(wd)
    rng = np.random.default_rng(8)
    v = (0.02 * rng.normal(size=(wl.V, 3))).astype(np.float32)
    vt = torch.from_numpy(v).cuda()
    s = cl.assemble(pd, wd, v=vt)
    nnzb = s["nnzb"]
    rp, ci, vals_ref, b_ref = om.assemble(wl.x0.astype(np.float64), v.astype(np.float64), pairs,
                                          w.astype(np.float64), wl.h)
    np.testing.assert_array_equal(_np(s["row_ptr"]), rp)
    np.testing.assert_array_equal(_np(s["col_idx"])[:nnzb], ci)
    vals = _np(s["vals"])[: 9 * nnzb].astype(np.float64).reshape(-1, 3, 3)
    assert H.block_errors(rp, ci, vals, vals_ref).max() <= 0
    assert H.rel_l2(_np(s["b"]).reshape(-1, 3), b_ref) <= 1e-5
    # the thickness forces act: b differs from the hold-penalty system's
    m0 = om.material.copy()
    m0[10] = 0.0
    _, _, _, b_hold = oracle.Mesh(wl.rest, wl.tris, m0, wl.pins).assemble(
        wl.x0.astype(np.float64), v.astype(np.float64), pairs, w.astype(np.float64), wl.h)
    assert H.rel_l2(b_hold, b_ref) > 1e-3
    dv_ref, _, _ = oracle.pcg(rp, ci, vals_ref, b_ref, tol=1e-12)
    dv = torch.zeros(cl.V * 3, device="cuda")
    info, st = pc.pc_pcg_solve(cl.ctx, s["row_ptr"], s["col_idx"], nnzb, s["vals"], s["dres"], s["b"], dv,
                               pc.solve_opts(tol=1e-9, precision=pc.PC_PREC_MIXED, max_iter=50000))
    assert st == pc.PC_OK and H.rel_l2(_np(dv), dv_ref) <= H.DV_RTOL


def test_proximity_steps_follow_the_oracle(pc):
    """Three steps, each with the query at the step's positions, against the oracle's
    query and step at the same FP32 state."""
    wl = wk.proximity_stack(21, 3, steps=3)
    cl = pc.Cloth(wl)
    om = oracle.Mesh.from_workload(wl)
    rings = px.one_rings(wl.V, wl.tris)
    for step in range(3):
        x = _np(cl.x).astype(np.float64)
        v = _np(cl.v).astype(np.float64)
        pairs, w = px.query(_np(cl.x), wl.tris, wl.material.contact_thickness, rings=rings)
        pd, wd = cl.proximity()
        np.testing.assert_array_equal(_np(pd), pairs)
        info, st = cl.step(pd, wd, tol=1e-9, precision=pc.PC_PREC_MIXED)
        assert st == pc.PC_OK
        dv_ref, _, _, _ = om.step(x, v, pairs, w.astype(np.float64), h=wl.h, tol=1e-12)
        dv = _np(cl.v).astype(np.float64) - v
        err = H.rel_l2(dv, dv_ref)
        print(f"proximity step {step}: dv rel err {err:.3e}")
        assert err <= H.DV_RTOL, step


def test_query_full_size_sampled(pc):
    """The paper-scale stack with the thickness model: the GPU's pairs of a random sample
    of vertices against the oracle's brute force for those vertices."""
    wl = wk.proximity_stack()
    cl = pc.Cloth(wl)
    pd, wd = cl.proximity()
    pairs, w = _np(pd), _np(wd)
    assert len(pairs) > wl.V  # every vertex faces the next sheet
    rng = np.random.default_rng(9)
    sample = np.sort(rng.choice(wl.V, 150, replace=False))
    want_p, want_w = px.query(wl.x0, wl.tris, wl.material.contact_thickness, vertices=sample)
    sel = np.isin(pairs[:, 0], sample)
    np.testing.assert_array_equal(pairs[sel], want_p)
    np.testing.assert_array_equal(w[sel], want_w)
