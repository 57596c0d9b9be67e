"""Learned warm start on the GPU (features, statistics, BF16 tensor-core inference and
back-propagation, Adam, training, the warm-started step) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as om
from paper_2008_00409_gb300 import workloads as wk
from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2008_00409_gb300 import build
    build.build()
    from paper_2008_00409_gb300 import pcloth
    return pcloth


def _d(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _params(seed):
    p = om.unpack(om.init_params(seed).copy())
    rng = np.random.default_rng(seed + 100)
    for b in ("b1", "b2", "b3"):
        p[b][:] = 0.1 * rng.normal(size=p[b].shape)
    return om.pack(p).astype(np.float32).astype(np.float64)  # FP32-representable


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    scale = np.array([0.5, 0.5, 0.5, 1e-2, 1e-2, 1e-2, 30.0, 30.0, 30.0, 1e-2, 1e-2, 1e-2])
    X = (rng.normal(size=(n, 12)) * scale + 0.1 * scale).astype(np.float32)
    dv = (X[:, 3:6] + 3e-3 * rng.normal(size=(n, 3))).astype(np.float32)
    return X, dv


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_features_match_oracle(pc):
    wl = H.small_contact_cloth()
    cl = pc.Cloth(wl)
    pairs, w = cl.contacts_device(0)
    rng = np.random.default_rng(1)
    v = (0.05 * rng.normal(size=(wl.V, 3))).astype(np.float32)
    dvp = (1e-3 * rng.normal(size=(wl.V, 3))).astype(np.float32)
    vt, dvpt = _d(v), _d(dvp)
    s = cl.assemble(pairs, w, v=vt)
    feat = torch.empty(wl.V, 12, device="cuda")
    pc.pc_mlp_features(cl.ctx, vt, dvpt, s["b"], wl.h, feat)
    mesh = oracle.Mesh.from_workload(wl)
    g = wl.material.as_array()[5:8]
    want = om.features(v, dvp, _np(s["b"]), mesh.mass, wl.h, g, om.edges_of(wl.tris), wl.rest)
    got = _np(feat)
    scale = np.abs(want).max(axis=0)
    assert np.all(np.abs(got - want) <= 2e-6 * scale + 1e-12)
    assert np.array_equal(got[:, 0:3], v) and np.array_equal(got[:, 3:6], dvp)


def test_stats_match_oracle(pc):
    X, dv = _rows(70001, 2)
    m = pc.pc_mlp_create()
    stats = torch.empty(30, device="cuda")
    pc.pc_mlp_stats(m, len(X), _d(X), _d(dv), stats)
    pc.pc_mlp_destroy(m)
    want = om.compute_stats(X.astype(np.float64), dv.astype(np.float64) - X[:, 3:6].astype(np.float64))
    assert np.allclose(_np(stats), want, rtol=2e-6, atol=0)


@pytest.mark.parametrize("n", [1, 16, 129, 1037])
def test_infer_matches_oracle(pc, n):
    X, dv = _rows(max(n, 64), 3)
    X = X[:n]
    params = _params(3)
    stats = om.compute_stats(X.astype(np.float64), dv[:n] - X[:, 3:6]).astype(np.float32).astype(np.float64)
    fixed = np.zeros(n, np.uint8)
    fixed[::7] = 1
    out = torch.full((n, 3), float("nan"), device="cuda")
    pc.pc_mlp_infer(n, _d(params), _d(stats), _d(X), _d(X[:, 3:6]), _d(fixed, np.uint8), out)
    got = _np(out)
    want_bf = om.predict(params, stats, X, X[:, 3:6], fixed.astype(bool), bf16=True)
    want_ex = om.predict(params, stats, X, X[:, 3:6], fixed.astype(bool))
    assert np.all(got[fixed == 1] == 0.0)
    free = fixed == 0
    dg, db, de = (a[free] - X[free, 3:6] for a in (got, want_bf, want_ex))
    assert _rel(dg, db) <= 2e-3
    assert _rel(dg, de) <= 3e-2


def test_grad_and_loss_match_oracle(pc):
    n = 3001
    X, dv = _rows(n, 4)
    params = _params(5)
    stats = om.compute_stats(X.astype(np.float64), dv - X[:, 3:6]).astype(np.float32).astype(np.float64)
    m = pc.pc_mlp_create()
    grad = torch.empty(om.N_PARAMS, device="cuda")
    loss = pc.pc_mlp_grad(m, n, None, _d(params), _d(stats), _d(X), _d(dv), grad)
    Xn = om.normalize_inputs(X, stats)
    Tn = om.normalize_targets(dv.astype(np.float64) - X[:, 3:6], stats)
    g_bf = om.grad(params, Xn, Tn, bf16=True)
    g_ex = om.grad(params, Xn, Tn)
    got = _np(grad)
    assert _rel(got, g_bf) <= 5e-3
    assert _rel(got, g_ex) <= 5e-2
    P_got, P_bf = om.unpack(got), om.unpack(g_bf)
    for name, _ in om.SHAPES:
        assert _rel(P_got[name], P_bf[name]) <= 1e-2, name
    y_bf = om.forward(params, Xn, bf16=True)["Y"]
    assert abs(loss - 0.5 * np.sum((y_bf - Tn) ** 2) / n) <= 1e-3 * loss
    # the same rows gathered from a larger array through a row list
    Xb, dvb = _rows(9000, 6)
    sel = np.random.default_rng(7).choice(9000, n, replace=False)
    Xb[sel], dvb[sel] = X, dv
    grad2 = torch.empty_like(grad)
    loss2 = pc.pc_mlp_grad(m, n, _d(sel, np.int32), _d(params), _d(stats), _d(Xb), _d(dvb), grad2)
    pc.pc_mlp_destroy(m)
    assert _rel(_np(grad2), g_bf) <= 5e-3 and abs(loss2 - loss) <= 1e-6 * loss


def test_adam_matches_oracle(pc):
    rng = np.random.default_rng(8)
    p0 = rng.normal(size=om.N_PARAMS).astype(np.float32)
    grads = [rng.normal(size=om.N_PARAMS).astype(np.float32) for _ in range(3)]
    m = pc.pc_mlp_create()
    p = _d(p0)
    opts = pc.adam_opts(lr=1e-2)
    pm, mm, vm = p0.astype(np.float64), np.zeros(om.N_PARAMS), np.zeros(om.N_PARAMS)
    for t, g in enumerate(grads, start=1):
        pc.pc_mlp_adam_apply(m, p, _d(g), opts)
        pm, mm, vm = om.adam_step(pm, mm, vm, g.astype(np.float64), t, lr=1e-2)
    pc.pc_mlp_destroy(m)
    assert _rel(_np(p) - p0, pm - p0) <= 1e-5


def test_training_learns_a_teacher_deterministically(pc):
    from paper_2008_00409_gb300 import warmstart as ws
    n = 40000
    rng = np.random.default_rng(9)
    X = rng.normal(size=(n, 12)).astype(np.float32)
    teacher = _params(11)
    dv = (X[:, 3:6] + om.forward(teacher, X)["Y"]).astype(np.float32)
    feat, dvt = _d(X), _d(dv)
    p_a, stats, losses = ws.train(feat, dvt, steps=400, batch=4096, lr=3e-3, seed=1, log_every=399)
    p_b, _, _ = ws.train(feat, dvt, steps=400, batch=4096, lr=3e-3, seed=1)
    assert torch.equal(p_a, p_b)  # fixed reduction order: bit-identical runs
    first = ws.dataset_loss(ws.init_params(1), stats, feat, dvt)
    last = ws.dataset_loss(p_a, stats, feat, dvt)
    assert last < 0.1 * first, (first, last)


def test_warm_start_steps(pc):
    from paper_2008_00409_gb300 import warmstart as ws
    train_wl = [wk.training_cloth(24, seed=500 + k, steps=30) for k in range(3)]
    feat, dv = ws.collect(train_wl, tol=1e-7)
    params, stats, _ = ws.train(feat, dv, steps=300, batch=8192, lr=3e-3, seed=2)
    eval_wl = wk.training_cloth(24, seed=777, steps=12)
    res = ws.evaluate(eval_wl, params, stats, steps=12, tol=1e-7)
    mlp = res[pc.PC_WARM_MLP]
    for mode, rec in res.items():
        assert max(rec["rel_res"]) <= 1e-7, mode
    en = np.array(mlp["guess_energy"])
    # the solve starts from the A-norm-optimal combination of the previous and learned
    # guesses: its CG energy is at most that of the zero, previous and learned guesses (the
    # previous guess is not a candidate on the first step)
    for k, used in enumerate(mlp["guess"]):
        cand = en[k] if k > 0 else np.array([en[k, 0], np.inf, en[k, 2]])
        e_used = mlp["combo_energy"][k]
        assert e_used <= cand.min() + 1e-9 * np.abs(cand[np.isfinite(cand)]).max(), (k, e_used, cand)
        assert used in (pc.PC_WARM_COMBINED, pc.PC_WARM_ZERO, pc.PC_WARM_PREV, pc.PC_WARM_MLP)
        if used == pc.PC_WARM_COMBINED:
            assert np.all(np.isfinite(mlp["guess_coef"][k]))
            if k == 0:
                assert mlp["guess_coef"][k][0] == 0.0
    assert mlp["guess"].count(pc.PC_WARM_COMBINED) >= len(mlp["guess"]) // 2
    # the trained network's guess has a smaller A-norm error than the zero guess
    assert np.mean(en[2:, 2] < 0.0) >= 0.8
    # and the learned warm start needs fewer PCG iterations than the zero guess in total
    assert sum(mlp["iters"]) < sum(res[pc.PC_WARM_ZERO]["iters"])
    # warm-started steps still follow the oracle
    cl = pc.Cloth(eval_wl)
    pc.pc_set_warm_mlp(cl.ctx, params, stats)
    mesh = oracle.Mesh.from_workload(eval_wl)
    dvo = torch.empty(eval_wl.V, 3, device="cuda")
    for t in range(4):
        pairs, w = eval_wl.contacts(t)
        pd, wd = cl.contacts_device(t)
        x0, v0 = _np(cl.x), _np(cl.v)
        cl.step(pd, wd, tol=1e-9, precision=pc.PC_PREC_MIXED, warm_start=pc.PC_WARM_MLP, dv_out=dvo, max_iter=50000)
        dv_ref, _, _, _ = mesh.step(x0, v0, pairs, w, h=eval_wl.h, tol=1e-12)
        err = H.rel_l2(_np(dvo), dv_ref)
        print(f"warm-started step {t}: dv rel err {err:.3e}")
        assert err <= H.DV_RTOL, t
    pc.pc_set_warm_mlp(cl.ctx, None, None)
