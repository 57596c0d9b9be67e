"""Checkpoint and resume: a run split by a save and a load into fresh contexts steps
exactly like the uninterrupted run (previous-step guess included); the Adam state
round-trips; the per-step log writes its fields."""
import json

import numpy as np
import pytest
import torch

from tests import _helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    from paper_2008_00409_gb300 import build
    build.build()
    from paper_2008_00409_gb300 import pcloth
    return pcloth


def _steps(pc, cl, wl, k0, k1, log=None):
    for k in range(k0, k1):
        pd, wd = cl.contacts_device(k)
        info, st = cl.step(pd, wd, tol=1e-8, precision=pc.PC_PREC_MIXED, warm_start=pc.PC_WARM_PREV)
        assert st == pc.PC_OK
        if log is not None:
            log.record(k, info, st)


def test_resume_is_bit_identical(pc, tmp_path):
    from paper_2008_00409_gb300 import checkpoint
    wl = H.small_contact_cloth()
    ref = pc.Cloth(wl)
    _steps(pc, ref, wl, 0, 4)
    a = pc.Cloth(wl)
    _steps(pc, a, wl, 0, 2)
    path = tmp_path / "run.npz"
    checkpoint.save(path, a, 2)
    a.close()
    b = pc.Cloth(wl)
    step, params, stats = checkpoint.load(path, b)
    assert step == 2 and params is None and stats is None
    _steps(pc, b, wl, step, 4)
    assert torch.equal(b.x, ref.x) and torch.equal(b.v, ref.v)
    # without the previous dv the resumed run differs (the guess matters)
    c = pc.Cloth(wl)
    checkpoint.load(path, c)
    pc.pc_set_prev_dv(c.ctx, None)
    _steps(pc, c, wl, 2, 4)
    assert not torch.equal(c.x, ref.x)


def test_adam_state_round_trip_and_log(pc, tmp_path):
    from paper_2008_00409_gb300 import checkpoint
    from oracle import mlp as om
    rng = np.random.default_rng(2)
    n = 4096
    feat = torch.from_numpy(rng.normal(size=(n, pc.PC_MLP_IN)).astype(np.float32)).cuda()
    target = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).cuda()
    params0 = torch.from_numpy(om.init_params(5).astype(np.float32)).cuda()
    stats = torch.zeros(pc.PC_MLP_NSTATS, device="cuda")
    m1 = pc.pc_mlp_create()
    pc.pc_mlp_stats(m1, n, feat, target, stats)
    opts = pc.pc_adam_opts()
    opts.lr, opts.beta1, opts.beta2, opts.eps = 1e-3, 0.9, 0.999, 1e-8
    pa = params0.clone()
    for _ in range(3):
        pc.pc_mlp_train_step(m1, n, None, pa, stats, feat, target, opts)
    wl = H.small_contact_cloth()
    cl = pc.Cloth(wl)
    path = tmp_path / "train.npz"
    checkpoint.save(path, cl, 0, mlp=m1, params=pa, stats=stats)
    m2 = pc.pc_mlp_create()
    _, pb, sb = checkpoint.load(path, pc.Cloth(wl), mlp=m2)
    assert torch.equal(pb, pa) and torch.equal(sb, stats)
    pc.pc_mlp_train_step(m1, n, None, pa, stats, feat, target, opts)
    pc.pc_mlp_train_step(m2, n, None, pb, sb, feat, target, opts)
    assert torch.equal(pa, pb)
    pc.pc_mlp_destroy(m1)
    pc.pc_mlp_destroy(m2)
    # per-step log
    logp = tmp_path / "steps.jsonl"
    pc.pc_set_profiling(cl.ctx, True)
    log = checkpoint.StepLog(logp, cl)
    _steps(pc, cl, wl, 0, 2, log)
    lines = [json.loads(s) for s in open(logp)]
    assert [d["step"] for d in lines] == [0, 1]
    for d in lines:
        assert d["status"] == 0 and d["iters"] > 0 and d["rel_res"] <= 1e-8 and d["nnzb"] > 0
        # this small cloth solves on the cluster schedule by default
        assert d["assembly_ms"] > 0 and d["cluster_us_per_iter"] > 0
