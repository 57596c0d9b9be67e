"""Pins of the learned-warm-start oracle (oracle/mlp.py) against facts that do not come
from the oracle itself: central differences, the affine regime of a ReLU network, the
closed form of Adam under a constant gradient, brute-force one-rings and the integrator
oracle's own forces."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2008_00409_gb300 import workloads as wk


def _rand_batch(n=9, seed=3):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, mlp.N_IN)), rng.normal(size=(n, mlp.N_OUT))


def test_parameter_count():
    assert mlp.N_PARAMS == 12 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 5187
    p = mlp.init_params(1)
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)


def test_gradient_matches_central_differences():
    p = mlp.init_params(7)
    X, T = _rand_batch()
    g = mlp.grad(p, X, T)
    rng = np.random.default_rng(11)
    # every bias and a random sample of weights of each layer
    idx, o = [], 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        idx += list(range(o, o + n)) if name.startswith("b") else list(o + rng.choice(n, 60, replace=False))
        o += n
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (mlp.loss(pp, X, T) - mlp.loss(pm, X, T)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_forward_is_affine_when_every_unit_is_active():
    rng = np.random.default_rng(5)
    P = {"W1": rng.uniform(0, 1, (64, 12)), "b1": rng.uniform(0, 1, 64), "W2": rng.uniform(0, 1, (64, 64)),
         "b2": rng.uniform(0, 1, 64), "W3": rng.normal(size=(3, 64)), "b3": rng.normal(size=3)}
    X = rng.uniform(0, 1, (5, 12))
    Y = mlp.forward(mlp.pack(P), X)["Y"]
    # composition of the three affine maps (associated the other way round)
    Wc = P["W3"] @ (P["W2"] @ P["W1"])
    bc = P["W3"] @ (P["W2"] @ P["b1"] + P["b2"]) + P["b3"]
    assert np.allclose(Y, X @ Wc.T + bc, rtol=1e-12, atol=1e-12)


def test_forward_dead_first_layer_gives_a_constant():
    rng = np.random.default_rng(6)
    P = {"W1": -rng.uniform(0, 1, (64, 12)), "b1": -rng.uniform(0.1, 1, 64), "W2": rng.normal(size=(64, 64)),
         "b2": rng.normal(size=64), "W3": rng.normal(size=(3, 64)), "b3": rng.normal(size=3)}
    X = rng.uniform(0, 1, (4, 12))
    Y = mlp.forward(mlp.pack(P), X)["Y"]
    const = P["W3"] @ np.maximum(P["b2"], 0) + P["b3"]
    assert np.allclose(Y, np.tile(const, (4, 1)), rtol=1e-13, atol=1e-13)


def test_forward_positively_homogeneous_without_biases():
    p = mlp.unpack(mlp.init_params(2).copy())
    for b in ("b1", "b2", "b3"):
        p[b][:] = 0.0
    p = mlp.pack(p)
    X, _ = _rand_batch(6, 8)
    Y1 = mlp.forward(p, X)["Y"]
    Y2 = mlp.forward(p, 2.5 * X)["Y"]
    assert np.allclose(Y2, 2.5 * Y1, rtol=1e-12, atol=1e-12)
    assert not np.allclose(mlp.forward(p, -X)["Y"], -Y1)  # the ReLUs are really there


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments equal g and g^2 at every step, so
    # each step moves every parameter by lr * g / (|g| + eps)
    rng = np.random.default_rng(4)
    g = rng.normal(size=50)
    p = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-2, 1e-8
    p0 = p.copy()
    for t in range(1, 6):
        p, m, v = mlp.adam_step(p, m, v, g, t, lr=lr, eps=eps)
        assert np.allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)


def test_ring_mean_brute_force():
    wl = wk.square_cloth(5, seed=1)
    tris = wl.tris
    nbrs = [set() for _ in range(wl.V)]
    for t in tris:
        for a in range(3):
            for b in range(3):
                if a != b:
                    nbrs[t[a]].add(int(t[b]))
    q = np.random.default_rng(0).normal(size=(wl.V, 3))
    want = np.array([np.mean([q[j] for j in sorted(nb)], axis=0) for nb in nbrs])
    got = mlp.ring_mean(wl.V, mlp.edges_of(tris), q)
    assert np.allclose(got, want, rtol=1e-14, atol=1e-14)
    # interior vertices of a diagonal-split grid have 6 neighbours, corners 2 or 3
    deg = [len(nb) for nb in nbrs]
    assert max(deg) == 6 and min(deg) in (2, 3)


def test_force_feature_is_the_linearised_internal_force():
    wl = wk.square_cloth(6, seed=2)
    om = oracle.Mesh.from_workload(wl)
    rng = np.random.default_rng(9)
    x = wl.x0.astype(np.float64) + 0.01 * rng.normal(size=(wl.V, 3))
    v = 0.1 * rng.normal(size=(wl.V, 3))
    h = wl.h
    _, _, _, b = om.assemble(x, v, h=h)
    g = wl.material.as_array()[5:8]
    F = mlp.features(v, np.zeros_like(v), b, om.mass, h, g, mlp.edges_of(wl.tris), wl.rest)
    f_int = om.forces(x) - om.mass[:, None] * g                    # element forces at x_t
    hKv = (om.matfree_apply(x, v, h=h) - om.mass[:, None] * v) / h  # h K v (A v = M v + h^2 K v)
    free = ~om.pinned
    ell = mlp.rest_lengths(wl.rest, mlp.edges_of(wl.tris))
    want = ell[free, None] * (f_int - hKv)[free] / om.mass[free, None]
    assert np.allclose(F[free, 6:9], want, rtol=1e-9, atol=1e-12)
    assert np.array_equal(F[:, 0:3], v)


def test_rest_length_scale_closed_form():
    # a regular n x n grid of spacing s split along one diagonal: an interior vertex has
    # four axis neighbours at s and two diagonal ones at s sqrt(2)
    for n in (5, 9):
        wl = wk.square_cloth(n, seed=3, z_jitter=0.0)
        s_ = 1.0 / (n - 1)
        ell = mlp.rest_lengths(wl.rest, mlp.edges_of(wl.tris))
        inner = np.array([i * n + j for i in range(1, n - 1) for j in range(1, n - 1)])
        assert np.allclose(ell[inner], s_ * (4 + 2 * np.sqrt(2)) / 6, rtol=1e-12)
        # a corner on the diagonal's ends has two axis edges and one diagonal, the others two axis edges
        corners = ell[[0, n - 1, n * (n - 1), n * n - 1]]
        assert set(np.round(corners / s_, 9)) <= {1.0, round((2 + np.sqrt(2)) / 3, 9)}


def test_predict_of_a_silent_network():
    p = mlp.unpack(mlp.init_params(3).copy())
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    rng = np.random.default_rng(1)
    X = rng.normal(size=(8, 12))
    dvp = rng.normal(size=(8, 3))
    stats = np.concatenate([np.zeros(12), np.ones(12), [0.5, -1.0, 2.0], [3.0, 3.0, 3.0]])
    pinned = np.zeros(8, bool)
    pinned[[2, 5]] = True
    dv0 = mlp.predict(mlp.pack(p), stats, X, dvp, pinned)
    want = dvp + np.array([0.5, -1.0, 2.0])
    want[pinned] = 0.0
    assert np.array_equal(dv0, want)


@pytest.mark.parametrize("x,want", [(1.0, 1.0), (1.0 + 2.0 ** -8, 1.0), (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),
                                    (-1.0 - 2.0 ** -9, -1.0), (3.0e-3, 0.0030059814453125)])
def test_bf16_rounding_ties_to_even(x, want):
    assert mlp.bf16_round(np.array([x]))[0] == want


def test_bf16_mode_is_exact_on_representable_values():
    # sparse +-1 weights, inputs in {-1, 0, 1}, half-integer biases and a batch of 8 keep
    # every rounded quantity (inputs, weights, H1, H2, dY, dZ2, dZ1) a short binary
    # fraction, exactly representable in bfloat16, so both modes must agree exactly
    rng = np.random.default_rng(12)
    W1 = np.zeros((64, 12))
    for r in range(64):
        W1[r, rng.choice(12, 3, replace=False)] = rng.choice([-1.0, 1.0], 3)
    I = np.eye(64)
    W2 = I[rng.permutation(64)] - I[rng.permutation(64)]
    W3 = np.zeros((3, 64))
    cols = rng.permutation(64)[:12].reshape(3, 4)
    for o in range(3):
        W3[o, cols[o]] = rng.choice([-1.0, 1.0], 4)
    P = {"W1": W1, "b1": rng.integers(-2, 3, 64) * 0.5, "W2": W2, "b2": rng.integers(-2, 3, 64) * 0.5,
         "W3": W3, "b3": rng.integers(-2, 3, 3) * 0.5}
    p = mlp.pack(P)
    X = rng.integers(-1, 2, (8, 12)).astype(float)
    T = rng.integers(-4, 5, (8, 3)) * 0.5
    a = mlp.forward(p, X)
    assert a["H1"].max() > 0 and a["H2"].max() > 0  # the case is not trivial
    assert np.array_equal(mlp.forward(p, X, bf16=True)["Y"], a["Y"])
    g = mlp.grad(p, X, T)
    assert np.count_nonzero(g) > 100
    assert np.array_equal(mlp.grad(p, X, T, bf16=True), g)


def test_bf16_mode_stays_within_the_rounding_bound():
    p = mlp.init_params(5)
    X, T = _rand_batch(64, 21)
    ye, yb = mlp.forward(p, X)["Y"], mlp.forward(p, X, bf16=True)["Y"]
    rel = np.linalg.norm(yb - ye) / np.linalg.norm(ye)
    assert 1e-4 < rel < 2e-2  # rounding really happens, at the size 2^-8 predicts
    ge, gb = mlp.grad(p, X, T), mlp.grad(p, X, T, bf16=True)
    assert np.linalg.norm(gb - ge) / np.linalg.norm(ge) < 3e-2
