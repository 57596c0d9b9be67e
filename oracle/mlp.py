"""FP64 reference of the learned warm start: features, the per-vertex MLP, its loss,
gradient and Adam update.

TEST INFRASTRUCTURE ONLY: imported by tests/ and never by the CUDA library, which shares
no code with this module.

The paper has no learned component. The warm start built on its integrator predicts
the initial guess of the Eq. 3 solve from per-vertex quantities available before the
solve:

* features (12 per vertex): the velocity v_i; the previous step's solution dv_prev_i;
  the internal force per unit mass at the first-order end-of-step position times the
  vertex's mean rest edge length l_i, l_i (b_i / h - m_i g) / m_i, where
  b = h (f(x_t) - h K(x_t) v_t) + h M g is the assembled right-hand side (so
  b_i / h - m_i g = f_int(x_t) - h (K v_t)_i; the length makes the membrane force's share
  independent of the grid spacing: force ~ stress x edge, mass ~ edge^2); and the mean of
  dv_prev over the vertex's edge neighbours (its one-ring).
* network: 12 -> 64 -> 64 -> 3, ReLU after the two hidden layers; inputs and targets
  are standardised with per-component means and standard deviations from the
  training set.
* target: the change of the solution from the previous step, dv - dv_prev, so that the
  prediction is dv0 = dv_prev + sd_y * y + mu_y (zero at pinned vertices).
* loss: L = 1/(2N) * sum over rows and outputs of (y - t)^2 on standardised targets.
* optimiser: Adam (Kingma and Ba 2015) with bias correction.

Parameter layout (one flat float vector): W1[64][12], b1[64], W2[64][64], b2[64],
W3[3][64], b3[3] (weights row-major [out][in]). Statistics layout: mu_x[12], sd_x[12],
mu_y[3], sd_y[3].
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 12, 64, 3
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5187
N_STATS = 2 * N_IN + 2 * N_OUT                       # 30
SD_FLOOR = 1e-12


def unpack(params):
    """Split the flat parameter vector into named arrays (views)."""
    p = np.asarray(params, dtype=np.float64).reshape(-1)
    assert p.size == N_PARAMS, p.size
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases (any start works for the tests)."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            bound = np.sqrt(6.0 / shape[1])
            parts[name] = rng.uniform(-bound, bound, size=shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts)


# --------------------------------------------------------------------------- features


def edges_of(tris) -> np.ndarray:
    """Unique undirected mesh edges (i < j) of a triangle list."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def ring_mean(V: int, edges, q) -> np.ndarray:
    """Mean of q over each vertex's edge neighbours (zero for an isolated vertex)."""
    q = np.asarray(q, dtype=np.float64).reshape(V, -1)
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    s = np.zeros_like(q)
    np.add.at(s, e[:, 0], q[e[:, 1]])
    np.add.at(s, e[:, 1], q[e[:, 0]])
    deg = np.zeros(V)
    np.add.at(deg, e[:, 0], 1.0)
    np.add.at(deg, e[:, 1], 1.0)
    return s / np.maximum(deg, 1.0)[:, None]


def rest_lengths(rest, edges) -> np.ndarray:
    """Mean rest length of each vertex's edges (zero for an isolated vertex)."""
    X = np.asarray(rest, dtype=np.float64).reshape(-1, 3)
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    L = np.linalg.norm(X[e[:, 1]] - X[e[:, 0]], axis=1)
    s = np.zeros(X.shape[0])
    deg = np.zeros(X.shape[0])
    np.add.at(s, e[:, 0], L)
    np.add.at(s, e[:, 1], L)
    np.add.at(deg, e[:, 0], 1.0)
    np.add.at(deg, e[:, 1], 1.0)
    return s / np.maximum(deg, 1.0)


def features(v, dv_prev, b, mass, h: float, gravity, edges, rest) -> np.ndarray:
    """The 12 raw features per vertex (see the module docstring)."""
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    V = v.shape[0]
    dvp = np.asarray(dv_prev, dtype=np.float64).reshape(V, 3)
    b = np.asarray(b, dtype=np.float64).reshape(V, 3)
    m = np.asarray(mass, dtype=np.float64).reshape(V)
    g = np.asarray(gravity, dtype=np.float64).reshape(3)
    f_int = b / h - m[:, None] * g[None, :]
    ell = rest_lengths(rest, edges)
    return np.concatenate([v, dvp, ell[:, None] * f_int / m[:, None], ring_mean(V, edges, dvp)], axis=1)


# --------------------------------------------------------------------------- statistics


def compute_stats(X, T) -> np.ndarray:
    """Per-component mean and (population) standard deviation of inputs and targets."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, N_IN)
    T = np.asarray(T, dtype=np.float64).reshape(-1, N_OUT)
    return np.concatenate([X.mean(0), np.maximum(X.std(0), SD_FLOOR), T.mean(0), np.maximum(T.std(0), SD_FLOOR)])


def split_stats(stats):
    s = np.asarray(stats, dtype=np.float64).reshape(-1)
    return s[:N_IN], s[N_IN:2 * N_IN], s[2 * N_IN:2 * N_IN + N_OUT], s[2 * N_IN + N_OUT:]


def normalize_inputs(X, stats) -> np.ndarray:
    mx, sx, _, _ = split_stats(stats)
    return (np.asarray(X, dtype=np.float64).reshape(-1, N_IN) - mx) / sx


def normalize_targets(T, stats) -> np.ndarray:
    _, _, my, sy = split_stats(stats)
    return (np.asarray(T, dtype=np.float64).reshape(-1, N_OUT) - my) / sy


# --------------------------------------------------------------------------- network


def _r(a, bf16: bool):
    return bf16_round(a) if bf16 else a


def forward(params, Xn, bf16: bool = False):
    """Pre-activations and activations of every layer for standardised inputs Xn.

    With bf16=True the values that the tensor-core kernels feed to their BF16 matrix
    products (inputs, weights, hidden activations) are rounded to bfloat16 first; sums,
    biases and the output stay in FP64."""
    P = unpack(params)
    W1, W2, W3 = (_r(P[k], bf16) for k in ("W1", "W2", "W3"))
    Xn = _r(np.asarray(Xn, dtype=np.float64).reshape(-1, N_IN), bf16)
    Z1 = Xn @ W1.T + P["b1"]
    H1 = _r(np.maximum(Z1, 0.0), bf16)
    Z2 = H1 @ W2.T + P["b2"]
    H2 = _r(np.maximum(Z2, 0.0), bf16)
    Y = H2 @ W3.T + P["b3"]
    return {"Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "Y": Y, "X": Xn}


def loss(params, Xn, Tn) -> float:
    Y = forward(params, Xn)["Y"]
    Tn = np.asarray(Tn, dtype=np.float64).reshape(-1, N_OUT)
    return 0.5 * float(np.sum((Y - Tn) ** 2)) / Y.shape[0]


def grad(params, Xn, Tn, bf16: bool = False) -> np.ndarray:
    """Gradient of `loss` by back-propagation through the three layers.

    With bf16=True, besides the forward rounding, the backward signals that enter BF16
    matrix products (dY, dZ2, dZ1) are rounded to bfloat16; bias gradients use the
    unrounded signals."""
    P = unpack(params)
    W2, W3 = _r(P["W2"], bf16), _r(P["W3"], bf16)
    Tn = np.asarray(Tn, dtype=np.float64).reshape(-1, N_OUT)
    a = forward(params, Xn, bf16)
    N = a["X"].shape[0]
    dY = (a["Y"] - Tn) / N
    dYr = _r(dY, bf16)
    g = {"W3": dYr.T @ a["H2"], "b3": dY.sum(0)}
    dZ2 = (dYr @ W3) * (a["Z2"] > 0.0)
    dZ2r = _r(dZ2, bf16)
    g["W2"] = dZ2r.T @ a["H1"]
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2r @ W2) * (a["Z1"] > 0.0)
    g["W1"] = _r(dZ1, bf16).T @ a["X"]
    g["b1"] = dZ1.sum(0)
    return pack(g)


def adam_step(params, m, v, g, t: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step number t >= 1); returns new (params, m, v)."""
    params = np.asarray(params, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def predict(params, stats, X, dv_prev, pinned=None, bf16: bool = False) -> np.ndarray:
    """Initial guess dv0 = dv_prev + de-standardised network output (0 at pins)."""
    _, _, my, sy = split_stats(stats)
    Y = forward(params, normalize_inputs(X, stats), bf16)["Y"]
    dv0 = np.asarray(dv_prev, dtype=np.float64).reshape(-1, 3) + Y * sy + my
    if pinned is not None:
        dv0[np.asarray(pinned, bool)] = 0.0
    return dv0


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))
