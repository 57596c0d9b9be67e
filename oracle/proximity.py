"""Proximity query of the one-sided thickness contact model (oracle).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's CPU
baseline, never by the product path (the CUDA library has its own query and shares no
code with this file).

The contact pairs of a step are the (vertex p, triangle t) pairs whose distance at x_t
is below the contact thickness delta, with t not touching p or any mesh-edge neighbour
of p (the one-ring of a flat sheet lies in p's own plane, at distances below delta on
fine meshes; those pairs are not contacts). The pair's weights are the barycentric
coordinates of the point of t closest to p. Pairs are listed by p, then by t.

The closest point follows the Voronoi-region classification of a point against a
triangle (Ericson, Real-Time Collision Detection, 2005, Sec. 5.1.5): vertex regions,
edge regions, then the face. Which region applies and whether the squared distance is
below delta^2 are decisions that floating point takes, so this file takes them in FP32
with one rounding per operation in a fixed order (no fused multiply-add), the same order
the CUDA query uses; the pair sets and weights of the two then agree exactly.

The paper's collision handling (spatial hashing and continuous collision detection,
Sec. 4) is not reproduced; this query is the proximity step that feeds contacts into
its implicit integrator (Sec. 2.5, Eq. 3).
"""
import numpy as np

F = np.float32


def _dot(u, v):
    # ((u.x v.x) + (u.y v.y)) + (u.z v.z), each operation rounded to FP32
    return (u[..., 0] * v[..., 0] + u[..., 1] * v[..., 1]) + u[..., 2] * v[..., 2]


def closest_point(p, a, b, c):
    """Barycentric weights (w_a, w_b, w_c) of the point of triangle (a, b, c) closest to
    p, and the squared distance, in FP32. Arrays of shape (..., 3) broadcast together."""
    p, a, b, c = (np.asarray(t, dtype=F) for t in (p, a, b, c))
    p, a, b, c = np.broadcast_arrays(p, a, b, c)
    one, zero = F(1), F(0)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ab = b - a
        ac = c - a
        ap = p - a
        d1 = _dot(ab, ap)
        d2 = _dot(ac, ap)
        bp = p - b
        d3 = _dot(ab, bp)
        d4 = _dot(ac, bp)
        cp = p - c
        d5 = _dot(ab, cp)
        d6 = _dot(ac, cp)
        vc = d1 * d4 - d3 * d2
        vb = d5 * d2 - d1 * d6
        va = d3 * d6 - d5 * d4
        t_ab = d1 / (d1 - d3)
        t_ac = d2 / (d2 - d6)
        e43 = d4 - d3
        e56 = d5 - d6
        t_bc = e43 / (e43 + e56)
        s = (va + vb) + vc
        f_v = vb / s
        f_w = vc / s
        # weights of b and c per region, in priority order (the first region that applies)
        shape = d1.shape
        wb = np.zeros(shape, F)
        wc = np.zeros(shape, F)
        done = np.zeros(shape, bool)

        def take(cond, vb_, vc_):
            nonlocal done
            m = cond & ~done
            wb[m] = np.broadcast_to(vb_, shape)[m]
            wc[m] = np.broadcast_to(vc_, shape)[m]
            done |= m

        take((d1 <= zero) & (d2 <= zero), zero, zero)                      # vertex a
        take((d3 >= zero) & (d4 <= d3), one, zero)                         # vertex b
        take((vc <= zero) & (d1 >= zero) & (d3 <= zero), t_ab, zero)       # edge ab
        take((d6 >= zero) & (d5 <= d6), zero, one)                         # vertex c
        take((vb <= zero) & (d2 >= zero) & (d6 <= zero), zero, t_ac)       # edge ac
        take((va <= zero) & (e43 >= zero) & (e56 >= zero), one - t_bc, t_bc)  # edge bc
        take(~(s > zero), zero, zero)                                      # degenerate: a
        take(np.ones(shape, bool), f_v, f_w)                               # face
        wa = (one - wb) - wc
        q = (a + ab * wb[..., None]) + ac * wc[..., None]
        r = p - q
        d2sq = _dot(r, r)
    return np.stack([wa, wb, wc], axis=-1), d2sq


def one_rings(V, tris):
    """Mesh-edge neighbours of every vertex (sets)."""
    nb = [set() for _ in range(V)]
    for t in np.asarray(tris):
        for i in range(3):
            for j in range(3):
                if i != j:
                    nb[int(t[i])].add(int(t[j]))
    return nb


def query(x, tris, delta, vertices=None, rings=None):
    """Contact pairs (p, a, b, c) and weights of the vertices `vertices` (all by default)
    against every triangle, by brute force: int32[P][4], float32[P][3], ordered by p then
    by triangle index."""
    x = np.asarray(x, dtype=F).reshape(-1, 3)
    tris = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    V = x.shape[0]
    rings = rings if rings is not None else one_rings(V, tris)
    d2max = F(delta) * F(delta)
    A, B, C = x[tris[:, 0]], x[tris[:, 1]], x[tris[:, 2]]
    # a conservative prefilter in FP64 (boxes grown by twice delta), then the exact test
    lo = np.minimum(np.minimum(A, B), C).astype(np.float64) - 2.0 * delta
    hi = np.maximum(np.maximum(A, B), C).astype(np.float64) + 2.0 * delta
    pairs, weights = [], []
    for p in (range(V) if vertices is None else vertices):
        xp = x[p].astype(np.float64)
        cand = np.nonzero(np.all((lo <= xp) & (xp <= hi), axis=1))[0]
        if cand.size == 0:
            continue
        near = rings[p] | {p}
        keep = [t for t in cand if not (int(tris[t, 0]) in near or int(tris[t, 1]) in near or int(tris[t, 2]) in near)]
        if not keep:
            continue
        keep = np.array(keep, dtype=np.int64)
        w, d2 = closest_point(x[p][None, :], A[keep], B[keep], C[keep])
        hit = d2 < d2max
        for t, ww in zip(keep[hit], w[hit]):
            pairs.append([p, *tris[t]])
            weights.append(ww)
    if not pairs:
        return np.zeros((0, 4), np.int32), np.zeros((0, 3), F)
    return np.array(pairs, np.int32), np.array(weights, F)
