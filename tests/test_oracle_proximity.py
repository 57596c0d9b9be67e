"""Pins for the one-sided thickness contact model and its proximity query (oracle).

The element E = kc/2 (delta - d)^2 (active while d(x_t) < delta, normal turned towards
the vertex at x_t) is pinned by finite differences, by the closed form of a vertex above
a triangle's centroid, by its inactivity beyond delta and by mirror symmetry. The FP32
closest point is pinned against dense sampling of the triangle in FP64 and against the
closed forms of each Voronoi region; the query against two aligned parallel grids, whose
pairs are known in closed form, and against the one-ring exclusion rule.
"""
import numpy as np
import pytest

import oracle
from oracle import proximity as px
from paper_2008_00409_gb300 import workloads as wk

DELTA = 1e-3


def _thick_mesh(delta=DELTA):
    m = wk.Material().as_array()
    m[10] = delta
    return oracle.Mesh(np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [0.0, 0.01, 0.0]]), [[0, 1, 2]], m)


TRI = np.array([[0.0, 0.0, 0.0], [0.012, 0.001, 0.0], [0.002, 0.011, 0.0]])


@pytest.mark.parametrize("side", [1.0, -1.0])
def test_thickness_contact_closed_form_above_centroid(side):
    M = _thick_mesh()
    kc = M.material[4]
    h = side * 0.4e-3
    c = TRI.mean(axis=0)
    xt = np.vstack([c + [0, 0, h], TRI])
    w = np.full(3, 1.0 / 3.0)
    E, f, H = M.element(2, xt, xt, aux=w)
    n = np.array([0.0, 0.0, np.sign(h)])  # turned towards the vertex
    assert E == pytest.approx(0.5 * kc * (DELTA - abs(h)) ** 2, rel=1e-12)
    np.testing.assert_allclose(f[0], kc * (DELTA - abs(h)) * n, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f[1:], np.tile(-kc * (DELTA - abs(h)) / 3 * n, (3, 1)), rtol=1e-12, atol=1e-15)
    s = np.array([1.0, -1 / 3, -1 / 3, -1 / 3])
    np.testing.assert_allclose(H, kc * np.einsum("k,l,a,b->klab", s, s, n, n), rtol=1e-12, atol=1e-12)


def test_thickness_contact_inactive_beyond_delta_and_fd():
    M = _thick_mesh()
    c = TRI.mean(axis=0)
    far = np.vstack([c + [0, 0, 1.5 * DELTA], TRI])
    E, f, H = M.element(2, far, far, aux=np.full(3, 1 / 3))
    assert E == 0.0 and not f.any() and not H.any()
    # active: forces are minus the energy gradient, the Hessian minus the force Jacobian
    rng = np.random.default_rng(4)
    w = np.array([0.2, 0.5, 0.3])
    xt = np.vstack([w @ TRI + [0, 0, 0.3e-3], TRI]) + 1e-5 * rng.normal(size=(4, 3))
    x = xt + 2e-5 * rng.normal(size=(4, 3))
    E, f, H = M.element(2, x, xt, aux=w)
    eps = 1e-8
    for i in range(4):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += eps
            xm[i, a] -= eps
            g = (M.element(2, xp, xt, aux=w)[0] - M.element(2, xm, xt, aux=w)[0]) / (2 * eps)
            assert f[i, a] == pytest.approx(-g, rel=1e-5, abs=1e-9)
            J = (M.element(2, xp, xt, aux=w)[1] - M.element(2, xm, xt, aux=w)[1]) / (2 * eps)
            np.testing.assert_allclose(H[:, i, :, a], -J, rtol=1e-5, atol=1e-6 * np.abs(H).max())


def test_zero_thickness_is_the_hold_penalty():
    m = wk.Material().as_array()
    M0 = oracle.Mesh(TRI, [[0, 1, 2]], m)
    rng = np.random.default_rng(5)
    xt = np.vstack([TRI.mean(0) + [0, 0, 0.5e-3], TRI])
    x = xt + 1e-4 * rng.normal(size=(4, 3))
    E, f, H = M0.element(2, x, xt, aux=np.full(3, 1 / 3))
    assert E > 0 and np.abs(f).max() > 0
    E0, f0, _ = M0.element(2, xt, xt, aux=np.full(3, 1 / 3))
    assert E0 == 0.0 and np.abs(f0).max() == 0.0


# ------------------------------------------------------------------ closest point


def _sampled_min(p, a, b, c, n=400):
    """Smallest distance from p to the triangle over a dense barycentric grid plus the
    exact projections onto the three edges (FP64)."""
    u = np.linspace(0, 1, n)
    U, W = np.meshgrid(u, u)
    m = U + W <= 1
    pts = a + np.outer(U[m], b - a) + np.outer(W[m], c - a)
    best = np.min(np.sum((pts - p) ** 2, axis=1))
    for s, e in ((a, b), (a, c), (b, c)):
        t = np.clip(np.dot(p - s, e - s) / np.dot(e - s, e - s), 0, 1)
        best = min(best, np.sum((s + t * (e - s) - p) ** 2))
    return best


def test_closest_point_matches_dense_sampling():
    rng = np.random.default_rng(6)
    for _ in range(200):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 1.5
        w, d2 = px.closest_point(p, a, b, c)
        assert w.dtype == np.float32 and abs(w.sum() - 1) < 1e-5 and w.min() > -1e-6
        q = w.astype(np.float64) @ np.vstack([a, b, c])
        ref = _sampled_min(p, a, b, c)
        # the FP32 answer is the minimum, not just a point of the triangle
        assert np.sum((q - p) ** 2) <= ref * (1 + 1e-4) + 1e-10
        assert float(d2) == pytest.approx(np.sum((q - p) ** 2), rel=1e-4, abs=1e-9)


def test_closest_point_regions_closed_form():
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    cases = [
        ([0.25, 0.25, 0.5], [0.5, 0.25, 0.25], 0.25),      # face: projection inside
        ([-1.0, -1.0, 0.0], [1, 0, 0], 2.0),                # vertex a
        ([2.0, -0.5, 0.0], [0, 1, 0], 1.25),                # vertex b
        ([-0.5, 2.0, 0.0], [0, 0, 1], 1.25),                # vertex c
        ([0.5, -1.0, 0.0], [0.5, 0.5, 0], 1.0),             # edge ab
        ([-1.0, 0.25, 0.0], [0.75, 0, 0.25], 1.0),          # edge ac
        ([1.0, 1.0, 0.0], [0, 0.5, 0.5], 0.5),              # edge bc
    ]
    for p, w_ref, d2_ref in cases:
        w, d2 = px.closest_point(p, a, b, c)
        np.testing.assert_allclose(w, w_ref, atol=1e-7)
        assert float(d2) == pytest.approx(d2_ref, rel=1e-6)


# ------------------------------------------------------------------ query


def _two_sheets(n=6, spacing=0.01, gap=1e-3):
    rest, tris, _ = wk.grid_piece(n, n, spacing * (n - 1), spacing * (n - 1))
    top = rest.copy()
    top[:, 2] += gap
    x = np.vstack([rest, top])
    T = np.vstack([tris, tris + len(rest)])
    return x, T, len(rest), tris


def test_query_on_aligned_sheets_closed_form():
    # every vertex faces the vertex of the other sheet at distance gap; the triangles of
    # that vertex are at exactly gap, every other triangle of that sheet is at least
    # sqrt(gap^2 + (spacing / sqrt 2)^2) away, and the own sheet is excluded (one-ring) or
    # farther than delta in the plane
    gap, spacing = 1e-3, 0.01
    x, T, nv, tris = _two_sheets(gap=gap, spacing=spacing)
    deg = np.bincount(tris.reshape(-1), minlength=nv)
    pairs, w = px.query(x, T, 1.5 * gap)
    assert len(pairs) == 2 * deg.sum()
    for (p, a, b, c), ww in zip(pairs, w):
        other = p + nv if p < nv else p - nv
        assert other in (a, b, c) and (p < nv) != (a < nv)
        np.testing.assert_allclose(ww[[a, b, c].index(other)], 1.0, atol=1e-6)
    assert np.all(np.diff(pairs[:, 0]) >= 0)  # ordered by vertex
    assert len(px.query(x, T, 0.9 * gap)[0]) == 0


def test_query_excludes_the_one_ring():
    # a single flat sheet (spacing s): every vertex is at distance 0 from its own triangles
    # and from the triangles of its neighbours (in the plane), all excluded; the nearest
    # triangle that touches neither p nor a neighbour is sqrt(2) s away (through the
    # diagonal vertex that is not a neighbour), so it comes in with delta = 1.5 s only
    s = 0.01
    rest, tris, _ = wk.grid_piece(5, 5, 4 * s, 4 * s)
    assert len(px.query(rest, tris, 1.4 * s)[0]) == 0
    pairs, _ = px.query(rest, tris, 1.5 * s)
    rings = px.one_rings(len(rest), tris)
    assert len(pairs) > 0
    for p, a, b, c in pairs:
        assert not ({a, b, c} & (rings[p] | {p}))
