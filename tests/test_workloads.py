"""The seeded synthetic inputs: the random-number source against its published outputs,
the workloads' sizes against the closed forms of their grids (and the scope table's
counts), and the contact sets against the rules that generate them. CPU only."""
import numpy as np
import pytest

import oracle
from paper_2008_00409_gb300 import workloads as wk


def test_splitmix64_published_outputs():
    """The first outputs of SplitMix64 seeded with 0 (Steele, Lea and Flood 2014): the
    generator state advances by the golden gamma, so counters 0, G, 2G, ... give them."""
    G = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        c = np.arange(5, dtype=np.uint64) * G
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(v) for v in wk.splitmix64(c)] == want


def test_uniform_and_normal_draws():
    u = wk.uniform(7, 3, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    # explicit positions: the same values wherever they are drawn from
    assert np.array_equal(wk.uniform(7, 3, 10, offset=1000), wk.uniform_at(7, 3, np.arange(1000, 1010)))
    z = wk.normal(7, 5, 200_000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    r = wk.randint(7, 9, 100_000, -8, 8)
    assert r.min() == -8 and r.max() == 8 and np.bincount(r + 8).min() > 5000


def _interior_edges(tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]).astype(np.int64)
    e.sort(1)
    _, counts = np.unique(e[:, 0] * (1 << 32) + e[:, 1], return_counts=True)
    assert counts.max() <= 2  # a manifold grid
    return int((counts == 2).sum())


@pytest.mark.parametrize("name,n,layers", [("square64", 64, 1), ("square512-contacts", 512, 1),
                                           ("stack3x526", 526, 3)])
def test_sizes_match_the_grid_closed_forms(name, n, layers):
    """n x n vertices per sheet, 2 (n-1)^2 triangles, (n-1)(3n-5) interior edges (hinges);
    the scope table's figures: 64^2 4,096 / 7,938 / 11,781; 512^2 262,144 / 522,242 /
    782,341; 3 x 526^2 830,028 / 1,653,750 / 2,477,475."""
    wl = wk.WORKLOADS[name]()
    assert wl.V == layers * n * n
    assert wl.T == layers * 2 * (n - 1) ** 2
    assert _interior_edges(wl.tris) == layers * (n - 1) * (3 * n - 5)
    table = {"square64": (4096, 7938, 11781), "square512-contacts": (262144, 522242, 782341),
             "stack3x526": (830028, 1653750, 2477475)}[name]
    assert (wl.V, wl.T, layers * (n - 1) * (3 * n - 5)) == table
    # triangles counter-clockwise seen from +z in the rest state
    r = wl.rest.astype(np.float64)
    a, b, c = r[wl.tris[:, 0]], r[wl.tris[:, 1]], r[wl.tris[:, 2]]
    assert (np.cross(b - a, c - a)[:, 2] > 0).all()
    # two pinned corners at the top edge of each sheet
    assert wl.pins.shape == (2 * layers,)
    for s, k in zip(wl.sheets, range(layers)):
        assert set(wl.pins[2 * k:2 * k + 2]) == {s.vbase + (s.ny - 1) * s.nx, s.vbase + s.ny * s.nx - 1}


def test_warm_start_evaluation_cloth_size():
    wl = wk.warm_start_eval()
    assert (wl.V, wl.T) == (501264, 999698) and wl.n_contacts == round(0.02 * 501264)


@pytest.mark.parametrize("name,nnzb", [("square64", 51724), ("square512-contacts", 3395596)])
def test_mesh_pattern_size_matches_the_table(name, nnzb):
    """Blocks of the contact-free pattern of the diagonal-triangulated grids: each vertex,
    its edge neighbours and its hinges' wing vertices (scope table: 51,724 and 3,395,596)."""
    wl = wk.WORKLOADS[name]()
    rp, ci = oracle.Mesh.from_workload(wl).pattern(None)
    assert int(rp[-1]) == nnzb


def test_paper_scale_jitter_and_flips():
    wl = wk.paper_scale()
    n = 526
    dx = 1.0 / (n - 1)
    for k, s in enumerate(wl.sheets):
        r = wl.rest[s.vbase:s.vbase + n * n].astype(np.float64).reshape(n, n, 3)
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        off_x, off_y = r[..., 0] - ii * dx, r[..., 1] - jj * dx
        ulp = 2.0 ** -23  # rest positions are float32 in [0, 1]
        assert np.abs(off_x).max() <= 0.2 * dx + ulp and np.abs(off_y).max() <= 0.2 * dx + ulp
        edge = (ii == 0) | (ii == n - 1) | (jj == 0) | (jj == n - 1)
        assert np.abs(off_x[edge]).max() <= ulp and np.abs(off_y[edge]).max() <= ulp  # boundary not jittered
        assert np.allclose(r[..., 2], k * 5e-4)  # sheets 0.5 mm apart
        frac = s.flip.mean()
        assert abs(frac - 0.1) < 4 * np.sqrt(0.1 * 0.9 / s.flip.size)


def _check_pairs(wl, pairs, w):
    P = wl.n_contacts
    assert pairs.shape == (P, 4) and w.shape == (P, 3)
    assert len(np.unique(pairs[:, 0])) == P  # distinct vertices
    assert not (pairs[:, 1:] == pairs[:, :1]).any()  # never a triangle of its own vertex
    tri_keys = {tuple(sorted(t)) for t in wl.tris.tolist()}
    assert all(tuple(sorted(t)) in tri_keys for t in pairs[:, 1:].tolist())
    assert (w > 0).all() and np.abs(w.astype(np.float64).sum(1) - 1.0).max() < 1e-6


def test_grid_contacts_follow_their_rule():
    """512^2 with 2% contacts: round(0.02 V) = 5,243 distinct vertices, each paired with a
    triangle of a quad within 8 cells (the fallback takes the next quad row), Dirichlet
    weights; the set depends only on (seed, step)."""
    wl = wk.dynamic_square()
    assert wl.n_contacts == 5243
    pairs, w = wl.contacts(0)
    _check_pairs(wl, pairs, w)
    n = 512
    p = pairs[:, 0]
    quad_i = pairs[:, 1:].min(1) % n  # the lowest vertex of a quad's triangles is its (i, j) corner or beside it
    quad_j = pairs[:, 1:].min(1) // n
    assert (np.abs(quad_i - p % n) <= 9).all() and (np.abs(quad_j - p // n) <= 9).all()
    again = wl.contacts(0)
    assert np.array_equal(again[0], pairs) and np.array_equal(again[1], w)
    other = wl.contacts(1)
    assert not np.array_equal(other[0], pairs)


def test_interlayer_contacts_follow_their_rule():
    """Paper scale: round(0.05 V) = 41,501 pairs, the triangle on an adjacent sheet in a quad
    touching the vertex's own grid position."""
    wl = wk.paper_scale()
    assert wl.n_contacts == 41501
    pairs, w = wl.contacts(3)
    _check_pairs(wl, pairs, w)
    n = 526
    layer_p = pairs[:, 0] // (n * n)
    layer_t = pairs[:, 1:] // (n * n)
    assert (layer_t == layer_t[:, :1]).all() and (np.abs(layer_t[:, 0] - layer_p) == 1).all()
    lp = pairs[:, 0] % (n * n)
    lt = pairs[:, 1:] % (n * n)
    assert (np.abs(lt % n - (lp % n)[:, None]) <= 1).all() and (np.abs(lt // n - (lp // n)[:, None]) <= 1).all()


def test_batched_garments_recipe():
    """64 garments with log-uniform triangle counts in [2e3, 2e5] on grids of side
    round(sqrt(T / 2)) + 1, stacked as disjoint row ranges; contacts stay inside a garment."""
    u = wk.garment_batch_union()
    assert len(u.parts) == 64 and u.inst_rows[0] == 0 and u.inst_rows[-1] == u.V
    sides = np.array([p.sheets[0].nx for p in u.parts])
    assert (2 * (sides - 1) ** 2 >= 0.9 * 2e3).all() and (2 * (sides - 1) ** 2 <= 1.1 * 2e5).all()
    assert 2.0e6 < u.T < 3.5e6
    pairs, w = u.contacts(0)
    inst = np.searchsorted(u.inst_rows, pairs, side="right") - 1
    assert (inst == inst[:, :1]).all()
    assert pairs.shape[0] == sum(p.n_contacts for p in u.parts)
