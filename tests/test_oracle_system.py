"""Pins for the oracle's assembled system (Sec. 2.5 Eq. 3, Sec. 3.2.2) and its solver.

Checked against things other than the oracle itself: brute-force coupling sets,
closed-form hinge counts, exact symmetry / positive definiteness, the element-by-
element (matrix-free) product, the closed-form free fall dv = h g, a FD Jacobian of
the assembled forces, and a dense Cholesky solve on tiny meshes.
"""
import numpy as np
import pytest

import oracle
from paper_2008_00409_gb300 import workloads as wk

MAT = wk.Material().as_array()
H_STEP = 1.0 / 200.0


def tiny_cloth(nx=6, ny=5, flip_prob=0.3, jitter=0.2, seed=7, contacts=4, pins=(0, 5)):
    rest, tris, flip = wk.grid_piece(nx, ny, 0.1, 0.08, jitter=jitter, flip_prob=flip_prob, seed=seed)
    rng = np.random.default_rng(seed)
    V = nx * ny
    x = rest.astype(np.float64) + 2e-3 * rng.normal(size=(V, 3))
    v = 0.05 * rng.normal(size=(V, 3))
    pairs, w = [], []
    for _ in range(contacts):
        while True:
            p = int(rng.integers(V))
            t = tris[int(rng.integers(len(tris)))]
            if p not in t:
                break
        pairs.append([p, *t])
        ww = rng.dirichlet([1, 1, 1])
        w.append(ww)
    pairs = np.array(pairs, np.int32).reshape(-1, 4)
    w = np.array(w).reshape(-1, 3)
    M = oracle.Mesh(rest, tris, MAT, pins)
    return M, rest, tris, x, v, pairs, w


def test_hinge_count_closed_form():
    # interior edges of an n x m diagonal-triangulated grid:
    # (n-1)m + n(m-1) + (n-1)(m-1) edges minus the 2(n-1) + 2(m-1) boundary edges
    for n, m in [(2, 2), (3, 4), (7, 5), (64, 64)]:
        rest, tris, _ = wk.grid_piece(n, m, 1.0, 1.0)
        M = oracle.Mesh(rest, tris, MAT)
        edges = (n - 1) * m + n * (m - 1) + (n - 1) * (m - 1)
        assert M.H == edges - 2 * (n - 1) - 2 * (m - 1)
    rest, tris, _ = wk.grid_piece(64, 64, 1.0, 1.0)
    assert oracle.Mesh(rest, tris, MAT).H == 11781


def test_pattern_equals_brute_force_coupling_set():
    M, rest, tris, x, v, pairs, w = tiny_cloth()
    rp, ci = M.pattern(pairs)
    coupled = np.zeros((M.V, M.V), bool)
    np.fill_diagonal(coupled, True)
    for group in list(tris) + list(M.hinges) + list(pairs):
        for a in group:
            for b in group:
                coupled[a, b] = True
    rows = np.repeat(np.arange(M.V), np.diff(rp))
    got = np.zeros_like(coupled)
    got[rows, ci] = True
    assert (got == coupled).all()
    assert len(ci) == coupled.sum()
    for r in range(M.V):  # columns ascending, no duplicates
        assert (np.diff(ci[rp[r]:rp[r + 1]]) > 0).all()


def test_hinge_wings_are_the_opposite_vertices():
    M, rest, tris, *_ = tiny_cloth(contacts=0)
    tset = {tuple(sorted(t)) for t in tris}
    for wa, wb, e0, e1 in M.hinges:
        assert tuple(sorted((wa, e0, e1))) in tset and tuple(sorted((wb, e0, e1))) in tset
        assert wa != wb


def test_system_symmetric_positive_definite_with_pins_and_contacts():
    M, rest, tris, x, v, pairs, w = tiny_cloth()
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP)
    A = oracle.dense(rp, ci, vals)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    np.linalg.cholesky(A)  # raises if not positive definite
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    for p in M.pins:  # pin rule
        assert (b[p] == 0).all()
        blk = A[3 * p:3 * p + 3]
        np.testing.assert_array_equal(blk[:, 3 * p:3 * p + 3], M.mass[p] * np.eye(3))
        assert np.count_nonzero(blk) == 3 and np.count_nonzero(A[:, 3 * p:3 * p + 3]) == 3


def test_matrix_free_identity():
    M, rest, tris, x, v, pairs, w = tiny_cloth(pins=())
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP, pins=False)
    rng = np.random.default_rng(11)
    for _ in range(3):
        p = rng.normal(size=(M.V, 3))
        y_mat = oracle.spmv(rp, ci, vals, p)
        y_free = M.matfree_apply(x, p, pairs, w, H_STEP)
        np.testing.assert_allclose(y_mat, y_free, rtol=1e-12, atol=1e-14 * np.abs(y_free).max())
        # and against a dense product
        np.testing.assert_allclose(oracle.dense(rp, ci, vals) @ p.reshape(-1), y_mat.reshape(-1), rtol=1e-12,
                                   atol=1e-15)


def test_translation_is_mass_only_and_forces_rigid_invariant():
    M, rest, tris, x, v, pairs, w = tiny_cloth(pins=())
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP, pins=False)
    for t in ([1.0, 0, 0], [0.3, -2.0, 0.7]):
        T = np.tile(np.array(t), (M.V, 1))
        y = oracle.spmv(rp, ci, vals, T)
        np.testing.assert_allclose(y, M.mass[:, None] * T, rtol=1e-10, atol=1e-12 * np.abs(vals).max())
    f0 = M.forces(x, pairs, w, xt=x)
    shift = np.array([0.5, -0.2, 1.5])
    f1 = M.forces(x + shift, pairs, w, xt=x + shift)
    np.testing.assert_allclose(f1, f0, rtol=1e-9, atol=1e-12 * np.abs(f0).max())


def test_assembled_hessian_is_force_jacobian_in_tension():
    # flat sheet in uniform biaxial tension: the membrane clamp is inactive and every
    # hinge sits at its rest angle, so -df/dx must equal the assembled K exactly
    rest, tris, _ = wk.grid_piece(5, 4, 0.1, 0.08, jitter=0.2, seed=3)
    M = oracle.Mesh(rest, tris, MAT)
    x = rest.astype(np.float64) * np.array([1.03, 1.05, 1.0])
    rng = np.random.default_rng(5)
    pairs = np.array([[0, 6, 7, 11], [13, 1, 2, 6]], np.int32)
    w = rng.dirichlet([1, 1, 1], size=2)
    xt = x + 1e-5 * rng.normal(size=x.shape)
    xt[:, 2] = 0.0
    x = xt.copy()
    rp, ci, K = M.hessian(x, pairs, w, xt=xt)
    Kd = oracle.dense(rp, ci, K)
    eps = 1e-7
    J = np.zeros_like(Kd)
    for j in range(3 * M.V):
        xp, xm = x.reshape(-1).copy(), x.reshape(-1).copy()
        xp[j] += eps
        xm[j] -= eps
        J[:, j] = (M.forces(xp.reshape(-1, 3), pairs, w, xt) - M.forces(xm.reshape(-1, 3), pairs, w, xt)).reshape(-1) / (2 * eps)
    np.testing.assert_allclose(Kd, -J, rtol=1e-5, atol=1e-6 * np.abs(Kd).max())


def test_rhs_is_first_order_expansion_of_force_at_predicted_positions():
    # b = h f(x + h v) to first order in h v (Eq. 2): the gap to the literal evaluation
    # is h * O(|h v|^2), so it shrinks 4x when h v halves; for a system whose forces are
    # linear in x (contacts and gravity only, frozen contact frames) it is exact
    # (flat sheet in biaxial tension: there the clamped, Gauss-Newton K is the exact -J)
    M, rest, tris, x, v, pairs, w = tiny_cloth(pins=())
    xt = rest.astype(np.float64) * np.array([1.03, 1.05, 1.0])
    gaps = []
    for s in (1.0, 0.5, 0.25):
        vv = 0.1 * s * v
        _, _, _, b = M.assemble(xt, vv, pairs, w, H_STEP, pins=False)
        f = M.forces(xt + H_STEP * vv, pairs, w, xt=xt)
        gaps.append(np.linalg.norm(b - H_STEP * f))
    assert 3.5 < gaps[0] / gaps[1] < 4.5 and 3.5 < gaps[1] / gaps[2] < 4.5
    mat = MAT.copy()
    mat[1] = 1e-9  # membrane off (tiny modulus keeps the mesh valid)
    mat[3] = 0.0   # bending off
    Ml = oracle.Mesh(rest, tris, mat)
    _, _, _, b = Ml.assemble(x, v, pairs, w, H_STEP, pins=False)
    f = Ml.forces(x + H_STEP * v, pairs, w, xt=x)
    np.testing.assert_allclose(b, H_STEP * f, rtol=1e-9, atol=1e-9 * np.abs(b).max())


def test_rhs_matches_dense_linearisation_with_pins():
    M, rest, tris, x, v, pairs, w = tiny_cloth()
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP)
    _, _, K = M.hessian(x, pairs, w, xt=x, pattern=(rp, ci))
    Kd = oracle.dense(rp, ci, K)
    ref = H_STEP * (M.forces(x, pairs, w, xt=x).reshape(-1) - H_STEP * Kd @ v.reshape(-1))
    ref = ref.reshape(-1, 3)
    ref[M.pins] = 0.0
    np.testing.assert_allclose(b, ref, rtol=1e-12, atol=1e-15)


def test_twenty_steps_stay_bounded():
    # the 64 x 64 cloth hanging from two corners: free-falling parts gain h g per step,
    # nothing may grow faster than that (a diverging integrator fails here)
    wl = wk.small_square()
    M = oracle.Mesh.from_workload(wl)
    x = wl.x0.astype(np.float64)
    v = wl.v0.astype(np.float64)
    for step in range(20):
        dv, x, v, info = M.step(x, v, h=wl.h, tol=1e-9)
        assert np.abs(v).max() <= (step + 1) * H_STEP * 9.81 * 1.5 + 0.1
    assert np.isfinite(x).all()


@pytest.mark.parametrize("v0", [(0.0, 0.0, 0.0), (0.4, -0.1, 0.2)])
def test_free_fall_closed_form(v0):
    # no pins, rest shape, uniform velocity: internal forces vanish at x + h v, A maps
    # translations to M t, so the exact solution is dv = h g for every vertex
    rest, tris, _ = wk.grid_piece(9, 7, 0.2, 0.15, jitter=0.2, flip_prob=0.2, seed=9)
    M = oracle.Mesh(rest, tris, MAT)
    x = rest.astype(np.float64)
    v = np.tile(np.array(v0), (M.V, 1))
    dv, x1, v1, info = M.step(x, v, h=H_STEP, tol=1e-13)
    np.testing.assert_allclose(dv, np.tile(H_STEP * MAT[5:8], (M.V, 1)), rtol=0, atol=1e-12)


def test_pcg_matches_dense_cholesky():
    M, rest, tris, x, v, pairs, w = tiny_cloth(nx=8, ny=8, contacts=6, pins=(56, 63))
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP)
    A = oracle.dense(rp, ci, vals)
    L = np.linalg.cholesky(A)
    ref = np.linalg.solve(L.T, np.linalg.solve(L, b.reshape(-1)))
    dv, it, rel = oracle.pcg(rp, ci, vals, b, tol=1e-13)
    assert rel <= 1e-12
    np.testing.assert_allclose(dv.reshape(-1), ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    assert (dv[M.pins] == 0).all()


def test_pcg_reports_non_convergence():
    M, rest, tris, x, v, pairs, w = tiny_cloth()
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP)
    with pytest.raises(oracle.OracleError):
        oracle.pcg(rp, ci, vals, b, tol=1e-14, max_iter=2)


def test_invalid_mesh_and_pairs_rejected():
    rest, tris, _ = wk.grid_piece(3, 3, 1.0, 1.0)
    with pytest.raises(oracle.OracleError):
        oracle.Mesh(rest, np.array([[0, 1, 9]]), MAT)
    with pytest.raises(oracle.OracleError):
        oracle.Mesh(rest, np.array([[0, 1, 1]]), MAT)
    M = oracle.Mesh(rest, tris, MAT)
    with pytest.raises(oracle.OracleError):
        M.pattern(np.array([[0, 0, 1, 2]]))


def test_batch_union_keeps_garments_disjoint():
    parts = [wk.garment(s, seed=5, stream=10 * k, contact_frac=0.05) for k, s in enumerate([6, 9, 7])]
    u = wk.batch_union(parts)
    assert u.V == sum(p.V for p in parts) and u.T == sum(p.T for p in parts)
    assert list(u.inst_rows) == [0, 36, 117, 166]
    inst = np.searchsorted(u.inst_rows, u.tris, side="right") - 1
    assert (inst == inst[:, :1]).all()
    pairs, w = u.contacts(0)
    pi = np.searchsorted(u.inst_rows, pairs, side="right") - 1
    assert (pi == pi[:, :1]).all() and len(pairs) == u.n_contacts
    M = oracle.Mesh.from_workload(u)
    assert M.H == sum(oracle.Mesh.from_workload(p).H for p in parts)


# ------------------------------------------------------------------ Rayleigh damping


def _damped(alpha, beta):
    m = MAT.copy()
    m[8], m[9] = alpha, beta
    return m


@pytest.mark.parametrize("alpha,beta", [(2.0, 0.0), (0.0, 0.02), (3.5, 0.01)])
def test_damped_translation_closed_form(alpha, beta):
    # rest shape, uniform velocity u, no pins: K u = 0, so stiffness damping does nothing
    # and mass damping gives the scalar backward Euler dv = h (g - alpha u) / (1 + h alpha)
    rest, tris, _ = wk.grid_piece(9, 7, 0.2, 0.15, jitter=0.2, flip_prob=0.2, seed=9)
    M = oracle.Mesh(rest, tris, _damped(alpha, beta))
    u = np.array([0.4, -0.1, 0.2])
    x = rest.astype(np.float64)
    v = np.tile(u, (M.V, 1))
    dv, x1, v1, info = M.step(x, v, h=H_STEP, tol=1e-13)
    want = H_STEP * (MAT[5:8] - alpha * u) / (1.0 + H_STEP * alpha)
    np.testing.assert_allclose(dv, np.tile(want, (M.V, 1)), rtol=0, atol=1e-12)


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (1.5, 0.0), (0.0, 0.03), (2.0, 0.01)])
def test_damped_free_vertex_matches_fd_backward_euler(alpha, beta):
    # one free vertex of a triangle in biaxial tension, the other two pinned at rest
    # velocity: the damped backward Euler step of that vertex, written out with the 3x3
    # stiffness taken as the central-difference Jacobian of the forces, must match the
    # assembled and solved system
    rest = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.02, 0.09, 0.0]])
    tris = np.array([[0, 1, 2]], np.int32)
    M = oracle.Mesh(rest, tris, _damped(alpha, beta), pins=[1, 2])
    x = rest * np.array([1.04, 1.06, 1.0])
    x[0] += np.array([0.001, -0.002, 0.0005])
    v = np.zeros((3, 3))
    v[0] = [0.3, -0.2, 0.5]
    f0 = M.forces(x)[0]
    eps = 1e-7
    K = np.zeros((3, 3))
    for j in range(3):
        xp, xm = x.copy(), x.copy()
        xp[0, j] += eps
        xm[0, j] -= eps
        K[:, j] = -(M.forces(xp, xt=xp)[0] - M.forces(xm, xt=xm)[0]) / (2 * eps)
    h, m = H_STEP, M.mass[0]
    A = (1 + h * alpha) * m * np.eye(3) + h * (h + beta) * K
    b = h * (f0 - alpha * m * v[0] - (h + beta) * K @ v[0])
    want = np.linalg.solve(A, b)
    rp, ci, vals, bb = M.assemble(x, v, h=h)
    got = np.linalg.solve(oracle.dense(rp, ci, vals), bb.reshape(-1)).reshape(-1, 3)
    np.testing.assert_allclose(got[0], want, rtol=1e-6, atol=1e-9 * np.abs(want).max())
    assert np.all(got[1:] == 0.0)


def test_damped_matrix_free_identity_and_dissipation():
    M0, rest, tris, x, v, pairs, w = tiny_cloth(pins=())
    M = oracle.Mesh(rest, tris, _damped(1.0, 0.02))
    rp, ci, vals, b = M.assemble(x, v, pairs, w, H_STEP, pins=False)
    rng = np.random.default_rng(12)
    p = rng.normal(size=(M.V, 3))
    y_free = M.matfree_apply(x, p, pairs, w, H_STEP)
    np.testing.assert_allclose(oracle.spmv(rp, ci, vals, p), y_free, rtol=1e-12, atol=1e-14 * np.abs(y_free).max())
    # the damping force -(alpha M + beta K) v does negative work: the damped system's
    # right-hand side differs from the undamped one by -h (alpha M + beta K) v, whose dot
    # product with v is negative for any v
    _, _, _, b0 = M0.assemble(x, v, pairs, w, H_STEP, pins=False)
    assert np.sum((b - b0) * v) < 0.0
