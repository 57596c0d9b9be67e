"""Pins for the oracle's element models (membrane, bending, contact, gravity).

The paper gives no force formulas and prints no worked example (Sec. 3.2 names the
assembly elements only), so each element is pinned by what the mathematics fixes:
forces against central finite differences of the energy, Hessians against finite
differences of the forces where the clamping is inactive, closed forms (uniaxial
stretch, folded hinge angle, free translation) and invariances.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2008_00409_gb300 import workloads as wk

MAT = wk.Material().as_array()


def _mesh_one_triangle(rest):
    return oracle.Mesh(rest, [[0, 1, 2]], MAT)


def _fd_grad(fun, x, eps=1e-7):
    x = np.array(x, dtype=np.float64)
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        xp = x.copy()
        xm = x.copy()
        xp[i] += eps
        xm[i] -= eps
        g[i] = (fun(xp) - fun(xm)) / (2 * eps)
    return g


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


REST_TRI = np.array([[0.0, 0.0, 0.0], [0.013, 0.001, 0.0], [0.004, 0.011, 0.0]])


def _aux_tri(M):
    return np.concatenate([M.Dminv[0], [M.area[0]]])


def test_membrane_rest_is_stress_free_and_rigid_invariant():
    M = _mesh_one_triangle(REST_TRI)
    aux = _aux_tri(M)
    E, f, _ = M.element(0, REST_TRI, aux=aux)
    assert abs(E) < 1e-20 and np.abs(f).max() < 1e-12
    R = _rot([0.3, -0.5, 0.8], 1.1)
    x = REST_TRI @ R.T + np.array([0.2, -0.7, 3.0])
    E, f, _ = M.element(0, x, aux=aux)
    assert abs(E) < 1e-16 and np.abs(f).max() < 1e-10


def test_membrane_uniaxial_stretch_closed_form():
    # unit right triangle stretched by s along x: G = diag((s^2-1)/2, 0),
    # W = A0 (mu + lam/2) (s^2 - 1)^2 / 4  (plane-stress Lame constants)
    rest = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1.0, 0]])
    M = _mesh_one_triangle(rest)
    E_, nu = MAT[1], MAT[2]
    mu, lam = E_ / (2 * (1 + nu)), E_ * nu / (1 - nu * nu)
    for s in (1.001, 1.1, 0.9):
        x = rest * np.array([s, 1.0, 1.0])
        W, f, _ = M.element(0, x, aux=_aux_tri(M))
        A0 = 0.5
        assert W == pytest.approx(A0 * (mu + lam / 2) * (s * s - 1) ** 2 / 4, rel=1e-12)
        # S11 = (2mu + lam)(s^2-1)/2; vertex 1 gets -A0 * s * S11 * (1/1) along x
        S11 = (2 * mu + lam) * (s * s - 1) / 2
        assert f[1, 0] == pytest.approx(-A0 * s * S11, rel=1e-12)
        assert abs(f.sum(0)).max() < 1e-9 * abs(f).max()


def test_membrane_forces_match_energy_gradient():
    M = _mesh_one_triangle(REST_TRI)
    aux = _aux_tri(M)
    rng = np.random.default_rng(1)
    for trial in range(5):
        x = REST_TRI @ _rot(rng.normal(size=3), rng.normal()).T + 0.003 * rng.normal(size=(3, 3))
        _, f, _ = M.element(0, x, aux=aux)
        g = _fd_grad(lambda y: M.element(0, y, aux=aux)[0], x, eps=1e-8)
        np.testing.assert_allclose(f, -g, rtol=1e-6, atol=1e-9 * np.abs(f).max())


def test_membrane_hessian_matches_fd_in_tension():
    # biaxial tension + rotation: S is positive definite, no clamping, exact Hessian
    M = _mesh_one_triangle(REST_TRI)
    aux = _aux_tri(M)
    x = (REST_TRI * np.array([1.08, 1.05, 1.0])) @ _rot([1, 2, 3], 0.7).T
    _, _, H = M.element(0, x, aux=aux)
    Hfd = np.zeros((3, 3, 3, 3))
    eps = 1e-8
    for l in range(3):
        for b in range(3):
            xp, xm = x.copy(), x.copy()
            xp[l, b] += eps
            xm[l, b] -= eps
            df = (M.element(0, xp, aux=aux)[1] - M.element(0, xm, aux=aux)[1]) / (2 * eps)
            Hfd[:, l, :, b] = -df
    np.testing.assert_allclose(H, Hfd, rtol=1e-5, atol=1e-6 * np.abs(H).max())


def test_membrane_hessian_clamped_is_psd_under_compression():
    M = _mesh_one_triangle(REST_TRI)
    aux = _aux_tri(M)
    x = REST_TRI * np.array([0.8, 0.9, 1.0])
    _, _, H = M.element(0, x, aux=aux)
    Hm = H.transpose(0, 2, 1, 3).reshape(9, 9)
    np.testing.assert_allclose(Hm, Hm.T, atol=1e-12 * np.abs(Hm).max())
    assert np.linalg.eigvalsh(Hm).min() > -1e-9 * np.abs(Hm).max()
    # and the exact Hessian (FD) is indefinite there, so the clamp is doing work
    Hfd = np.zeros((9, 9))
    eps = 1e-8
    for j in range(9):
        xp, xm = x.copy().reshape(-1), x.copy().reshape(-1)
        xp[j] += eps
        xm[j] -= eps
        Hfd[:, j] = -(M.element(0, xp.reshape(3, 3), aux=aux)[1] - M.element(0, xm.reshape(3, 3), aux=aux)[1]).reshape(-1) / (2 * eps)
    assert np.linalg.eigvalsh(0.5 * (Hfd + Hfd.T)).min() < -1e-6 * np.abs(Hfd).max()


# ------------------------------------------------------------------------- bending

HINGE = np.array([[0.5, 1.0, 0.0], [0.5, -1.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])  # wings, edge


def test_hinge_angle_closed_form_fold():
    # rotate wing 0 about the edge (x axis) by phi: the dihedral angle is -phi with the
    # orientation convention of the oracle (lifting wing 0 gives a negative angle)
    for phi in (1e-4, 0.3, 1.2, 2.5):
        x = HINGE.copy()
        x[0] = [0.5, math.cos(phi), math.sin(phi)]
        th, _ = oracle.hinge_angle(*x)
        assert th == pytest.approx(-phi, rel=1e-12, abs=1e-15)
        x[0] = [0.5, math.cos(phi), -math.sin(phi)]
        th, _ = oracle.hinge_angle(*x)
        assert th == pytest.approx(phi, rel=1e-12)


def test_hinge_angle_gradient_matches_fd_and_is_translation_free():
    rng = np.random.default_rng(2)
    for trial in range(6):
        x = HINGE + 0.2 * rng.normal(size=(4, 3))
        th, g = oracle.hinge_angle(*x)
        gfd = _fd_grad(lambda y: oracle.hinge_angle(*y)[0], x, eps=1e-7)
        np.testing.assert_allclose(g, gfd, rtol=1e-6, atol=1e-8)
        assert np.abs(g.sum(0)).max() < 1e-12 * np.abs(g).max()
        # rotation about any axis leaves theta unchanged
        R = _rot(rng.normal(size=3), 0.9)
        assert oracle.hinge_angle(*(x @ R.T))[0] == pytest.approx(th, abs=1e-12)


def test_bending_energy_force_and_gauss_newton_hessian():
    M = _mesh_one_triangle(REST_TRI)  # material only
    kb = MAT[3]
    ch, th0 = 3.7, 0.1
    x = HINGE.copy()
    x[0] = [0.5, math.cos(0.4), -math.sin(0.4)]  # theta = 0.4
    E, f, H = M.element(1, x, aux=[ch, th0])
    assert E == pytest.approx(kb * ch * (0.4 - th0) ** 2, rel=1e-12)
    g = _fd_grad(lambda y: M.element(1, y, aux=[ch, th0])[0], x, eps=1e-7)
    np.testing.assert_allclose(f, -g, rtol=1e-6, atol=1e-12)
    th, dth = oracle.hinge_angle(*x)
    np.testing.assert_allclose(H, 2 * kb * ch * np.einsum("ka,lb->klab", dth, dth), rtol=1e-12, atol=1e-20)
    # at theta = theta_rest the Gauss-Newton Hessian is the exact Hessian
    E, f, H = M.element(1, x, aux=[ch, 0.4])
    Hfd = np.zeros((4, 4, 3, 3))
    eps = 1e-6
    for l in range(4):
        for b in range(3):
            xp, xm = x.copy(), x.copy()
            xp[l, b] += eps
            xm[l, b] -= eps
            Hfd[:, l, :, b] = -(M.element(1, xp, aux=[ch, 0.4])[1] - M.element(1, xm, aux=[ch, 0.4])[1]) / (2 * eps)
    np.testing.assert_allclose(H, Hfd, rtol=1e-5, atol=1e-7 * np.abs(H).max())


# ------------------------------------------------------------------------- contact

def test_contact_force_hessian_and_hold():
    M = _mesh_one_triangle(REST_TRI)
    kc = MAT[4]
    rng = np.random.default_rng(3)
    xt = np.array([[0.3, 0.3, 0.05], [0, 0, 0], [1, 0, 0.1], [0, 1, -0.05]]) + 0.01 * rng.normal(size=(4, 3))
    w = np.array([0.2, 0.5, 0.3])
    E, f, H = M.element(2, xt, xt, aux=w)
    assert abs(E) < 1e-20 and np.abs(f).max() < 1e-14  # d = d0 at x_t
    x = xt + 0.01 * rng.normal(size=(4, 3))
    E, f, H = M.element(2, x, xt, aux=w)
    g = _fd_grad(lambda y: M.element(2, y, xt, aux=w)[0], x, eps=1e-7)
    np.testing.assert_allclose(f, -g, rtol=1e-6, atol=1e-9)
    # frozen-frame penalty is quadratic: the FD Hessian is exact and equals kc (s s^T) x (n n^T)
    n = np.cross(xt[2] - xt[1], xt[3] - xt[1])
    n /= np.linalg.norm(n)
    s = np.array([1.0, -w[0], -w[1], -w[2]])
    np.testing.assert_allclose(H, kc * np.einsum("k,l,a,b->klab", s, s, n, n), rtol=1e-12, atol=1e-12)
    # the force is perpendicular to the partner plane and sums to zero
    assert np.abs(f.sum(0)).max() < 1e-10 * np.abs(f).max()
    assert np.abs(np.cross(f[0], n)).max() < 1e-10 * np.abs(f).max()


def test_gravity_and_lumped_mass():
    rest, tris, _ = wk.grid_piece(5, 4, 0.4, 0.3)
    M = oracle.Mesh(rest, tris, MAT)
    # total mass = density x area; each vertex gets a third of each incident triangle
    assert M.mass.sum() == pytest.approx(MAT[0] * 0.4 * 0.3, rel=1e-6)
    corner = M.mass[0]  # vertex (0,0) lies in both triangles of quad (0,0)
    inc = [t for t in range(M.T) if 0 in tris[t]]
    assert corner == pytest.approx(sum(MAT[0] * M.area[t] / 3 for t in inc), rel=1e-12)
    f = M.forces(rest)
    np.testing.assert_allclose(f, M.mass[:, None] * MAT[5:8][None, :], atol=1e-12)


# ------------------------------------------------------------------------- membrane clamp, mixed-sign stress
#
# Draped cloth is usually stretched one way and compressed the other, so the second
# Piola-Kirchhoff stress S has one positive and one negative principal value and the
# clamp keeps only the positive one. The exact Hessian (finite differences of the forces)
# contains the geometric term A0 (g_k . S g_l) I; the clamped one replaces S by its
# positive part. So the oracle's Hessian must equal H_fd + A0 (g_k . (S+ - S) g_l) I with
# S+ from numpy's symmetric eigendecomposition, S from the deformation gradient chosen
# here, and g the shape gradients of the rest triangle computed here.

def _stvk_stress(Fd):
    E_, nu = MAT[1], MAT[2]
    mu, lam = E_ / (2 * (1 + nu)), E_ * nu / (1 - nu * nu)
    G = 0.5 * (Fd.T @ Fd - np.eye(2))
    return 2 * mu * G + lam * np.trace(G) * np.eye(2)


def _positive_part(S):
    w, Q = np.linalg.eigh(S)
    return Q @ np.diag(np.maximum(w, 0.0)) @ Q.T


def _rot2(t):
    return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])


def _clamp_case(name):
    """Rest triangle in the xy plane with its first edge along +x (so the oracle's material
    frame is the world's x, y), an in-plane deformation Fd (2x2) and a rigid motion."""
    right = np.array([[0.0, 0.0], [0.012, 0.0], [0.0, 0.010]])
    general = np.array([[0.0, 0.0], [0.012, 0.0], [0.004, 0.010]])
    I3, zero = np.eye(3), np.zeros(3)
    if name == "axes-stretch-x":   # S diagonal (b = 0 exactly), stretch along the first axis: a >= c
        return right, np.diag([1.06, 0.95]), I3, zero
    if name == "axes-stretch-y":   # b = 0, stretch along the second axis: a < c
        return right, np.diag([0.95, 1.06]), I3, zero
    # principal axes at theta: the positive eigenvector is (cos theta, sin theta), so
    # |l1 - a| = (l1 - l2) sin^2 theta and |l1 - c| = (l1 - l2) cos^2 theta
    if name == "rotated-30deg":    # |l1 - a| < |l1 - c|
        Q = _rot2(math.radians(30))
        return general, Q @ np.diag([1.05, 0.94]) @ Q.T, _rot([0.3, -0.5, 0.8], 1.1), np.array([0.2, -0.7, 3.0])
    if name == "rotated-60deg":    # |l1 - a| > |l1 - c|
        Q = _rot2(math.radians(60))
        return general, Q @ np.diag([1.05, 0.94]) @ Q.T, _rot([-0.2, 0.9, 0.1], 2.3), np.array([-1.0, 0.4, 0.5])
    if name == "shear-rotation":   # non-symmetric Fd: a rotation inside the deformation gradient
        return general, _rot2(0.4) @ np.array([[1.04, 0.03], [-0.02, 0.955]]), _rot([1, 1, 0], 0.5), zero
    raise KeyError(name)


def _clamp_expectation(rest2d, Fd, S_plus):
    Dm = (rest2d[1:] - rest2d[0]).T                    # columns: the two rest edges
    g = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]]) @ np.linalg.inv(Dm)
    A0 = 0.5 * abs(np.linalg.det(Dm))
    corr = A0 * np.einsum("kc,cd,ld->kl", g, S_plus - _stvk_stress(Fd), g)
    return corr[:, :, None, None] * np.eye(3)[None, None]


def _fd_hessian(M, x, aux, eps=1e-8):
    Hfd = np.zeros((3, 3, 3, 3))
    for l in range(3):
        for b in range(3):
            xp, xm = x.copy(), x.copy()
            xp[l, b] += eps
            xm[l, b] -= eps
            Hfd[:, l, :, b] = -(M.element(0, xp, aux=aux)[1] - M.element(0, xm, aux=aux)[1]) / (2 * eps)
    return Hfd


@pytest.mark.parametrize("name", ["axes-stretch-x", "axes-stretch-y", "rotated-30deg", "rotated-60deg",
                                  "shear-rotation"])
def test_membrane_clamp_mixed_sign_matches_eigendecomposition(name):
    rest2d, Fd, R, t = _clamp_case(name)
    rest = np.c_[rest2d, np.zeros(3)]
    M = _mesh_one_triangle(rest)
    aux = _aux_tri(M)
    x = np.c_[rest2d @ Fd.T, np.zeros(3)] @ R.T + t
    S = _stvk_stress(Fd)
    lam = np.linalg.eigvalsh(S)
    assert lam[0] < 0.0 < lam[1], "the state must have one stretched and one compressed direction"
    a, b, c, l1 = S[0, 0], S[0, 1], S[1, 1], lam[1]
    if name.startswith("axes"):
        assert b == 0.0 and ((a >= c) == name.endswith("x"))
    elif name == "rotated-30deg":
        assert b != 0.0 and abs(l1 - a) < abs(l1 - c)
    elif name == "rotated-60deg":
        assert b != 0.0 and abs(l1 - a) > abs(l1 - c)
    _, _, H = M.element(0, x, aux=aux)
    Hfd = _fd_hessian(M, x, aux)
    want = Hfd + _clamp_expectation(rest2d, Fd, _positive_part(S))
    tol = 1e-6 * np.abs(H).max()
    np.testing.assert_allclose(H, want, rtol=1e-5, atol=tol)
    # the check is sensitive to the eigenvector: swapping its components (or keeping the
    # negative eigenvalue's vector) moves the Hessian by far more than the tolerance
    w, Q = np.linalg.eigh(S)
    v = Q[:, 1]
    for wrong in (np.array([v[1], v[0]]), Q[:, 0]):
        S_wrong = l1 * np.outer(wrong, wrong)
        bad = Hfd + _clamp_expectation(rest2d, Fd, S_wrong)
        assert np.abs(H - bad).max() > 100 * tol


def test_membrane_clamp_random_mixed_sign_states():
    rng = np.random.default_rng(7)
    rest2d = np.array([[0.0, 0.0], [0.012, 0.0], [0.004, 0.010]])
    M = _mesh_one_triangle(np.c_[rest2d, np.zeros(3)])
    aux = _aux_tri(M)
    done = 0
    while done < 12:
        Q = _rot2(rng.uniform(0, math.pi))
        Fd = _rot2(rng.uniform(-1, 1)) @ Q @ np.diag([rng.uniform(1.01, 1.1), rng.uniform(0.9, 0.99)]) @ Q.T
        S = _stvk_stress(Fd)
        lam = np.linalg.eigvalsh(S)
        if not (lam[0] < 0.0 < lam[1]):
            continue
        R = _rot(rng.normal(size=3), rng.normal())
        x = np.c_[rest2d @ Fd.T, np.zeros(3)] @ R.T + rng.normal(size=3)
        _, _, H = M.element(0, x, aux=aux)
        want = _fd_hessian(M, x, aux) + _clamp_expectation(rest2d, Fd, _positive_part(S))
        np.testing.assert_allclose(H, want, rtol=1e-5, atol=1e-6 * np.abs(H).max())
        done += 1
