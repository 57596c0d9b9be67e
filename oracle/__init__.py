"""FP64 CPU oracle for the implicit-integrator hot path (Sec. 2.5 Eq. 1-3, Sec. 3.2).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The CUDA library never
imports, links or calls anything here, and nothing here calls the CUDA library.

The arithmetic lives in ``pcloth_oracle.c`` (plain C, double precision); this module
compiles it with gcc on first use and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcloth_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpcloth_oracle.so")
_lock = threading.Lock()
_lib = None

OM_OK, OM_ERR_ARG, OM_ERR_PATTERN, OM_ERR_CAPACITY, OM_ERR_NOT_CONVERGED = 0, -1, -2, -3, -4

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (plain -O2, no fast-math, no -march; OpenMP
    spreads the product's rows and the solver's vector loops over the host cores)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def num_threads() -> int:
    """Threads the oracle's parallel loops use (OMP_NUM_THREADS, else every core)."""
    return int(lib().om_num_threads())


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.om_mesh_create.restype = ctypes.c_void_p
        L.om_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, _i, _d, _d, ctypes.c_int, _i]
        L.om_mesh_destroy.argtypes = [ctypes.c_void_p]
        L.om_mesh_num_hinges.argtypes = [ctypes.c_void_p]
        L.om_mesh_get.argtypes = [ctypes.c_void_p, _d, _d, _d, _i, _d, _d]
        L.om_energy.restype = ctypes.c_double
        L.om_energy.argtypes = [ctypes.c_void_p, _d, ctypes.c_int, _i, _d, _d]
        L.om_forces.argtypes = [ctypes.c_void_p, _d, ctypes.c_int, _i, _d, _d, _d]
        L.om_pattern.restype = ctypes.c_long
        L.om_pattern.argtypes = [ctypes.c_void_p, ctypes.c_int, _i, _i, _i, ctypes.c_long]
        L.om_hessian.argtypes = [ctypes.c_void_p, _d, ctypes.c_int, _i, _d, _d, _i, _i, _d]
        L.om_assemble.argtypes = [ctypes.c_void_p, _d, _d, ctypes.c_int, _i, _d, ctypes.c_double, ctypes.c_int,
                                  _i, _i, _d, _d]
        L.om_matfree_apply.argtypes = [ctypes.c_void_p, _d, ctypes.c_int, _i, _d, ctypes.c_double, _d, _d]
        L.om_element.restype = ctypes.c_double
        L.om_element.argtypes = [ctypes.c_void_p, ctypes.c_int, _d, _d, _d, _d, _d]
        L.om_hinge_angle.restype = ctypes.c_double
        L.om_hinge_angle.argtypes = [_d, _d, _d, _d, _d]
        L.om_spmv.argtypes = [ctypes.c_int, _i, _i, _d, _d, _d]
        L.om_pcg.argtypes = [ctypes.c_int, _i, _i, _d, _d, _d, ctypes.c_double, ctypes.c_int, _d]
        L.om_num_threads.restype = ctypes.c_int
        L.om_num_threads.argtypes = []
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _pd(a):
    return a.ctypes.data_as(_d) if a is not None else None


def _pi(a):
    return a.ctypes.data_as(_i) if a is not None else None


class OracleError(RuntimeError):
    pass


class Mesh:
    """Rest state of one cloth: lumped masses, rest edge matrices, hinges (FP64)."""

    def __init__(self, rest, tris, material, pins=()):
        self.rest = _f64(rest).reshape(-1, 3)
        self.tris = _i32(tris).reshape(-1, 3)
        m = _f64(material).reshape(-1)
        # {rho, E, nu, kb, kc, g[3]}, optionally the Rayleigh damping pair (alpha, beta) and
        # the contact thickness delta (zeros when absent)
        self.material = np.concatenate([m, np.zeros(max(0, 11 - m.size))])[:11].copy()
        self.pins = _i32(pins).reshape(-1)
        self.V = self.rest.shape[0]
        self.T = self.tris.shape[0]
        self._h = lib().om_mesh_create(self.V, self.T, _pi(self.tris), _pd(self.rest), _pd(self.material),
                                       int(self.pins.size), _pi(self.pins))
        if not self._h:
            raise OracleError("invalid mesh (index out of range, degenerate triangle or non-manifold edge)")
        self.H = lib().om_mesh_num_hinges(self._h)
        self.mass = np.zeros(self.V)
        self.Dminv = np.zeros((self.T, 4))
        self.area = np.zeros(self.T)
        self.hinges = np.zeros((max(self.H, 1), 4), np.int32)[: self.H]
        self.hcoef = np.zeros(self.H)
        self.hrest = np.zeros(self.H)
        hb = np.zeros((max(self.H, 1), 4), np.int32)
        lib().om_mesh_get(self._h, _pd(self.mass), _pd(self.Dminv), _pd(self.area), _pi(hb), _pd(self.hcoef),
                          _pd(self.hrest))
        self.hinges = hb[: self.H].copy()
        self.pinned = np.zeros(self.V, bool)
        self.pinned[self.pins] = True

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.om_mesh_destroy(h)
            self._h = None

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.rest, wl.tris, wl.material.as_array(), wl.pins)

    # -- energy and forces ------------------------------------------------------------
    @staticmethod
    def _contacts(pairs, w):
        pairs = _i32(pairs if pairs is not None else np.zeros((0, 4))).reshape(-1, 4)
        w = _f64(w if w is not None else np.zeros((0, 3))).reshape(-1, 3)
        return pairs, w

    def energy(self, x, pairs=None, w=None, xt=None) -> float:
        pairs, w = self._contacts(pairs, w)
        x = _f64(x).reshape(-1, 3)
        xt = x if xt is None else _f64(xt).reshape(-1, 3)
        return lib().om_energy(self._h, _pd(x), len(pairs), _pi(pairs), _pd(w), _pd(xt))

    def forces(self, x, pairs=None, w=None, xt=None) -> np.ndarray:
        pairs, w = self._contacts(pairs, w)
        x = _f64(x).reshape(-1, 3)
        xt = x if xt is None else _f64(xt).reshape(-1, 3)
        f = np.zeros((self.V, 3))
        st = lib().om_forces(self._h, _pd(x), len(pairs), _pi(pairs), _pd(w), _pd(xt), _pd(f))
        if st:
            raise OracleError(f"om_forces: {st}")
        return f

    # -- pattern and assembly ---------------------------------------------------------
    def pattern(self, pairs=None):
        pairs, _ = self._contacts(pairs, None)
        rp = np.zeros(self.V + 1, np.int32)
        ci = np.zeros(1, np.int32)
        n = lib().om_pattern(self._h, len(pairs), _pi(pairs), _pi(rp), _pi(ci), 0)
        if n < 0:
            raise OracleError(f"om_pattern: {n}")
        ci = np.zeros(max(n, 1), np.int32)
        n2 = lib().om_pattern(self._h, len(pairs), _pi(pairs), _pi(rp), _pi(ci), n)
        assert n2 == n
        return rp, ci[:n]

    def hessian(self, x, pairs=None, w=None, xt=None, pattern=None):
        pairs, w = self._contacts(pairs, w)
        x = _f64(x).reshape(-1, 3)
        xt = x if xt is None else _f64(xt).reshape(-1, 3)
        rp, ci = pattern if pattern is not None else self.pattern(pairs)
        vals = np.zeros((len(ci), 3, 3))
        st = lib().om_hessian(self._h, _pd(x), len(pairs), _pi(pairs), _pd(w), _pd(xt), _pi(rp), _pi(ci), _pd(vals))
        if st:
            raise OracleError(f"om_hessian: {st}")
        return rp, ci, vals

    def assemble(self, x, v, pairs=None, w=None, h=1.0 / 200.0, pins=True, pattern=None):
        """Eq. 3 system: A = M + h^2 K(x_t), b = h (f(x_t) - h K(x_t) v_t) (the first-order
        expansion of h f(x_t + h v_t), Eq. 2), with the pin rule. With Rayleigh damping
        (alpha, beta) in the material: A = (1 + h alpha) M + h (h + beta) K,
        b = h (f(x_t) - alpha M v_t - (h + beta) K v_t)."""
        pairs, w = self._contacts(pairs, w)
        x = _f64(x).reshape(-1, 3)
        v = _f64(v).reshape(-1, 3)
        rp, ci = pattern if pattern is not None else self.pattern(pairs)
        vals = np.zeros((len(ci), 3, 3))
        b = np.zeros((self.V, 3))
        st = lib().om_assemble(self._h, _pd(x), _pd(v), len(pairs), _pi(pairs), _pd(w), float(h), int(bool(pins)),
                               _pi(rp), _pi(ci), _pd(vals), _pd(b))
        if st:
            raise OracleError(f"om_assemble: {st}")
        return rp, ci, vals, b

    def matfree_apply(self, x, p, pairs=None, w=None, h=1.0 / 200.0):
        pairs, w = self._contacts(pairs, w)
        x = _f64(x).reshape(-1, 3)
        p = _f64(p).reshape(-1, 3)
        y = np.zeros((self.V, 3))
        st = lib().om_matfree_apply(self._h, _pd(x), len(pairs), _pi(pairs), _pd(w), float(h), _pd(p), _pd(y))
        if st:
            raise OracleError(f"om_matfree_apply: {st}")
        return y

    def element(self, kind: int, x, xt=None, aux=()):
        """One element: kind 0 membrane, 1 bending, 2 contact. Returns (E, f, H)."""
        n = 3 if kind == 0 else 4
        x = _f64(x).reshape(n, 3)
        xt = x if xt is None else _f64(xt).reshape(n, 3)
        aux = _f64(aux)
        f = np.zeros((n, 3))
        H = np.zeros((n, n, 3, 3))
        E = lib().om_element(self._h, kind, _pd(x), _pd(xt), _pd(aux), _pd(f), _pd(H))
        return E, f, H

    # -- one time step ----------------------------------------------------------------
    def step(self, x, v, pairs=None, w=None, h=1.0 / 200.0, tol=1e-12, max_iter=100000, dv0=None):
        """Assemble Eq. 3, solve it with Jacobi-PCG, then v += dv, x += h v."""
        rp, ci, vals, b = self.assemble(x, v, pairs, w, h)
        dv, it, rel = pcg(rp, ci, vals, b, dv0, tol=tol, max_iter=max_iter)
        v1 = _f64(v).reshape(-1, 3) + dv
        x1 = _f64(x).reshape(-1, 3) + h * v1
        return dv, x1, v1, {"iters": it, "rel_res": rel, "nnzb": len(ci)}


def hinge_angle(x1, x2, x3, x4):
    g = np.zeros(12)
    th = lib().om_hinge_angle(_pd(_f64(x1)), _pd(_f64(x2)), _pd(_f64(x3)), _pd(_f64(x4)), _pd(g))
    return th, g.reshape(4, 3)


def spmv(rp, ci, vals, x) -> np.ndarray:
    rp, ci = _i32(rp), _i32(ci)
    vals = _f64(vals)
    x = _f64(x).reshape(-1, 3)
    V = len(rp) - 1
    y = np.zeros((V, 3))
    lib().om_spmv(V, _pi(rp), _pi(ci), _pd(vals), _pd(x), _pd(y))
    return y


def pcg(rp, ci, vals, b, x0=None, tol=1e-12, max_iter=100000, check=True):
    """Jacobi-PCG; returns (x, iterations, true relative residual). Raises if not
    converged within max_iter (unless check is False: then the last iterate returns)."""
    rp, ci = _i32(rp), _i32(ci)
    vals = _f64(vals)
    b = _f64(b).reshape(-1, 3)
    V = len(rp) - 1
    x = np.zeros((V, 3)) if x0 is None else _f64(x0).reshape(-1, 3).copy()
    info = np.zeros(2)
    st = lib().om_pcg(V, _pi(rp), _pi(ci), _pd(vals), _pd(b), _pd(x), float(tol), int(max_iter), _pd(info))
    if st == OM_ERR_NOT_CONVERGED and check:
        raise OracleError(f"om_pcg: not converged after {int(info[0])} iterations (rel res {info[1]:.3e})")
    return x, int(info[0]), float(info[1])


def dense(rp, ci, vals) -> np.ndarray:
    """Dense 3V x 3V matrix of a BSR3x3 (tests on tiny meshes)."""
    V = len(rp) - 1
    A = np.zeros((3 * V, 3 * V))
    vals = np.asarray(vals).reshape(-1, 3, 3)
    for r in range(V):
        for s in range(rp[r], rp[r + 1]):
            c = ci[s]
            A[3 * r:3 * r + 3, 3 * c:3 * c + 3] = vals[s]
    return A
