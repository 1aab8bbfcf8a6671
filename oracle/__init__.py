"""ctypes wrapper of the FP64 CPU LDG oracle (``ldg_oracle.cpp``).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline import this package. It never imports the product package, and the
product never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldg_oracle.cpp")
_LIB = os.path.join(_HERE, "libldg_oracle.so")

POISSON, CONVDIFF, EULER, NS = 0, 1, 2, 3
(CASE_ZERO, CASE_SINSIN, CASE_EXPSIN, CASE_POLY2, CASE_LINEAR, CASE_VORTEX, CASE_CONST, CASE_ROTATION,
 CASE_CYLINDER, CASE_REST, CASE_CYLINDER_START) = range(11)

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", _LIB, _SRC])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _D, _I64,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.orc_create_curved.restype = ctypes.c_void_p
        L.orc_create_curved.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _D, _I64,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _D,
                                        ctypes.c_void_p]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_radd.argtypes = [ctypes.c_void_p, _D]
        L.orc_ndof.restype = ctypes.c_int64
        L.orc_ndof.argtypes = [ctypes.c_void_p]
        L.orc_set_time.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
        for name in ("orc_residual", "orc_q", "orc_mass"):
            getattr(L, name).argtypes = [ctypes.c_void_p, _D, _D]
        L.orc_residual_with_q.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.orc_jvp.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.orc_residual_some.argtypes = [ctypes.c_void_p, _D, ctypes.c_int64, _I64, _D]
        L.orc_jvp_some.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_int64, _I64, _D]
        L.orc_residual_complex.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.orc_jacobian_cs.argtypes = [ctypes.c_void_p, _D, _D]
        L.orc_project.argtypes = [ctypes.c_void_p, ctypes.c_double, _D]
        L.orc_interpolate.argtypes = [ctypes.c_void_p, ctypes.c_double, _D]
        L.orc_l2_error.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, _D, _D]
        L.orc_gmres.restype = ctypes.c_int
        L.orc_gmres.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), _D, ctypes.c_int]
        L.orc_newton.restype = ctypes.c_int
        L.orc_newton.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.orc_sizes.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 5
        L.orc_neighbours.argtypes = [ctypes.c_void_p, _I64]
        L.orc_ref_rules.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, _D]
        L.orc_basis.argtypes = [ctypes.c_void_p, ctypes.c_int64, _D, _D, _D]
    return _lib


class _Stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("gmres_iters", ctypes.c_int),
                ("jv_calls", ctypes.c_int), ("residual_calls", ctypes.c_int),
                ("r0", ctypes.c_double), ("rfinal", ctypes.c_double)]


def _p(a):
    return a.ctypes.data_as(_D)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


DIRK11, DIRK22, DIRK33, DIRK34 = 1, 2, 3, 4


def dirk_tableau(scheme):
    """Butcher tableaus (A, b, c) of singly diagonally implicit Runge-Kutta schemes:
    DIRK11 backward Euler; DIRK22 and DIRK33 the L-stable, stiffly accurate schemes
    of Alexander (1977), two stages order 2 and three stages order 3; DIRK34 the
    three-stage order-4 A-stable scheme of Crouzeix (1975). Each diagonal gamma is
    computed from its defining equation."""
    if scheme == DIRK11:
        return [[1.0]], [1.0], [1.0]
    if scheme == DIRK22:
        g = 1.0 - 1.0 / np.sqrt(2.0)                     # root of g^2 - 2 g + 1/2 in (0, 1)
        return [[g, 0.0], [1.0 - g, g]], [1.0 - g, g], [g, 1.0]
    if scheme == DIRK33:
        # gamma: the root in (1/3, 1/2) of g^3 - 3 g^2 + 3/2 g - 1/6 = 0
        lo, hi = 1.0 / 3.0, 0.5
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if (mid ** 3 - 3 * mid ** 2 + 1.5 * mid - 1.0 / 6.0) * (lo ** 3 - 3 * lo ** 2 + 1.5 * lo - 1.0 / 6.0) > 0:
                lo = mid
            else:
                hi = mid
        g = 0.5 * (lo + hi)
        t2 = (1.0 + g) / 2.0
        b1 = -(6 * g * g - 16 * g + 1) / 4.0
        b2 = (6 * g * g - 20 * g + 5) / 4.0
        return [[g, 0.0, 0.0], [t2 - g, g, 0.0], [b1, b2, g]], [b1, b2, g], [g, t2, 1.0]
    if scheme == DIRK34:
        g = np.cos(np.pi / 18.0) / np.sqrt(3.0) + 0.5
        d = 1.0 / (6.0 * (2.0 * g - 1.0) ** 2)
        return ([[g, 0.0, 0.0], [0.5 - g, g, 0.0], [2 * g, 1 - 4 * g, g]], [d, 1 - 2 * d, d],
                [g, 0.5, 1.0 - g])
    raise ValueError("unknown DIRK scheme")


class Oracle:
    """One LDG problem (mesh, p, quadrature, model) on the CPU in FP64."""

    def __init__(self, mesh, p: int, model: int, case: int, mu=(), nq1: int | None = None):
        if nq1 is None:
            nq1 = p + 2 if (model in (EULER, NS) or mesh.etype in (0, 3)) else p + 1
        self.mesh, self.p, self.nq1, self.model, self.case = mesh, p, nq1, model, case
        xyz = _c(mesh.xyz)
        vid = _c(mesh.vid, np.int64)
        mu = _c(np.asarray(mu, dtype=np.float64).reshape(-1))
        pg = int(getattr(mesh, "pg", 0) or 0)
        # wall marks (gas models) apply to affine and curved meshes alike
        bc = None if getattr(mesh, "bc", None) is None else np.ascontiguousarray(mesh.bc, dtype=np.uint8)
        if pg > 0 or bc is not None:
            xgeo = _c(mesh.xgeo) if pg > 0 else None
            self._keep = (xgeo, bc)
            self._h = lib().orc_create_curved(mesh.etype, p, nq1, mesh.n_elem, _p(xyz), vid.ctypes.data_as(_I64),
                                              model, case, len(mu), _p(mu) if len(mu) else None, pg,
                                              _p(xgeo) if pg > 0 else None,
                                              None if bc is None else bc.ctypes.data)
        else:
            self._h = lib().orc_create(mesh.etype, p, nq1, mesh.n_elem, _p(xyz), vid.ctypes.data_as(_I64),
                                       model, case, len(mu), _p(mu) if len(mu) else None)
        if not self._h:
            raise ValueError("oracle rejected the mesh")
        a = [ctypes.c_int() for _ in range(5)]
        lib().orc_sizes(self._h, *[ctypes.byref(x) for x in a])
        self.npe, self.ncu, self.nd, self.nqv, self.nfq = [x.value for x in a]
        self.ndof = int(lib().orc_ndof(self._h))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def set_time(self, scheme: int, t: float, dt: float, un=None, unm1=None):
        un = None if un is None else _c(un)
        unm1 = None if unm1 is None else _c(unm1)
        lib().orc_set_time(self._h, scheme, t, dt, _p(un) if un is not None else None,
                           _p(unm1) if unm1 is not None else None)

    def set_radd(self, radd=None):
        """A constant vector added to every later residual (None clears it)."""
        self._radd = None if radd is None else _c(radd)
        lib().orc_set_radd(self._h, _p(self._radd) if self._radd is not None else None)

    def dirk_step(self, u, t, dt, scheme, **newton_kw):
        """One DIRK step of M du/dt + R_s(u) = 0 from (t, u) to t + dt (Section 2.2 names
        DIRK as the paper's time scheme). Stage i solves
            M (U_i - u) / (dt a_ii) + R_s(U_i) + sum_{j<i} (a_ij / a_ii) R_s(U_j) = 0
        by Newton-GMRES (BDF1 residual with step dt a_ii at t + c_i dt, plus the constant
        sum), with R_s(U_j) the spatial residual of the converged stage. Stage slopes
        K_i = -M^{-1} R_s(U_i) follow from U_i = u + dt sum_{j<=i} a_ij K_j, and the step
        returns u + dt sum_i b_i K_i. Returns (u_new, total Newton stats)."""
        A, b, c = dirk_tableau(scheme)
        s = len(b)
        un = _c(u).copy()
        Rs, Ks = [], []
        Ui = un.copy()
        stats = {"newton_iters": 0, "gmres_iters": 0}
        for i in range(s):
            g = A[i][i]
            radd = np.zeros(self.ndof)
            for j in range(i):
                radd += (A[i][j] / g) * Rs[j]
            self.set_time(1, t + c[i] * dt, g * dt, un)
            self.set_radd(radd)
            Ui, rc, st = self.newton(Ui, **newton_kw)
            if rc != 0:
                raise RuntimeError(f"oracle DIRK stage {i} did not converge (rc {rc})")
            stats["newton_iters"] += st["newton_iters"]
            stats["gmres_iters"] += st["gmres_iters"]
            self.set_radd(None)
            self.set_time(0, t + c[i] * dt, 1.0)
            Rs.append(self.residual(Ui))
            k = (Ui - un) / (g * dt)
            for j in range(i):
                k -= (A[i][j] / g) * Ks[j]
            Ks.append(k)
        unew = un.copy()
        for i in range(s):
            unew += dt * b[i] * Ks[i]
        return unew, stats

    def residual(self, u):
        u = _c(u)
        r = np.empty(self.ndof)
        lib().orc_residual(self._h, _p(u), _p(r))
        return r

    def jvp(self, u, v):
        u, v = _c(u), _c(v)
        r = np.empty(self.ndof)
        lib().orc_jvp(self._h, _p(u), _p(v), _p(r))
        return r

    def residual_with_q(self, u, q):
        """R(u) of Eq. 1b with q given per element ([E][ncu][nd][npe]) instead of formed."""
        u, q = _c(u), _c(q)
        r = np.empty(self.ndof)
        lib().orc_residual_with_q(self._h, _p(u), _p(q), _p(r))
        return r

    def residual_some(self, u, elems):
        u = _c(u)
        el = _c(elems, np.int64)
        r = np.empty(len(el) * self.npe * self.ncu)
        lib().orc_residual_some(self._h, _p(u), len(el), el.ctypes.data_as(_I64), _p(r))
        return r.reshape(len(el), self.ncu, self.npe)

    def jvp_some(self, u, v, elems):
        u, v = _c(u), _c(v)
        el = _c(elems, np.int64)
        r = np.empty(len(el) * self.npe * self.ncu)
        lib().orc_jvp_some(self._h, _p(u), _p(v), len(el), el.ctypes.data_as(_I64), _p(r))
        return r.reshape(len(el), self.ncu, self.npe)

    def residual_complex(self, u, ui):
        u, ui = _c(u), _c(ui)
        rr, ri = np.empty(self.ndof), np.empty(self.ndof)
        lib().orc_residual_complex(self._h, _p(u), _p(ui), _p(rr), _p(ri))
        return rr + 1j * ri

    def jacobian_cs(self, u):
        u = _c(u)
        J = np.empty((self.ndof, self.ndof))
        lib().orc_jacobian_cs(self._h, _p(u), _p(J))
        return J

    def q(self, u):
        u = _c(u)
        q = np.empty(self.mesh.n_elem * self.ncu * self.nd * self.npe)
        lib().orc_q(self._h, _p(u), _p(q))
        return q

    def mass(self, u):
        u = _c(u)
        r = np.empty(self.ndof)
        lib().orc_mass(self._h, _p(u), _p(r))
        return r

    def project(self, t: float = 0.0):
        u = np.empty(self.ndof)
        lib().orc_project(self._h, t, _p(u))
        return u

    def interpolate(self, t: float = 0.0):
        u = np.empty(self.ndof)
        lib().orc_interpolate(self._h, t, _p(u))
        return u

    def l2_error(self, u, t: float = 0.0):
        u = _c(u)
        eu, eq = ctypes.c_double(), ctypes.c_double()
        lib().orc_l2_error(self._h, _p(u), t, ctypes.byref(eu), ctypes.byref(eq))
        return eu.value, eq.value

    def gmres(self, u, b, m=30, rtol=1e-10, maxit=1000):
        u, b = _c(u), _c(b)
        x = np.empty(self.ndof)
        its = ctypes.c_int()
        hist = np.zeros(maxit + 2)
        rc = lib().orc_gmres(self._h, _p(u), _p(b), _p(x), m, rtol, maxit, ctypes.byref(its), _p(hist),
                             len(hist))
        return x, its.value, rc, hist[: its.value + 1]

    def newton(self, u, m=30, newton_rtol=1e-8, gmres_rtol=1e-3, max_newton=20, max_gmres=2000):
        u = _c(u).copy()
        st = _Stats()
        rc = lib().orc_newton(self._h, _p(u), m, newton_rtol, gmres_rtol, max_newton, max_gmres,
                              ctypes.byref(st))
        return u, rc, {k: getattr(st, k) for k, _ in _Stats._fields_}

    def neighbours(self):
        nf = {0: 3, 1: 4, 2: 6, 3: 4}[self.mesh.etype]
        nb = np.empty(self.mesh.n_elem * nf, dtype=np.int64)
        lib().orc_neighbours(self._h, nb.ctypes.data_as(_I64))
        return nb.reshape(self.mesh.n_elem, nf)

    def ref_rules(self):
        nodes = np.empty((self.npe, 3))
        qx = np.empty((self.nqv, 3))
        qw = np.empty(self.nqv)
        fs = np.empty((self.nfq, 2))
        fw = np.empty(self.nfq)
        lib().orc_ref_rules(self._h, _p(nodes), _p(qx), _p(qw), _p(fs), _p(fw))
        return nodes, qx, qw, fs, fw

    def basis(self, xi):
        xi = _c(np.atleast_2d(xi))
        m = xi.shape[0]
        if xi.shape[1] < 3:
            xi = _c(np.hstack([xi, np.zeros((m, 3 - xi.shape[1]))]))
        phi = np.empty((m, self.npe))
        dphi = np.empty((m, self.npe, self.nd))
        lib().orc_basis(self._h, m, _p(xi), _p(phi), _p(dphi))
        return phi, dphi
