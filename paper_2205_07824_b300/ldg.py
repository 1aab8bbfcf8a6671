"""Python binding of the C-ABI in ``include/ldg.h`` (argument marshalling only).

Every computation runs in ``libldg.so``'s CUDA kernels; PyTorch only supplies
device memory and the stream. There is no CPU fallback: constructing a context
without the compiled library or without a CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libldg.so")

TRI, QUAD, HEX = 0, 1, 2
POISSON, CONVDIFF, EULER, NS = 0, 1, 2, 3
(CASE_ZERO, CASE_SINSIN, CASE_EXPSIN, CASE_POLY2, CASE_LINEAR, CASE_VORTEX, CASE_CONST, CASE_ROTATION,
 CASE_CYLINDER, CASE_REST, CASE_CYLINDER_START) = range(11)
STEADY, BDF1, BDF2 = 0, 1, 2
DIRK11, DIRK22, DIRK33, DIRK34 = 1, 2, 3, 4
FP64, FP32, F32X2 = 0, 1, 2
# tensor-core contractions (Euler on affine quadrilaterals): BF16 hi/lo splits, or one BF16 product
TC_BF16X3, TC_BF16 = 3, 4
PC_NONE, PC_BJACOBI, PC_MLP, PC_MLP_BJ, PC_RB_BJ = 0, 1, 2, 3, 4
FORCING_FIXED, FORCING_LAST = 0, 1
BASIS_FP64, BASIS_F32X2 = 0, 1
JV_AUTO, JV_STAGE = 0, 1
STAGE_R, STAGE_HOM = 0, 1
STATUS = {0: "LDG_OK", -1: "LDG_ERR_ARG", -2: "LDG_ERR_CUDA", -3: "LDG_ERR_UNSUPPORTED",
          -4: "LDG_ERR_NONFINITE", -5: "LDG_ERR_MAXIT", -6: "LDG_ERR_MESH"}


class LDGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Mesh(ctypes.Structure):
    _fields_ = [("elem_type", ctypes.c_int), ("n_elem", ctypes.c_int64),
                ("xyz", ctypes.POINTER(ctypes.c_double)), ("vid", ctypes.POINTER(ctypes.c_int64)),
                ("geom_order", ctypes.c_int), ("xgeo", ctypes.POINTER(ctypes.c_double)),
                ("bc", ctypes.POINTER(ctypes.c_uint8))]


def _mesh_desc(mesh, keep):
    """ldg_mesh_desc of a mesh (curved map points and wall marks when it has them);
    the arrays it points to are appended to ``keep``."""
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    vid = np.ascontiguousarray(mesh.vid, dtype=np.int64)
    keep += [xyz, vid]
    pg = int(getattr(mesh, "pg", 0) or 0)
    xgeo = bc = None
    if pg > 0:
        xgeo = np.ascontiguousarray(mesh.xgeo, dtype=np.float64)
        keep.append(xgeo)
    if getattr(mesh, "bc", None) is not None:
        bc = np.ascontiguousarray(mesh.bc, dtype=np.uint8)
        keep.append(bc)
    return _Mesh(mesh.etype, mesh.n_elem, xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 vid.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), pg,
                 xgeo.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if xgeo is not None else None,
                 bc.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if bc is not None else None)


class _Model(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("case_id", ctypes.c_int), ("n_mu", ctypes.c_int),
                ("mu", ctypes.POINTER(ctypes.c_double))]


class _Options(ctypes.Structure):
    _fields_ = [("nq1", ctypes.c_int), ("gmres_m", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("max_newton", ctypes.c_int), ("newton_rtol", ctypes.c_double), ("gmres_rtol", ctypes.c_double),
                ("krylov_precision", ctypes.c_int), ("precond", ctypes.c_int), ("pc_refresh", ctypes.c_int),
                ("newton_forcing", ctypes.c_int), ("pc_reuse", ctypes.c_int), ("krylov_basis", ctypes.c_int),
                ("jv_form", ctypes.c_int), ("rb_size", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("gmres_iters", ctypes.c_int), ("jv_calls", ctypes.c_int),
                ("residual_calls", ctypes.c_int), ("r0", ctypes.c_double), ("rfinal", ctypes.c_double),
                ("lin_resid", ctypes.c_double), ("elapsed_ms", ctypes.c_double), ("status", ctypes.c_int),
                ("pc_setups", ctypes.c_int), ("pc_fallbacks", ctypes.c_int), ("newton_backtracks", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("linear_init", ctypes.c_int)]


class TrainReport(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double), ("steps", ctypes.c_int),
                ("elapsed_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Loads ``libldg.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2205_07824_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p
        L.ldg_version.restype = ctypes.c_char_p
        L.ldg_kernel_launches.restype = ctypes.c_int64
        L.ldg_last_error.restype = ctypes.c_char_p
        L.ldg_last_error.argtypes = [vp]
        L.ldg_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Mesh), ctypes.c_int, ctypes.POINTER(_Model),
                                 ctypes.POINTER(_Options), vp]
        L.ldg_destroy.argtypes = [vp]
        L.ldg_set_stream.argtypes = [vp, vp]
        L.ldg_sizes.argtypes = [vp, i64p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]
        L.ldg_set_time.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.ldg_residual.argtypes = [vp, dp, dp]
        L.ldg_jvp.argtypes = [vp, dp, dp, dp]
        L.ldg_jvp_noalloc.argtypes = [vp, dp, dp, dp]
        L.ldg_jvp_prec.argtypes = [vp, ctypes.c_int, dp, dp, dp]
        L.ldg_jvp_after_residual.argtypes = [vp, ctypes.c_int, dp, dp, dp]
        L.ldg_jvp_fd.argtypes = [vp, ctypes.c_int, dp, dp, dp]
        L.ldg_dirk_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, ctypes.c_void_p]
        L.ldg_rb_set_basis.argtypes = [vp, dp, ctypes.c_int]
        L.ldg_rb_count.argtypes = [vp]
        L.ldg_wave_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, dp, dp, dp, ctypes.c_void_p]
        L.ldg_diag_blocks.argtypes = [vp, ctypes.c_int, dp, dp]
        L.ldg_precond_setup.argtypes = [vp, dp]
        L.ldg_precond_apply.argtypes = [vp, dp, dp]
        L.ldg_mlp_init.argtypes = [vp, ctypes.c_uint64]
        L.ldg_mlp_params.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), i64p]
        L.ldg_mlp_loss_grad.argtypes = [vp, dp, dp, dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]
        L.ldg_mlp_train.argtypes = [vp, dp, dp, dp, ctypes.c_int64, ctypes.POINTER(TrainOpts),
                                    ctypes.POINTER(TrainReport)]
        L.ldg_mlp_apply.argtypes = [vp, dp, dp, dp]
        L.ldg_newton_collect_updates.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(SolveReport)]
        L.ldg_halo_features.argtypes = [vp, dp, dp]
        L.ldg_q_stage.argtypes = [vp, ctypes.c_int, ctypes.c_int64, dp, dp]
        L.ldg_residual_stage.argtypes = [vp, ctypes.c_int, ctypes.c_int64, dp, dp, dp]
        L.ldg_shard_setup.argtypes = [vp, ctypes.c_int64, ctypes.c_void_p]
        L.ldg_shard_residual.argtypes = [vp, dp, dp]
        L.ldg_shard_jvp.argtypes = [vp, dp, dp]
        L.ldg_shard_gmres.argtypes = [vp, dp, dp, ctypes.POINTER(SolveReport)]
        L.ldg_mlp_bj_apply.argtypes = [vp, dp, dp]
        L.ldg_newton_gmres_collect.argtypes = [vp, dp, dp, dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(SolveReport)]
        L.ldg_q.argtypes = [vp, dp, dp]
        L.ldg_interpolate.argtypes = [vp, ctypes.c_double, dp]
        L.ldg_project.argtypes = [vp, ctypes.c_double, dp]
        L.ldg_jvp_host.argtypes = [vp, ctypes.c_int, dp, dp, dp]
        L.ldg_jvp_host_many.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p)]
        L.ldg_jv_describe.restype = ctypes.c_char_p
        L.ldg_jv_describe.argtypes = [vp, ctypes.c_int]
        L.ldg_l2_error.argtypes = [vp, dp, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
        L.ldg_gmres.argtypes = [vp, dp, dp, dp, ctypes.POINTER(SolveReport)]
        L.ldg_newton_gmres.argtypes = [vp, dp, ctypes.POINTER(SolveReport)]
        L.ldg_newton_gmres_host.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveReport)]
        ip = ctypes.POINTER(ctypes.c_int)
        L.ldg_autotune.argtypes = [vp, ctypes.c_int, ip, ctypes.POINTER(ctypes.c_double)]
        L.ldg_set_tile.argtypes = [vp, ctypes.c_int]
        L.ldg_get_tile.argtypes = [vp, ip, ip, ip, ip]
        L.ldg_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(_Mesh), ip,
                                       ctypes.POINTER(_Model), ctypes.POINTER(_Options), vp]
        L.ldg_batch_destroy.argtypes = [vp]
        L.ldg_batch_sizes.argtypes = [vp, i64p, i64p, i64p, ip]
        L.ldg_batch_residual.argtypes = [vp, dp, dp]
        L.ldg_batch_set_time.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.ldg_batch_jvp.argtypes = [vp, ctypes.c_int, dp, dp, dp]
        L.ldg_batch_autotune.argtypes = [vp, ctypes.c_int, ip]
        L.ldg_batch_solve.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(SolveReport), ctypes.POINTER(ctypes.c_double)]
        L.ldg_batch_kernel_executions.restype = ctypes.c_int64
        L.ldg_batch_kernel_executions.argtypes = [vp]
        L.ldg_batch_last_error.restype = ctypes.c_char_p
        L.ldg_batch_last_error.argtypes = [vp]
        _lib = L
    return _lib


def _ptr(t, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous float64 CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name}: needs {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def kernel_launches() -> int:
    """Kernels launched by libldg.so so far in this process."""
    return int(lib().ldg_kernel_launches())


class LDG:
    """One LDG operator (mesh, order p, model) resident on the current CUDA device.

    The keyword options mirror ``ldg_options`` in ``include/ldg.h``: solver sizes and
    tolerances, ``krylov_precision`` (FP64, FP32, F32X2, TC_BF16X3 or TC_BF16 Krylov J.v;
    FP32 preconditioner with FP32 and the tensor-core forms),
    ``precond`` (none, block-Jacobi, learned, reduced basis + block-Jacobi), ``rb_size``,
    ``pc_refresh``, and three solve policies
    that default to their plain form: ``newton_forcing`` (FORCING_LAST: a Newton step's
    linear solve stops at what the Newton tolerance still needs), ``pc_reuse`` (the
    block-Jacobi blocks are built every pc_reuse solve calls) and ``krylov_basis``
    (BASIS_F32X2: Gram-Schmidt on (hi, lo) float pairs, an emulated FP64). ``jv_form``
    (JV_STAGE) keeps the quadrature-point stage kernels for the J.v of linear models on
    affine quadrilaterals and hexahedra, which otherwise take the nodal kernels."""

    def __init__(self, mesh, p: int, model: int, case: int, mu=(), nq1: int = 0, gmres_m: int = 30,
                 max_restarts: int = 50, max_newton: int = 20, newton_rtol: float = 1e-8,
                 gmres_rtol: float = 1e-3, krylov_precision: int = 0, precond: int = 0, pc_refresh: int = 0,
                 newton_forcing: int = 0, pc_reuse: int = 1, krylov_basis: int = 0, jv_form: int = 0,
                 rb_size: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("LDG needs a CUDA device (no CPU fallback)")
        L = lib()
        self._xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        self._vid = np.ascontiguousarray(mesh.vid, dtype=np.int64)
        self._mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1))
        self._keep_mesh = []
        md = _mesh_desc(mesh, self._keep_mesh)
        mo = _Model(model, case, len(self._mu),
                    self._mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if len(self._mu) else None)
        op = _Options(nq1, gmres_m, max_restarts, max_newton, newton_rtol, gmres_rtol, krylov_precision, precond,
                      pc_refresh, newton_forcing, pc_reuse, krylov_basis, jv_form, rb_size)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = L.ldg_create(ctypes.byref(h), ctypes.byref(md), p, ctypes.byref(mo), ctypes.byref(op),
                          ctypes.c_void_p(stream.cuda_stream))
        self._h = h
        if rc != 0:
            msg = L.ldg_last_error(h).decode() if h.value else "invalid arguments"
            L.ldg_destroy(h)
            self._h = None
            raise LDGError(rc, msg)
        n, npe, ncu, dim = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.ldg_sizes(h, ctypes.byref(n), ctypes.byref(npe), ctypes.byref(ncu), ctypes.byref(dim))
        self.n_dof, self.n_pe, self.n_cu, self.dim = n.value, npe.value, ncu.value, dim.value
        self.n_elem, self.p, self.model = mesh.n_elem, p, model

    def close(self):
        if getattr(self, "_h", None):
            lib().ldg_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, rc):
        if rc != 0:
            raise LDGError(rc, lib().ldg_last_error(self._h).decode())

    # ------------------------------------------------------------- tiles
    def set_stream(self, stream):
        """Stream of all later launches of this context (a torch.cuda.Stream)."""
        self._check(lib().ldg_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def autotune(self, force: bool = False):
        """Times the compiled tiles on this mesh and keeps the fastest J.v; returns (tile, ms)."""
        t, ms = ctypes.c_int(), ctypes.c_double()
        self._check(lib().ldg_autotune(self._h, int(force), ctypes.byref(t), ctypes.byref(ms)))
        return t.value, ms.value

    def set_tile(self, tile: int):
        self._check(lib().ldg_set_tile(self._h, tile))

    def get_tile(self):
        """(tile, elements per CTA of the q-stage, residual and J.v kernels)."""
        v = [ctypes.c_int() for _ in range(4)]
        self._check(lib().ldg_get_tile(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def empty(self, n=None):
        import torch
        return torch.empty(self.n_dof if n is None else n, dtype=torch.float64, device="cuda")

    def set_time(self, scheme: int, t: float, dt: float = 1.0, un=None, unm1=None):
        n = self.n_dof
        self._check(lib().ldg_set_time(self._h, scheme, t, dt, _ptr(un, n, "un") if un is not None else None,
                                       _ptr(unm1, n, "unm1") if unm1 is not None else None))

    def residual(self, u, out=None):
        out = self.empty() if out is None else out
        self._check(lib().ldg_residual(self._h, _ptr(u, self.n_dof, "u"), _ptr(out, self.n_dof, "out")))
        return out

    def jvp(self, u, v, out=None):
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_jvp(self._h, _ptr(u, n, "u"), _ptr(v, n, "v"), _ptr(out, n, "out")))
        return out

    def jvp_prec(self, precision: int, u, v, out=None):
        """J.v in FP64 (precision FP64), FP32 (FP32), (hi, lo) float-pair arithmetic
        (F32X2, emulated FP64; the nodal kernels of the linear models only) or with the
        contractions on the tensor cores (TC_BF16X3 / TC_BF16; Euler on affine
        quadrilaterals); FP64 in memory."""
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_jvp_prec(self._h, precision, _ptr(u, n, "u"), _ptr(v, n, "v"), _ptr(out, n, "out")))
        return out

    def dirk_step(self, u, t: float, dt: float, scheme: int = 3, check=True):
        """One DIRK step in place from t to t + dt (scheme: DIRK11/22/33/34 = 1..4)."""
        rep = SolveReport()
        rc = lib().ldg_dirk_step(self._h, scheme, t, dt, _ptr(u, self.n_dof, "u"), ctypes.byref(rep))
        if check:
            self._check(rc)
        return rep.as_dict()

    def wave_step(self, u, q, w=None, t: float = 0.0, dt: float = 0.01, scheme: int = 3, alpha: float = 1.0,
                  beta: float = 0.0, check=True):
        """One DIRK step of the wave model in place (ldg_wave_step): u (n_dof), q (n_dof * dim)
        and optionally w (n_dof), from t to t + dt."""
        rep = SolveReport()
        n = self.n_dof
        rc = lib().ldg_wave_step(self._h, scheme, t, dt, alpha, beta, _ptr(u, n, "u"), _ptr(q, n * self.dim, "q"),
                                 None if w is None else _ptr(w, n, "w"), ctypes.byref(rep))
        if check:
            self._check(rc)
        return rep.as_dict()

    def rb_set_basis(self, W):
        """Replace the reduced basis of PC_RB_BJ by the rows of W ([k][n_dof] CUDA tensor)."""
        k = 0 if W is None else int(W.shape[0])
        ptr = None if k == 0 else _ptr(W, k * self.n_dof, "W")
        self._check(lib().ldg_rb_set_basis(self._h, ptr, k))

    def rb_count(self) -> int:
        """Vectors in the reduced basis now."""
        return int(lib().ldg_rb_count(self._h))

    def jvp_fd(self, u, v, order: int = 1, out=None):
        """Finite-difference J.v (order 1 forward, 2 central) from two FP64 residuals."""
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_jvp_fd(self._h, order, _ptr(u, n, "u"), _ptr(v, n, "v"), _ptr(out, n, "out")))
        return out

    def jvp_after_residual(self, precision: int, u, v, out=None):
        """J.v at the state of the last residual call, reusing its q(u) (Newton-Krylov form)."""
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_jvp_after_residual(self._h, precision, _ptr(u, n, "u"), _ptr(v, n, "v"),
                                                 _ptr(out, n, "out")))
        return out

    def diag_blocks(self, u, precision: int = 0, out=None):
        """Exact element-diagonal blocks of J(u), [n_elem][n_loc][n_loc] column-major per element."""
        nloc = self.n_cu * self.n_pe
        out = self.empty(self.n_elem * nloc * nloc) if out is None else out
        self._check(lib().ldg_diag_blocks(self._h, precision, _ptr(u, self.n_dof, "u"),
                                          _ptr(out, self.n_elem * nloc * nloc, "out")))
        return out

    def precond_setup(self, u):
        self._check(lib().ldg_precond_setup(self._h, _ptr(u, self.n_dof, "u")))

    def precond_apply(self, x, out=None):
        out = self.empty() if out is None else out
        self._check(lib().ldg_precond_apply(self._h, _ptr(x, self.n_dof, "x"), _ptr(out, self.n_dof, "out")))
        return out

    # ------------------------------------------------ learned preconditioner
    def mlp_init(self, seed: int = 0):
        self._check(lib().ldg_mlp_init(self._h, seed))

    def mlp_params(self, theta=None):
        """Get (theta None) or set the network parameters as an FP64 numpy vector."""
        cnt = ctypes.c_int64(0)
        self._check(lib().ldg_mlp_params(self._h, 1, None, ctypes.byref(cnt)))
        if theta is None:
            buf = np.empty(cnt.value)
            self._check(lib().ldg_mlp_params(self._h, 1, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             ctypes.byref(cnt)))
            return buf
        buf = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(lib().ldg_mlp_params(self._h, 0, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(cnt)))

    def mlp_loss_grad(self, X, T, U):
        n_pairs = X.numel() // (self.n_cu * self.n_pe)
        loss = ctypes.c_double()
        cnt = ctypes.c_int64(0)
        self._check(lib().ldg_mlp_params(self._h, 1, None, ctypes.byref(cnt)))
        g = np.empty(cnt.value)
        self._check(lib().ldg_mlp_loss_grad(self._h, _ptr(X, X.numel(), "X"), _ptr(T, T.numel(), "T"),
                                            _ptr(U, U.numel(), "U"), n_pairs,
                                            ctypes.byref(loss), g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return loss.value, g

    def mlp_train(self, X, T, U, epochs=50, batch=4096, lr=1e-3, seed=0, linear_init=True):
        n_pairs = X.numel() // (self.n_cu * self.n_pe)
        rep = TrainReport()
        o = TrainOpts(epochs, batch, lr, seed, int(linear_init))
        self._check(lib().ldg_mlp_train(self._h, _ptr(X, X.numel(), "X"), _ptr(T, T.numel(), "T"),
                                        _ptr(U, U.numel(), "U"), n_pairs, ctypes.byref(o), ctypes.byref(rep)))
        return rep.as_dict()

    def mlp_apply(self, u, x, out=None):
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_mlp_apply(self._h, _ptr(u, n, "u"), _ptr(x, n, "x"), _ptr(out, n, "out")))
        return out

    def newton_gmres_collect(self, u, X, T, U, capacity):
        """Block-Jacobi Newton-GMRES that also stores (v_j, M^-1 v_j, u) per Arnoldi vector into
        X, T, U [capacity][n_dof]."""
        rep = SolveReport()
        cnt = ctypes.c_int(0)
        n = self.n_dof
        self._check(lib().ldg_newton_gmres_collect(self._h, _ptr(u, n, "u"), _ptr(X, capacity * n, "X"),
                                                   _ptr(T, capacity * n, "T"), _ptr(U, capacity * n, "U"),
                                                   capacity, ctypes.byref(cnt), ctypes.byref(rep)))
        return cnt.value, rep.as_dict()

    def newton_collect_updates(self, u, X, T, U, capacity, which=1):
        """Block-Jacobi Newton-GMRES that stores (residual, update) pairs as features and
        targets ([capacity][n_dof] each): X = BJ^-1 r, U = its scaled neighbour traces, T = the
        update. which: 1 Newton steps (R(u_k), delta_k), 2 Arnoldi steps (J z_j, z_j), 3 both."""
        rep = SolveReport()
        cnt = ctypes.c_int(0)
        n = self.n_dof
        self._check(lib().ldg_newton_collect_updates(self._h, _ptr(u, n, "u"), _ptr(X, capacity * n, "X"),
                                                     _ptr(T, capacity * n, "T"), _ptr(U, capacity * n, "U"),
                                                     capacity, int(which), ctypes.byref(cnt), ctypes.byref(rep)))
        return cnt.value, rep.as_dict()

    def halo_features(self, z, out=None):
        """Neighbour traces of z at each element's face nodes, scaled by 1 / ||z_K||."""
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_halo_features(self._h, _ptr(z, n, "z"), _ptr(out, n, "out")))
        return out

    def mlp_bj_apply(self, x, out=None):
        """The learned block-Jacobi correction y = M(x) (after precond_setup)."""
        out = self.empty() if out is None else out
        n = self.n_dof
        self._check(lib().ldg_mlp_bj_apply(self._h, _ptr(x, n, "x"), _ptr(out, n, "out")))
        return out

    # ----------------------------------------------------- stages and sharded use
    def q_stage(self, mode: int, n_owned: int, u, out):
        """q of elements [0, n_owned) (``ldg_q_stage``; mode STAGE_R or STAGE_HOM)."""
        self._check(lib().ldg_q_stage(self._h, mode, n_owned, _ptr(u, self.n_dof, "u"),
                                      _ptr(out, self.n_dof * self.dim, "out")))
        return out

    def residual_stage(self, mode: int, n_owned: int, u, q, out):
        """R (STAGE_R) or the homogeneous J.v (STAGE_HOM) of elements [0, n_owned)."""
        qp = None if q is None else _ptr(q, self.n_dof * self.dim, "q")
        self._check(lib().ldg_residual_stage(self._h, mode, n_owned, _ptr(u, self.n_dof, "u"), qp,
                                             _ptr(out, self.n_dof, "out")))
        return out

    def shard_setup(self, n_owned: int, comm):
        """Element-sharded use: owned elements [0, n_owned) and an ``ldg_comm`` transport
        (``shard.make_comm``), which must stay alive as long as the context uses it."""
        self._comm = comm
        self._check(lib().ldg_shard_setup(self._h, n_owned, ctypes.byref(comm)))

    def shard_residual(self, u, out=None):
        out = self.empty() if out is None else out
        self._check(lib().ldg_shard_residual(self._h, _ptr(u, self.n_dof, "u"), _ptr(out, self.n_dof, "out")))
        return out

    def shard_jvp(self, v, out=None):
        out = self.empty() if out is None else out
        self._check(lib().ldg_shard_jvp(self._h, _ptr(v, self.n_dof, "v"), _ptr(out, self.n_dof, "out")))
        return out

    def shard_gmres(self, b, x=None):
        x = self.empty() if x is None else x
        rep = SolveReport()
        self._check(lib().ldg_shard_gmres(self._h, _ptr(b, self.n_dof, "b"), _ptr(x, self.n_dof, "x"),
                                          ctypes.byref(rep)))
        return x, rep.as_dict()

    def jvp_noalloc(self, u, v, out):
        """J.v through ldg_jvp_noalloc (static device scratch; no allocation in the call)."""
        n = self.n_dof
        self._check(lib().ldg_jvp_noalloc(self._h, _ptr(u, n, "u"), _ptr(v, n, "v"), _ptr(out, n, "out")))
        return out

    def q(self, u, out=None):
        out = self.empty(self.n_dof * self.dim) if out is None else out
        self._check(lib().ldg_q(self._h, _ptr(u, self.n_dof, "u"), _ptr(out, self.n_dof * self.dim, "out")))
        return out

    def interpolate(self, t: float = 0.0, out=None):
        out = self.empty() if out is None else out
        self._check(lib().ldg_interpolate(self._h, t, _ptr(out, self.n_dof, "out")))
        return out

    def jv_kernels(self, precision: int = 0) -> str:
        """The kernels that form this operator's J.v in `precision` (``ldg_jv_describe``)."""
        return lib().ldg_jv_describe(self._h, int(precision)).decode()

    def _host_ptr(self, a, name):
        if a is None:
            return None
        ok = a.dtype == np.float64 and a.size == self.n_dof if isinstance(a, np.ndarray) else \
            (not a.is_cuda and str(a.dtype) == "torch.float64" and a.numel() == self.n_dof and a.is_contiguous())
        if not ok or (isinstance(a, np.ndarray) and not a.flags.c_contiguous):
            raise TypeError(f"{name}: expected a contiguous float64 host array of n_dof elements")
        return ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())

    def jvp_host(self, precision, u, v, out):
        """J(u) v with HOST buffers (``ldg_jvp_host``): u (or None for linear models), v and
        out are contiguous float64 numpy arrays or CPU tensors of n_dof entries."""
        hp = self._host_ptr
        self._check(lib().ldg_jvp_host(self._h, int(precision), hp(u, "u"), hp(v, "v"), hp(out, "out")))
        return out

    def jvp_host_many(self, precision, u, vs, outs):
        """J(u) v_i for a sequence of directions in HOST memory (``ldg_jvp_host_many``): the
        copies of each direction run beside the J.v of its neighbours. vs and outs are
        equal-length sequences of contiguous float64 host arrays (numpy or CPU tensors,
        pinned for the overlap); an output must not be the input of a later direction."""
        if len(vs) != len(outs) or not vs:
            raise ValueError("vs and outs: equal, non-zero lengths")
        k = len(vs)
        pv = (ctypes.c_void_p * k)(*[self._host_ptr(v, "v") for v in vs])
        po = (ctypes.c_void_p * k)(*[self._host_ptr(o, "out") for o in outs])
        self._check(lib().ldg_jvp_host_many(self._h, int(precision), self._host_ptr(u, "u"), k, pv, po))
        return outs

    def project(self, t: float = 0.0, out=None):
        """L2 projection of the analytic case at time t (``ldg_project``)."""
        out = self.empty() if out is None else out
        self._check(lib().ldg_project(self._h, t, _ptr(out, self.n_dof, "out")))
        return out

    def l2_error(self, u, t: float = 0.0):
        """Relative L2 errors (E(u_h), E(q_h)) against the analytic case (``ldg_l2_error``)."""
        eu, eq = ctypes.c_double(), ctypes.c_double()
        self._check(lib().ldg_l2_error(self._h, _ptr(u, self.n_dof, "u"), t, ctypes.byref(eu), ctypes.byref(eq)))
        return eu.value, eq.value

    def gmres(self, u, b, x=None):
        x = self.empty() if x is None else x
        rep = SolveReport()
        n = self.n_dof
        rc = lib().ldg_gmres(self._h, _ptr(u, n, "u"), _ptr(b, n, "b"), _ptr(x, n, "x"), ctypes.byref(rep))
        self._check(rc)
        return x, rep.as_dict()

    def newton_gmres(self, u, check=True):
        rep = SolveReport()
        rc = lib().ldg_newton_gmres(self._h, _ptr(u, self.n_dof, "u"), ctypes.byref(rep))
        if check:
            self._check(rc)
        return rep.as_dict()

    def newton_gmres_host(self, u: np.ndarray, check=True):
        if u.dtype != np.float64 or not u.flags.c_contiguous or u.size < self.n_dof:
            raise TypeError("u: expected a contiguous float64 numpy array of n_dof elements")
        rep = SolveReport()
        rc = lib().ldg_newton_gmres_host(self._h, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(rep))
        if check:
            self._check(rc)
        return rep.as_dict()


class Batch:
    """Many independent steady problems (per-instance mesh, order p and parameters mu)
    solved together; see the batched section of ``include/ldg.h``.

    meshes: list of synth.Mesh; ps: orders; mus: per-instance parameter sequences;
    cases: per-instance analytic case (int or list). The batch vector is one float64
    CUDA tensor of ``n_total`` entries; instance i is ``u[offsets[i]:offsets[i] + n_dof[i]]``.
    The solver options are those of ``LDG`` (``pc_refresh`` aside); the forcing term is
    applied per instance.
    """

    def __init__(self, meshes, ps, model: int, cases, mus, nq1: int = 0, gmres_m: int = 30,
                 max_restarts: int = 50, max_newton: int = 20, newton_rtol: float = 1e-8,
                 gmres_rtol: float = 1e-3, krylov_precision: int = 0, precond: int = 0, newton_forcing: int = 0,
                 pc_reuse: int = 1, krylov_basis: int = 0, jv_form: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device (no CPU fallback)")
        L = lib()
        n = len(meshes)
        if isinstance(cases, int):
            cases = [cases] * n
        self._keep = []
        md = (_Mesh * n)()
        mo = (_Model * n)()
        for i, m in enumerate(meshes):
            xyz = np.ascontiguousarray(m.xyz, dtype=np.float64)
            vid = np.ascontiguousarray(m.vid, dtype=np.int64)
            mu = np.ascontiguousarray(np.asarray(mus[i], dtype=np.float64).reshape(-1))
            self._keep += [xyz, vid, mu]
            md[i] = _mesh_desc(m, self._keep)
            mo[i] = _Model(model, int(cases[i]), len(mu),
                           mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if len(mu) else None)
        pa = (ctypes.c_int * n)(*[int(p) for p in ps])
        op = _Options(nq1, gmres_m, max_restarts, max_newton, newton_rtol, gmres_rtol, krylov_precision, precond, 0,
                      newton_forcing, pc_reuse, krylov_basis, jv_form, 0)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = L.ldg_batch_create(ctypes.byref(h), n, md, pa, mo, ctypes.byref(op), ctypes.c_void_p(stream.cuda_stream))
        self._h = h
        if rc != 0:
            msg = L.ldg_batch_last_error(h).decode() if h.value else "invalid arguments"
            L.ldg_batch_destroy(h)
            self._h = None
            raise LDGError(rc, msg)
        tot = ctypes.c_int64()
        off = (ctypes.c_int64 * n)()
        nd = (ctypes.c_int64 * n)()
        ng = ctypes.c_int()
        L.ldg_batch_sizes(h, ctypes.byref(tot), off, nd, ctypes.byref(ng))
        self.n_inst, self.n_total, self.n_groups = n, tot.value, ng.value
        self.offsets, self.n_dof = list(off), list(nd)

    def close(self):
        if getattr(self, "_h", None):
            lib().ldg_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, rc):
        if rc != 0:
            raise LDGError(rc, lib().ldg_batch_last_error(self._h).decode())

    def empty(self):
        import torch
        return torch.empty(self.n_total, dtype=torch.float64, device="cuda")

    def slice(self, u, i):
        return u[self.offsets[i]:self.offsets[i] + self.n_dof[i]]

    def set_time(self, scheme: int, t: float, dt: float = 1.0, un=None, unm1=None):
        n = self.n_total
        self._check(lib().ldg_batch_set_time(self._h, scheme, t, dt,
                                             _ptr(un, n, "un") if un is not None else None,
                                             _ptr(unm1, n, "unm1") if unm1 is not None else None))

    def residual(self, u, out=None):
        out = self.empty() if out is None else out
        n = self.n_total
        self._check(lib().ldg_batch_residual(self._h, _ptr(u, n, "u"), _ptr(out, n, "out")))
        return out

    def jvp(self, u, v, precision: int = 0, out=None):
        out = self.empty() if out is None else out
        n = self.n_total
        self._check(lib().ldg_batch_jvp(self._h, precision, _ptr(u, n, "u"), _ptr(v, n, "v"), _ptr(out, n, "out")))
        return out

    def autotune(self, force: bool = False):
        tiles = (ctypes.c_int * self.n_groups)()
        self._check(lib().ldg_batch_autotune(self._h, int(force), tiles))
        return list(tiles)

    def solve(self, u, use_graph: bool = True, check: bool = True):
        """Newton-GMRES of every instance in place; returns (reports, elapsed_ms)."""
        reps = (SolveReport * self.n_inst)()
        ms = ctypes.c_double()
        rc = lib().ldg_batch_solve(self._h, _ptr(u, self.n_total, "u"), int(use_graph), reps, ctypes.byref(ms))
        if check:
            self._check(rc)
        return [r.as_dict() for r in reps], ms.value

    def kernel_executions(self) -> int:
        return int(lib().ldg_batch_kernel_executions(self._h))
