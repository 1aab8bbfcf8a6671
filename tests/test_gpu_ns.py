"""Compressible Navier-Stokes (Section 2.1) on the GPU against the FP64 CPU oracle.

The residual and the exact J.v (dual numbers through u and through q = -grad u,
whose tangent is the homogeneous q-stage of the direction) meet the FP64 parity
bar on periodic and far-field meshes, with the BDF2 time terms, for p = 1..4 and
every tile; the FP32 J.v sits at FP32 round-off; the allocation-free J.v is the
same product bit for bit; the element-diagonal blocks from coloured probing equal
the oracle's complex-step Jacobian; BDF2 Newton-GMRES steps of the viscous vortex
reach the Newton tolerance when the oracle recomputes the residual, and the
batched solver gives the single-context solution."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu

MU = (1.4, 10.0, 0.72)


def _box(n, periodic=True, affine=SHEAR2):
    return synth.quad_box(n, hi=(10.0, 10.0), periodic=(periodic, periodic), affine=affine)


def _r_jv(mesh, p, case, mu=MU, seed=1, bdf=False):
    o, g = pair(mesh, p, oracle.NS, case, mu=mu)
    u = synth.random_euler_state(mesh.n_elem, o.npe, seed)
    v = synth.random_vector(o.ndof, seed + 100)
    if bdf:
        un = synth.random_euler_state(mesh.n_elem, o.npe, seed + 1)
        unm1 = synth.random_euler_state(mesh.n_elem, o.npe, seed + 2)
        o.set_time(2, 0.3, 0.05, un, unm1)
        g.set_time(2, 0.3, 0.05, cuda(un), cuda(unm1))
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what=f"R p={p}")
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what=f"J.v p={p}")
    return o, g, u, v


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_periodic_vortex(p):
    # 7 x 5 elements: several CTA tiles with a ragged last one
    _r_jv(_box((7, 5)), p, oracle.CASE_VORTEX)


@pytest.mark.parametrize("p,case", [(2, oracle.CASE_VORTEX), (3, oracle.CASE_ROTATION)])
def test_far_field_boundaries(p, case):
    mesh = synth.quad_box((5, 4), affine=SHEAR2) if case == oracle.CASE_ROTATION else _box((5, 4), periodic=False)
    _r_jv(mesh, p, case)


def test_bdf2_time_terms_and_penalty():
    _r_jv(_box((4, 6)), 3, oracle.CASE_VORTEX, mu=(1.3, 50.0, 0.9, 0.2), bdf=True)


def test_every_tile_and_noalloc():
    mesh = _box((6, 5))
    o, g, u, v = _r_jv(mesh, 2, oracle.CASE_VORTEX)
    ref = o.jvp(u, v)
    for t in range(4):
        g.set_tile(t)
        assert g.get_tile()[0] == t
        assert_parity(host(g.residual(cuda(u))), o.residual(u), what=f"R tile {t}")
        assert_parity(host(g.jvp(cuda(u), cuda(v))), ref, what=f"J.v tile {t}")
    g.set_tile(0)
    jv = host(g.jvp(cuda(u), cuda(v)))
    out = cuda(np.zeros(o.ndof))
    g.jvp_noalloc(cuda(u), cuda(v), out)
    assert np.array_equal(host(out), jv)
    # the Newton-Krylov form: q(u) of the last residual reused
    cu = cuda(u)
    g.residual(cu)
    assert np.array_equal(host(g.jvp_after_residual(0, cu, cuda(v))), jv)


def test_fp32_jvp_error():
    mesh = _box((8, 7))
    o, g = pair(mesh, 3, oracle.NS, oracle.CASE_VORTEX, mu=MU)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 1)
    v = synth.random_vector(o.ndof, 2)
    ref = o.jvp(u, v)
    err = np.linalg.norm(host(g.jvp_prec(1, cuda(u), cuda(v))) - ref) / np.linalg.norm(ref)
    print(f"NS FP32 J.v relative error vs FP64 oracle: {err:.2e}")
    assert 1e-10 < err < 2e-5
    # the FP32 J.v reads FP32 copies of u and q(u) written by the residual's q-stage: after a
    # residual at u it gives bitwise the J.v that forms q(u) itself
    jv32 = host(g.jvp_prec(1, cuda(u), cuda(v)))
    cu = cuda(u)
    g.residual(cu)
    assert np.array_equal(host(g.jvp_after_residual(1, cu, cuda(v))), jv32)


def test_diag_blocks_match_complex_step_jacobian():
    mesh = _box((4, 5))
    o, g = pair(mesh, 2, oracle.NS, oracle.CASE_VORTEX, mu=MU)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 5)
    o.set_time(2, 0.1, 0.05, u, u)
    g.set_time(2, 0.1, 0.05, cuda(u), cuda(u))
    nloc = o.npe * o.ncu
    J = o.jacobian_cs(u)
    ref = np.stack([J[e * nloc:(e + 1) * nloc, e * nloc:(e + 1) * nloc] for e in range(mesh.n_elem)])
    blk = host(g.diag_blocks(cuda(u))).reshape(mesh.n_elem, nloc, nloc)
    assert_parity(blk.transpose(0, 2, 1), ref, what="NS diag blocks")
    blk32 = host(g.diag_blocks(cuda(u), precision=1)).reshape(mesh.n_elem, nloc, nloc)
    assert np.linalg.norm(blk32.transpose(0, 2, 1) - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("kprec", [0, 1])
def test_newton_bdf2_block_jacobi(kprec):
    """Two BDF2 steps of the vortex at Re = 100, p = 3, with block-Jacobi; the oracle's
    residual at the GPU solution meets the Newton tolerance and the oracle's own
    Newton solve gives the same state."""
    mesh = _box(12, affine=None)
    mu = (1.4, 100.0, 0.72)
    dt = 0.05
    o, g = pair(mesh, 3, oracle.NS, oracle.CASE_VORTEX, mu=mu, newton_rtol=1e-8, gmres_rtol=1e-3,
                krylov_precision=kprec, precond=1)
    un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
    for k in range(2):
        t1 = (k + 1) * dt
        o.set_time(2, t1, dt, un, unm1)
        g.set_time(2, t1, dt, cuda(un), cuda(unm1))
        u = cuda(un)
        rep = g.newton_gmres(u)
        assert rep["status"] == 0 and rep["rfinal"] <= 1e-8 * rep["r0"], rep
        ug = host(u)
        assert np.linalg.norm(o.residual(ug)) <= 1.5e-8 * rep["r0"]
        if k == 0:
            uo, rc, st = o.newton(un.copy(), m=30, newton_rtol=1e-10, gmres_rtol=1e-6)
            assert rc == 0
            assert np.linalg.norm(ug - uo) <= 1e-7 * np.linalg.norm(uo)
        unm1, un = un, ug


def test_batch_matches_single_contexts():
    from paper_2205_07824_b300.ldg import LDG, Batch
    mesh = _box(8, affine=None)
    mus = [(1.4, 50.0, 0.72), (1.4, 200.0, 0.72), (1.3, 100.0, 1.0)]
    dt = 0.05
    b = Batch([mesh] * 3, [2] * 3, oracle.NS, oracle.CASE_VORTEX, mus, gmres_m=20, precond=1)
    u0 = np.concatenate([oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_VORTEX, mu).interpolate(0.0) for mu in mus])
    um1 = np.concatenate([oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_VORTEX, mu).interpolate(-dt) for mu in mus])
    v = synth.random_vector(b.n_total, 9)
    b.set_time(2, dt, dt, cuda(u0), cuda(um1))
    r = host(b.residual(cuda(u0)))
    jv = host(b.jvp(cuda(u0), cuda(v)))
    bu = cuda(u0)
    reps, _ = b.solve(bu)
    bu = host(bu)
    for i, mu in enumerate(mus):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        o = oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_VORTEX, mu)
        o.set_time(2, dt, dt, u0[sl], um1[sl])
        assert_parity(r[sl], o.residual(u0[sl]), what=f"batch R {i}")
        assert_parity(jv[sl], o.jvp(u0[sl], v[sl]), what=f"batch J.v {i}")
        g = LDG(mesh, 2, oracle.NS, oracle.CASE_VORTEX, mu, gmres_m=20, precond=1)
        g.set_time(2, dt, dt, cuda(u0[sl]), cuda(um1[sl]))
        ui = cuda(u0[sl])
        rep = g.newton_gmres(ui)
        assert reps[i]["status"] == 0 and reps[i]["newton_iters"] == rep["newton_iters"]
        assert np.linalg.norm(bu[sl] - host(ui)) <= 1e-7 * np.linalg.norm(host(ui))
        assert np.linalg.norm(o.residual(bu[sl])) <= 1.5e-8 * reps[i]["r0"]
