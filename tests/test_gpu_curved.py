"""Curved quadrilaterals and solid walls on the GPU against the FP64 CPU oracle.

Per-point metrics, normals and element mass inverses (sampled on the host from
the degree-pg element maps) drive the same fused stage kernels; the q-stage takes
the weak form with the element's own mass matrix. Residual, q and the exact J.v
meet the FP64 parity bar for every model on warped boxes and O-grids with walls;
the element-diagonal blocks equal the oracle's complex-step Jacobian blocks; a
BDF2 Newton-GMRES step of the viscous flow past a cylinder converges and the
oracle confirms its residual; batched curved instances equal single solves."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import assert_parity, cuda, host

pytestmark = pytest.mark.gpu

NS_MU = (1.4, 10.0, 0.72)


def _pair(mesh, p, model, case, mu, **kw):
    from paper_2205_07824_b300.ldg import LDG
    o = oracle.Oracle(mesh, p, model, case, mu)
    g = LDG(mesh, p, model, case, mu, nq1=o.nq1, **kw)
    assert g.n_dof == o.ndof
    return o, g


def _gas_state(mesh, npe, seed, dp=0.0):
    u = synth.random_euler_state(mesh.n_elem, npe, seed).reshape(mesh.n_elem, 4, npe)
    u[:, 3] += dp
    return u.ravel()


def _cyl(n_r=3, n_t=16, pg=3, jitter=0.3):
    return synth.o_grid(n_r, n_t, pg, outer=("circle", 3.0), first=0.1, jitter=jitter, seed=3)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("model", [oracle.POISSON, oracle.CONVDIFF])
def test_scalar_warped_box(p, model):
    mesh = synth.warped_box((6, 5), 3, amp=0.15)
    mu = (1.0, 1.0) if model == oracle.POISSON else (0.05, 0.3, 1.0, 0.5)
    o, g = _pair(mesh, p, model, oracle.CASE_SINSIN, mu)
    u, v = synth.random_vector(o.ndof, 1), synth.random_vector(o.ndof, 2)
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R")
    assert_parity(host(g.q(cuda(u))), o.q(u), what="q")
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="J.v")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_navier_stokes_cylinder_walls(p):
    mesh = _cyl()
    o, g = _pair(mesh, p, oracle.NS, oracle.CASE_CYLINDER, NS_MU)
    u, v = _gas_state(mesh, o.npe, 3, dp=15.0), synth.random_vector(o.ndof, 4)
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R")
    assert_parity(host(g.q(cuda(u))), o.q(u), what="q")
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="J.v")
    out = cuda(np.zeros(o.ndof))
    g.jvp_noalloc(cuda(u), cuda(v), out)
    assert_parity(host(out), o.jvp(u, v), what="J.v noalloc")


@pytest.mark.parametrize("p", [2, 3])
def test_euler_cylinder_walls_and_tiles(p):
    mesh = _cyl()
    o, g = _pair(mesh, p, oracle.EULER, oracle.CASE_CYLINDER, (1.4,))
    u, v = _gas_state(mesh, o.npe, 5, dp=15.0), synth.random_vector(o.ndof, 6)
    r_ref, jv_ref = o.residual(u), o.jvp(u, v)
    for t in (0, 1):
        g.set_tile(t)
        assert_parity(host(g.residual(cuda(u))), r_ref, what=f"R tile {t}")
        assert_parity(host(g.jvp(cuda(u), cuda(v))), jv_ref, what=f"J.v tile {t}")


def test_ns_warped_periodic_vortex_bdf2():
    mesh = synth.warped_box((5, 4), 2, hi=(10.0, 10.0), periodic=(True, True), amp=0.2)
    o, g = _pair(mesh, 3, oracle.NS, oracle.CASE_VORTEX, (1.3, 50.0, 0.9, 0.2))
    u, v = _gas_state(mesh, o.npe, 7), synth.random_vector(o.ndof, 8)
    un, unm1 = _gas_state(mesh, o.npe, 9), _gas_state(mesh, o.npe, 10)
    o.set_time(2, 0.3, 0.05, un, unm1)
    g.set_time(2, 0.3, 0.05, cuda(un), cuda(unm1))
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R")
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="J.v")


def test_interpolation_and_free_stream():
    mesh = _cyl(jitter=0.3)
    o, g = _pair(mesh, 3, oracle.NS, oracle.CASE_CYLINDER, NS_MU)
    ui = host(g.interpolate(0.0))
    assert_parity(ui, o.interpolate(), what="interpolate")
    o0, g0 = _pair(mesh, 3, oracle.NS, oracle.CASE_CYLINDER_START, NS_MU)
    assert_parity(host(g0.interpolate(0.0)), o0.interpolate(), what="interpolate start state")
    # away from walls the free stream is preserved: far-field-only O-grid
    m2 = synth.o_grid(3, 16, 3, outer=("circle", 3.0), jitter=0.3, wall=False)
    o2, g2 = _pair(m2, 3, oracle.NS, oracle.CASE_CYLINDER, NS_MU)
    r = host(g2.residual(g2.interpolate(0.0)))
    assert np.abs(r).max() < 1e-11 * 17.0


def test_fp32_jvp_error():
    mesh = _cyl()
    o, g = _pair(mesh, 3, oracle.NS, oracle.CASE_CYLINDER, NS_MU)
    u, v = _gas_state(mesh, o.npe, 11, dp=15.0), synth.random_vector(o.ndof, 12)
    ref = o.jvp(u, v)
    err = np.linalg.norm(host(g.jvp_prec(1, cuda(u), cuda(v))) - ref) / np.linalg.norm(ref)
    print(f"curved NS FP32 J.v relative error: {err:.2e}")
    assert 1e-10 < err < 2e-5
    # the FP32 J.v reads FP32 copies of u and q(u) written by the residual's q-stage: after a
    # residual at u it gives bitwise the J.v that forms q(u) itself
    jv32 = host(g.jvp_prec(1, cuda(u), cuda(v)))
    cu = cuda(u)
    g.residual(cu)
    assert np.array_equal(host(g.jvp_after_residual(1, cu, cuda(v))), jv32)


@pytest.mark.parametrize("model", [oracle.EULER, oracle.NS])
def test_diag_blocks_match_complex_step(model):
    mesh = synth.o_grid(2, 10, 3, outer=("circle", 2.0), jitter=0.3, seed=5)
    mu = (1.4,) if model == oracle.EULER else NS_MU
    o, g = _pair(mesh, 2, model, oracle.CASE_CYLINDER, mu)
    u = _gas_state(mesh, o.npe, 13, dp=15.0)
    o.set_time(2, 0.1, 0.05, u, u)
    g.set_time(2, 0.1, 0.05, cuda(u), cuda(u))
    nloc = o.npe * o.ncu
    J = o.jacobian_cs(u)
    ref = np.stack([J[e * nloc:(e + 1) * nloc, e * nloc:(e + 1) * nloc] for e in range(mesh.n_elem)])
    blk = host(g.diag_blocks(cuda(u))).reshape(mesh.n_elem, nloc, nloc)
    assert_parity(blk.transpose(0, 2, 1), ref, what="diag blocks")
    blk32 = host(g.diag_blocks(cuda(u), precision=1)).reshape(mesh.n_elem, nloc, nloc)
    assert np.linalg.norm(blk32.transpose(0, 2, 1) - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("kprec", [0, 1])
def test_cylinder_bdf2_newton_block_jacobi(kprec):
    """One BDF2 step (dt = 0.1) of the flow past the cylinder at Re = 100 from the
    free stream, p = 3, block-Jacobi; the oracle recomputes the final residual."""
    mesh = synth.o_grid(4, 24, 3, outer=("rect", (-4.0, 8.0, -4.0, 4.0)), first=0.1, jitter=0.2, seed=7)
    mu = (1.4, 100.0, 0.72)
    o, g = _pair(mesh, 3, oracle.NS, oracle.CASE_CYLINDER, mu, newton_rtol=1e-8, gmres_rtol=1e-3,
                 krylov_precision=kprec, precond=1)
    dt = 0.1
    un = o.interpolate()
    o.set_time(2, dt, dt, un, un)
    g.set_time(2, dt, dt, cuda(un), cuda(un))
    u = cuda(un)
    rep = g.newton_gmres(u)
    assert rep["status"] == 0 and rep["rfinal"] <= 1e-8 * rep["r0"], rep
    assert np.linalg.norm(o.residual(host(u))) <= 1.5e-8 * rep["r0"]
    assert rep["newton_iters"] >= 1


def test_batch_curved_instances():
    from paper_2205_07824_b300.ldg import LDG, Batch
    mesh = _cyl(n_r=3, n_t=12)
    mus = [(1.4, 50.0, 0.72), (1.4, 400.0, 0.72)]
    b = Batch([mesh] * 2, [2] * 2, oracle.NS, oracle.CASE_CYLINDER, mus, gmres_m=20, precond=1)
    u = np.concatenate([_gas_state(mesh, 9, 20 + i, dp=15.0) for i in range(2)])
    v = synth.random_vector(b.n_total, 21)
    r = host(b.residual(cuda(u)))
    jv = host(b.jvp(cuda(u), cuda(v)))
    for i, mu in enumerate(mus):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        o = oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_CYLINDER, mu)
        assert_parity(r[sl], o.residual(u[sl]), what=f"batch R {i}")
        assert_parity(jv[sl], o.jvp(u[sl], v[sl]), what=f"batch J.v {i}")
    # BDF2 step from the free stream, batched vs single contexts
    dt = 0.1
    u0 = np.concatenate([oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_CYLINDER, mu).interpolate() for mu in mus])
    b.set_time(2, dt, dt, cuda(u0), cuda(u0))
    bu = cuda(u0)
    reps, _ = b.solve(bu)
    bu = host(bu)
    for i, mu in enumerate(mus):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        g = LDG(mesh, 2, oracle.NS, oracle.CASE_CYLINDER, mu, gmres_m=20, precond=1)
        g.set_time(2, dt, dt, cuda(u0[sl]), cuda(u0[sl]))
        ui = cuda(u0[sl])
        rep = g.newton_gmres(ui)
        assert reps[i]["status"] == 0 and reps[i]["newton_iters"] == rep["newton_iters"]
        assert np.linalg.norm(bu[sl] - host(ui)) <= 1e-7 * np.linalg.norm(host(ui))


def test_newton_step_halving_keeps_the_impulsive_start_finite():
    """The impulsively started cylinder (free stream up to the no-slip wall, Re = 673,
    dt = 0.1) drives full Newton steps to non-finite states. With step control, a step
    after which ||R|| grows more than tenfold (or becomes non-finite) is halved: the
    solve reports its halvings and ends at the Newton cap with a finite state, not with
    a non-finite one."""
    from paper_2205_07824_b300.ldg import LDG
    mesh = synth.cylinder_mesh(25, 100, 3, seed=7)
    g = LDG(mesh, 3, oracle.NS, oracle.CASE_CYLINDER, (1.4, 673.0, 0.72), newton_rtol=1e-8, gmres_rtol=1e-3,
            krylov_precision=1, precond=1, max_newton=10)
    u0 = g.interpolate(0.0)
    g.set_time(2, 0.1, 0.1, u0, u0.clone())
    u = u0.clone()
    rep = g.newton_gmres(u, check=False)
    assert rep["newton_backtracks"] >= 1, rep
    assert rep["status"] in (0, -5), rep
    assert np.all(np.isfinite(host(u)))


def test_full_navier_stokes_cylinder_40000_p3_sampled():
    """Navier-Stokes past the cylinder on the full mesh of the time-to-1e-8 workload
    (40,000 curved quadrilaterals, 100 layers x 400 around, p = 3, Re = 673, Mach 0.2
    far field, no-slip wall): the kernels run on the whole state, and the oracle
    evaluates R and J.v on a sample of elements (wall layer, outer layer, interior),
    each with the q-stage of its face neighbours."""
    mesh = synth.cylinder_mesh(100, 400, 3, seed=7)
    o, g = _pair(mesh, 3, oracle.NS, oracle.CASE_CYLINDER, (1.4, 673.0, 0.72))
    u = _gas_state(mesh, o.npe, 5, dp=15.0)
    v = synth.random_vector(o.ndof, 6)
    rng = np.random.default_rng(1)
    el = np.unique(np.concatenate([[0, 399, 200, mesh.n_elem - 1, mesh.n_elem - 400, mesh.n_elem // 2],
                                   rng.integers(0, mesh.n_elem, 30)]))
    shape = (-1, 4, o.npe)
    r = host(g.residual(cuda(u))).reshape(shape)[el]
    assert_parity(r, o.residual_some(u, el), what="R cylinder 40,000 p=3")
    jv = host(g.jvp(cuda(u), cuda(v))).reshape(shape)[el]
    assert_parity(jv, o.jvp_some(u, v, el), what="J.v cylinder 40,000 p=3")
