"""Curved (isoparametric) triangles on the GPU against the FP64 CPU oracle.

The host samples each triangle's degree-pg map at the collapsed Gauss points (metric
w det J d xi / dx, face normals and w sJ, physical coordinates, the element mass
inverses); the same fused stage kernels as on curved quadrilaterals then run on the
triangle's reference operators. Residual, q and the exact J.v meet the FP64 parity bar
on the annulus 0.5 <= r <= 1 for maps of degree 1..3 and p = 1..4; a straight-sided
map (degree 1) gives the affine triangle context's operator; a Newton-GMRES solve
lands on the oracle's solution; the element-diagonal blocks equal the oracle's
Jacobian blocks; batched instances equal single contexts."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu

CD_MU = (0.05, 0.3, 1.0, 0.5)


def _mu(model):
    return (1.0, 1.0) if model == oracle.POISSON else CD_MU


@pytest.mark.parametrize("pg", [1, 2, 3])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("model", [oracle.POISSON, oracle.CONVDIFF])
def test_curved_triangle_parity(model, p, pg):
    """3 x 10 cells of the annulus (60 triangles: several CTAs of every tile and a ragged
    last one), sin(pi x) sin(pi y) data on the boundary and in the source."""
    mesh = synth.tri_annulus(3, 10, pg)
    o, g = pair(mesh, p, model, oracle.CASE_SINSIN, _mu(model))
    u, v = synth.random_vector(o.ndof, 1), synth.random_vector(o.ndof, 2)
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R")
    assert_parity(host(g.q(cuda(u))), o.q(u), what="q")
    jv = o.jvp(u, v)
    assert_parity(host(g.jvp(cuda(u), cuda(v))), jv, what="J.v")
    for t in (0, 1):
        g.set_tile(t)
        assert_parity(host(g.jvp(cuda(u), cuda(v))), jv, what=f"J.v tile {t}")


@pytest.mark.parametrize("p", [1, 3])
def test_straight_sided_map_gives_the_affine_operator(p):
    """Degree-1 maps are the triangles' affine maps: the curved context's residual and
    J.v equal those of the affine context on the same vertices (a normal turned the
    wrong way, a face weight off by sJ or a transposed metric would differ)."""
    from paper_2205_07824_b300.ldg import LDG
    curved = synth.tri_annulus(2, 12, 1)
    flat = synth.Mesh(curved.etype, curved.xyz, curved.vid, "tri_annulus_flat")
    mu = CD_MU
    gc = LDG(curved, p, oracle.CONVDIFF, oracle.CASE_SINSIN, mu, nq1=p + 2)
    ga = LDG(flat, p, oracle.CONVDIFF, oracle.CASE_SINSIN, mu, nq1=p + 2)
    n = gc.n_dof
    u, v = synth.random_vector(n, 3), synth.random_vector(n, 4)
    assert_parity(host(gc.residual(cuda(u))), host(ga.residual(cuda(u))), what="R curved vs affine")
    assert_parity(host(gc.jvp(cuda(u), cuda(v))), host(ga.jvp(cuda(u), cuda(v))), what="J.v curved vs affine")
    assert "k_qstage_curved" in gc.jv_kernels()


def test_interpolation_and_blocks():
    mesh = synth.tri_annulus(2, 8, 3)
    o, g = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_SINSIN, CD_MU)
    assert_parity(host(g.interpolate(0.0)), o.interpolate(), what="interpolate")
    n, nloc = o.ndof, o.npe * o.ncu
    z = np.zeros(n)
    J = np.stack([o.jvp(z, e) for e in np.eye(n)], axis=1)
    ref = np.stack([J[e * nloc:(e + 1) * nloc, e * nloc:(e + 1) * nloc] for e in range(mesh.n_elem)])
    blk = host(g.diag_blocks(cuda(z))).reshape(mesh.n_elem, nloc, nloc)
    assert_parity(blk.transpose(0, 2, 1), ref, what="diag blocks")


def test_newton_gmres_reaches_the_oracle_solution():
    """Poisson on the annulus (4 x 16 cells, p = 2, quadratic maps), block-Jacobi
    GMRES to 1e-12: the GPU solution is the oracle's own (to the solve tolerance) and its
    oracle residual is at the solve tolerance; the L2 error against sin(pi x) sin(pi y),
    from the oracle, is that of the converged discretisation."""
    mesh = synth.tri_annulus(4, 16, 2)
    o, g = pair(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0), newton_rtol=1e-12, gmres_rtol=1e-12,
                gmres_m=60, max_restarts=200, precond=1)
    u = cuda(np.zeros(o.ndof))
    r0 = np.linalg.norm(o.residual(np.zeros(o.ndof)))
    rep = g.newton_gmres(u)
    assert rep["status"] == 0, rep
    ug = host(u)
    assert np.linalg.norm(o.residual(ug)) <= 1e-10 * r0
    uo, rc, _ = o.newton(np.zeros(o.ndof), newton_rtol=1e-12, gmres_rtol=1e-12, m=60, max_gmres=5000)
    assert rc == 0
    assert np.linalg.norm(ug - uo) <= 1e-9 * np.linalg.norm(uo)
    eg, eo = o.l2_error(ug)[0], o.l2_error(uo)[0]
    assert abs(eg - eo) <= 1e-6 * eo and eo < 1e-2, (eg, eo)


def test_fp32_jvp_and_unsupported_calls():
    from paper_2205_07824_b300.ldg import F32X2, LDG
    mesh = synth.tri_annulus(3, 10, 2)
    o, g = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_SINSIN, CD_MU)
    u, v = synth.random_vector(o.ndof, 5), synth.random_vector(o.ndof, 6)
    ref = o.jvp(u, v)
    err = np.linalg.norm(host(g.jvp_prec(1, cuda(u), cuda(v))) - ref) / np.linalg.norm(ref)
    print(f"curved triangle FP32 J.v relative error: {err:.2e}")
    assert 1e-10 < err < 1e-5
    with pytest.raises(RuntimeError):
        g.l2_error(cuda(u))
    with pytest.raises(RuntimeError):
        LDG(mesh, 3, oracle.CONVDIFF, oracle.CASE_SINSIN, CD_MU, nq1=5, krylov_precision=F32X2)


def test_batch_curved_triangles():
    from paper_2205_07824_b300.ldg import LDG, Batch
    meshes = [synth.tri_annulus(2, 8, 2), synth.tri_annulus(3, 9, 3)]
    mus = [CD_MU, (0.1, 0.2, -0.5, 0.3)]
    b = Batch(meshes, [2, 2], oracle.CONVDIFF, oracle.CASE_SINSIN, mus, gmres_m=30, precond=1,
              newton_rtol=1e-10, gmres_rtol=1e-10, max_restarts=100)
    u = synth.random_vector(b.n_total, 7)
    v = synth.random_vector(b.n_total, 8)
    r = host(b.residual(cuda(u)))
    jv = host(b.jvp(cuda(u), cuda(v)))
    for i, (m, mu) in enumerate(zip(meshes, mus)):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        o = oracle.Oracle(m, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, mu)
        assert_parity(r[sl], o.residual(u[sl]), what=f"batch R {i}")
        assert_parity(jv[sl], o.jvp(u[sl], v[sl]), what=f"batch J.v {i}")
    bu = cuda(np.zeros(b.n_total))
    reps, _ = b.solve(bu)
    bu = host(bu)
    for i, (m, mu) in enumerate(zip(meshes, mus)):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        g = LDG(m, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, mu, gmres_m=30, precond=1, newton_rtol=1e-10,
                gmres_rtol=1e-10, max_restarts=100)
        ui = cuda(np.zeros(g.n_dof))
        rep = g.newton_gmres(ui)
        assert reps[i]["status"] == 0 and rep["status"] == 0
        assert np.linalg.norm(bu[sl] - host(ui)) <= 1e-8 * np.linalg.norm(host(ui))
