"""Block-Jacobi preconditioner: the extracted element-diagonal blocks equal those
of the oracle's complex-step dense Jacobian, the block inverse applies as its
definition says, and preconditioned Newton-GMRES reaches the same solution with
far fewer Krylov iterations."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu


def _dense_diag_blocks(J, E, nloc):
    return np.stack([J[e * nloc:(e + 1) * nloc, e * nloc:(e + 1) * nloc] for e in range(E)])


@pytest.mark.parametrize("mesh,p,model,case", [
    (lambda: synth.quad_box((4, 3), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2), 2, oracle.EULER,
     oracle.CASE_VORTEX),
    (lambda: synth.quad_box((3, 3), hi=(10.0, 10.0)), 1, oracle.EULER, oracle.CASE_VORTEX),
    (lambda: synth.tri_square(3, affine=SHEAR2), 2, oracle.POISSON, oracle.CASE_SINSIN),
    (lambda: synth.hex_box((2, 2, 3), affine=SHEAR3), 1, oracle.CONVDIFF, oracle.CASE_EXPSIN),
])
def test_diag_blocks_match_complex_step_jacobian(mesh, p, model, case):
    m = mesh()
    o, g = pair(m, p, model, case)
    u = synth.random_euler_state(m.n_elem, o.npe, 5) if model == oracle.EULER else synth.random_vector(o.ndof, 5)
    if model == oracle.EULER:
        o.set_time(2, 0.1, 0.05, u, u)
        g.set_time(2, 0.1, 0.05, cuda(u), cuda(u))
    nloc = o.npe * o.ncu
    ref = _dense_diag_blocks(o.jacobian_cs(u), m.n_elem, nloc)           # [E][row][col]
    blk = host(g.diag_blocks(cuda(u))).reshape(m.n_elem, nloc, nloc)     # [E][col][row]
    assert_parity(blk.transpose(0, 2, 1), ref, what="diag blocks")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_block_inverse_applies(p):
    """Block sizes 16, 36, 64, 100 (the compile-time-size inversion), FP64 and FP32."""
    mesh = synth.quad_box((5, 4), hi=(10.0, 10.0), periodic=(True, True))
    for prec, tol in ((0, 1e-11), (1, 1e-4)):
        o, g = pair(mesh, p, oracle.EULER, oracle.CASE_VORTEX, krylov_precision=prec, precond=1)
        u = o.interpolate(0.0)
        g.set_time(2, 0.05, 0.05, cuda(u), cuda(u))
        g.precond_setup(cuda(u))
        x = synth.random_vector(o.ndof, 3)
        y = host(g.precond_apply(cuda(x)))
        nloc = o.npe * o.ncu
        B = host(g.diag_blocks(cuda(u))).reshape(mesh.n_elem, nloc, nloc)
        back = np.einsum("ecr,ec->er", B, y.reshape(mesh.n_elem, nloc)).ravel()
        assert np.linalg.norm(back - x) <= tol * np.linalg.norm(x), prec


@pytest.mark.parametrize("kprec", [0, 1])
def test_block_jacobi_newton_bdf2(kprec):
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    reps = {}
    for pc in (0, 1):
        o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3,
                    krylov_precision=kprec, precond=pc)
        un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
        g.set_time(2, dt, dt, cuda(un), cuda(unm1))
        u = cuda(un)
        reps[pc] = g.newton_gmres(u)
        assert reps[pc]["rfinal"] <= 1e-8 * reps[pc]["r0"]
        if pc:
            o.set_time(2, dt, dt, un, unm1)
            ug = host(u)
            assert np.linalg.norm(o.residual(ug)) <= 1.5e-8 * reps[pc]["r0"]
    print("GMRES iterations without / with block-Jacobi:", reps[0]["gmres_iters"], reps[1]["gmres_iters"])
    assert reps[1]["gmres_iters"] * 3 < reps[0]["gmres_iters"]
    assert reps[1]["pc_setups"] == 1


def test_block_jacobi_poisson_512_triangles():
    """2-D Poisson on 512 triangles, p = 2, with the block-Jacobi preconditioner (blocks by coloured probing)."""
    mesh = synth.tri_square(16)
    o, g = pair(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN, gmres_rtol=1e-10, newton_rtol=1e-9, max_newton=1,
                max_restarts=400, precond=1)
    u = cuda(np.zeros(o.ndof))
    rep = g.newton_gmres(u)
    assert rep["rfinal"] <= 1e-9 * rep["r0"]
    uo, rc, st = o.newton(np.zeros(o.ndof), m=200, newton_rtol=1e-10, gmres_rtol=1e-12, max_newton=2)
    assert np.linalg.norm(host(u) - uo) <= 1e-8 * np.linalg.norm(uo)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_diag_blocks_fp32_match_fp64(p):
    """The FP32 block columns (eight tangents per launch) against the FP64 ones."""
    mesh = synth.quad_box((4, 5), hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, p, oracle.EULER, oracle.CASE_VORTEX)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 11)
    g.set_time(2, 0.1, 0.05, cuda(u), cuda(u))
    b64 = host(g.diag_blocks(cuda(u), precision=0))
    b32 = host(g.diag_blocks(cuda(u), precision=1))
    assert np.linalg.norm(b32 - b64) <= 2e-6 * np.linalg.norm(b64)
