"""The reduced-basis preconditioner (LDG_PC_RB_BJ) on the GPU: its apply equals the
oracle's P^{-1} r = C r + B^{-1} (r - J C r) for the same basis, it is the identity on the
preconditioned subspace, and in a sequence of implicit time steps the Newton updates
it collects leave the solutions those of block-Jacobi."""
import numpy as np
import pytest

import oracle
from oracle import rbpc
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, cuda, host, pair

pytestmark = pytest.mark.gpu

MU = (0.1, 1.0, 1.0, 0.5)


def _dense_jacobian(o, u):
    return np.stack([o.jvp(u, e) for e in np.eye(o.ndof)], axis=1)


@pytest.mark.parametrize("k", [0, 3, 8])
def test_rb_apply_matches_the_oracle_and_is_exact_on_the_subspace(k):
    import torch
    from paper_2205_07824_b300.ldg import PC_RB_BJ
    mesh = synth.quad_box((4, 3), affine=SHEAR2)
    o, g = pair(mesh, 2, oracle.CONVDIFF, oracle.CASE_ZERO, mu=MU, precond=PC_RB_BJ, rb_size=8)
    n = o.ndof
    u = synth.random_vector(n, 1)
    J = _dense_jacobian(o, u)
    Binv = rbpc.block_jacobi_inverse(J, o.npe * o.ncu)
    rng = np.random.default_rng(9)
    V = rng.standard_normal((n, k))
    g.rb_set_basis(cuda(np.ascontiguousarray(V.T)) if k else None)
    assert g.rb_count() == k
    cu = cuda(u)
    g.precond_setup(cu)
    x = rng.standard_normal(n)
    got = host(g.precond_apply(cuda(x)))
    ref = rbpc.rb_apply(J, Binv, V, x)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref), k
    if k:
        w = V @ rng.standard_normal(k)
        jw = host(g.jvp(cu, cuda(w)))
        back = host(g.precond_apply(cuda(jw)))
        assert np.linalg.norm(back - w) <= 1e-10 * np.linalg.norm(w)


def test_rb_basis_collects_newton_updates_and_keeps_the_block_jacobi_solutions():
    """BDF2 steps of the Euler vortex (16 x 16 quads, p = 3) with PC_RB_BJ and with
    PC_BJACOBI: the same states to the Newton tolerance; the reduced basis fills with
    the Newton updates up to rb_size; the total GMRES iterations are reported."""
    import torch
    from paper_2205_07824_b300.ldg import LDG, PC_BJACOBI, PC_RB_BJ
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt, steps = 0.05, 8
    out = {}
    for pc in (PC_BJACOBI, PC_RB_BJ):
        g = LDG(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, (1.4,), gmres_m=30, newton_rtol=1e-10, gmres_rtol=1e-6,
                precond=pc, rb_size=12)
        un, unm1 = g.interpolate(0.0), g.interpolate(-dt)
        its = 0
        for s in range(steps):
            g.set_time(2, (s + 1) * dt, dt, un, unm1)
            u = un.clone()
            rep = g.newton_gmres(u)
            assert rep["status"] == 0, rep
            its += rep["gmres_iters"]
            unm1, un = un, u
        out[pc] = (host(un), its, g.rb_count())
    uB, itB, _ = out[PC_BJACOBI]
    uR, itR, kR = out[PC_RB_BJ]
    assert kR == 12
    assert np.linalg.norm(uR - uB) <= 1e-8 * np.linalg.norm(uB)
    print(f"GMRES iterations over {steps} steps: block-Jacobi {itB}, reduced basis + block-Jacobi {itR}")
    assert itR <= itB
