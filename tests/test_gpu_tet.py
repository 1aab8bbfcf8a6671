"""Tetrahedra on the GPU against the FP64 CPU oracle (Section 4.1's element).

Residual, q and J.v meet the FP64 parity bar for Poisson and convection-diffusion,
p = 1..4, on sheared, ragged and periodic meshes and with both tile shapes (the
neighbour traces come from face nodes permuted into each element's own face-node
order); the element-diagonal blocks equal the oracle's complex-step Jacobian blocks;
and the GPU solves of Section 4.1's Poisson problem on the unit cube reproduce
Table 3's convergence rates at the table's finer meshes."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR3, assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("model", [oracle.POISSON, oracle.CONVDIFF])
@pytest.mark.parametrize("periodic", [False, True])
def test_residual_q_jvp(p, model, periodic):
    mesh = synth.tet_cube(3, hi=(1.5, 1.5, 1.5), periodic=(periodic,) * 3, affine=None if periodic else SHEAR3)
    mu = (1.0, 1.0) if model == oracle.POISSON else (0.05, 0.3, 1.0, 0.5, 0.25)
    o, g = pair(mesh, p, model, oracle.CASE_SINSIN, mu=mu)
    u, v = synth.random_vector(o.ndof, 1), synth.random_vector(o.ndof, 2)
    for t in (0, 1):
        g.set_tile(t)
        assert_parity(host(g.residual(cuda(u))), o.residual(u), what=f"R tile {t}")
        assert_parity(host(g.q(cuda(u))), o.q(u), what=f"q tile {t}")
        assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what=f"J.v tile {t}")
    jv32 = host(g.jvp_prec(1, cuda(u), cuda(v)))
    ref = o.jvp(u, v)
    assert np.linalg.norm(jv32 - ref) <= 2e-5 * np.linalg.norm(ref)


def test_diag_blocks_match_complex_step():
    mesh = synth.tet_cube(2, affine=SHEAR3)
    o, g = pair(mesh, 1, oracle.CONVDIFF, oracle.CASE_SINSIN, mu=(0.05, 0.3, 1.0, 0.5, 0.25))
    u = synth.random_vector(o.ndof, 5)
    nloc = o.npe
    J = o.jacobian_cs(u)
    ref = np.stack([J[e * nloc:(e + 1) * nloc, e * nloc:(e + 1) * nloc] for e in range(mesh.n_elem)])
    blk = host(g.diag_blocks(cuda(u))).reshape(mesh.n_elem, nloc, nloc)
    assert_parity(blk.transpose(0, 2, 1), ref, what="diag blocks")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_table3_rates_on_gpu(p):
    """Section 4.1: -lap u = f on the unit cube, u = sin(pi x) sin(pi y) sin(pi z),
    structured tetrahedral meshes, 1/n = 4, 8, 16. The GPU solves (Newton-GMRES with
    block-Jacobi to 1e-10) and measures the L2 errors of u_h and of q_h (ldg_l2_error; on
    the coarsest mesh they equal the oracle's to 1e-12). The rates between n = 8 and 16
    match Table 3's row 1/n = 16 within 0.25 and approach p + 1 and p."""
    gold = json.load(open(os.path.join(GOLD, "table3_rates.json")))
    errs = []
    for n in (4, 8, 16):
        mesh = synth.tet_cube(n)
        o, g = pair(mesh, p, oracle.POISSON, oracle.CASE_SINSIN, mu=(1.0, 1.0), newton_rtol=1e-10,
                    gmres_rtol=1e-10, max_restarts=400, precond=1)
        u = cuda(np.zeros(o.ndof))
        rep = g.newton_gmres(u)
        assert rep["status"] == 0, rep
        errs.append(g.l2_error(u))
        if n == 4:
            # the tolerance of tests/test_gpu_l2.py: 1e-12 relative plus the rounding floor
            # of the pointwise u_h (1e-14) and of the q-stage's parity bar (2e-12 (1 + E(q_h)))
            ou, oq = o.l2_error(host(u))
            assert abs(errs[-1][0] - ou) <= 1e-12 * ou + 1e-14, (errs[-1], ou)
            assert abs(errs[-1][1] - oq) <= 1e-12 * oq + 2e-12 * (1.0 + oq), (errs[-1], oq)
    e = np.array(errs)
    ru = np.log2(e[1, 0] / e[2, 0])
    rq = np.log2(e[1, 1] / e[2, 1])
    print(f"p={p}: u errors {e[:, 0]}, q errors {e[:, 1]}, rates 8->16 u {ru:.2f} q {rq:.2f}")
    assert abs(ru - gold["u_rate_row16"][str(p)]) < 0.25, (ru, e)
    assert abs(rq - gold["q_rate_row16"][str(p)]) < 0.25, (rq, e)
