"""L2 projection and relative L2 errors on the GPU (Section 4.1's error measure,
Table 3) against the FP64 CPU oracle's, on every affine element type."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu

CASES = [
    ("tri", lambda: synth.tri_square(5, affine=SHEAR2), 2, oracle.POISSON, oracle.CASE_SINSIN),
    ("tri_p5", lambda: synth.tri_unstructured(4, seed=3), 5, oracle.CONVDIFF, oracle.CASE_EXPSIN),
    ("quad", lambda: synth.quad_box((6, 5), affine=SHEAR2), 3, oracle.CONVDIFF, oracle.CASE_EXPSIN),
    ("hex", lambda: synth.hex_box(3, affine=SHEAR3), 2, oracle.POISSON, oracle.CASE_SINSIN),
    ("hex_p4", lambda: synth.hex_box((3, 2, 2)), 4, oracle.CONVDIFF, oracle.CASE_EXPSIN),
    ("tet", lambda: synth.tet_cube(2, affine=SHEAR3), 3, oracle.POISSON, oracle.CASE_SINSIN),
    ("euler", lambda: synth.quad_box(4, hi=(10.0, 10.0), periodic=(True, True)), 3, oracle.EULER,
     oracle.CASE_VORTEX),
]


@pytest.mark.parametrize("name,mk,p,model,case", CASES, ids=[c[0] for c in CASES])
def test_project_matches_oracle(name, mk, p, model, case):
    mesh = mk()
    o, g = pair(mesh, p, model, case)
    for t in (0.0, 0.3):
        assert_parity(host(g.project(t)), o.project(t), what=f"{name} projection t={t}")


@pytest.mark.parametrize("name,mk,p,model,case", CASES, ids=[c[0] for c in CASES])
def test_l2_error_matches_oracle(name, mk, p, model, case):
    mesh = mk()
    o, g = pair(mesh, p, model, case)
    rng = np.random.default_rng(11)
    # A discrete state near the exact field, and one far from it. Both sides sum the same
    # integrals in different orders: the pointwise u_h carries FP64 rounding of about
    # 2^-52 sum_i |phi_i u_i| <~ 1e-15 |u|, so E(u_h) agrees to 1e-12 of itself plus 1e-14
    # absolute (what matters when u_h - u is small). q_h itself comes from the q-stage,
    # which meets the 1e-12 parity bar relative to ||q_h|| <= (1 + E(q_h)) ||q||: E(q_h)
    # agrees to 1e-12 of itself plus 2e-12 (1 + E(q_h)) absolute.
    for u in (o.interpolate() + 1e-3 * rng.standard_normal(o.ndof), synth.random_vector(o.ndof, 4)):
        eu, eq = g.l2_error(cuda(u))
        ou, oq = o.l2_error(u)
        assert abs(eu - ou) <= 1e-12 * ou + 1e-14, (name, eu, ou)
        if model in (oracle.POISSON, oracle.CONVDIFF):
            assert abs(eq - oq) <= 1e-12 * oq + 2e-12 * (1.0 + oq), (name, eq, oq)
        else:
            assert eq == 0.0


def test_projection_error_falls_at_order_p_plus_1():
    """The projection is the best L2 approximation: its error falls at order p + 1."""
    errs = []
    for n in (4, 8):
        mesh = synth.quad_box(n)
        _, g = pair(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN)
        errs.append(g.l2_error(g.project(0.0))[0])
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - 3.0) < 0.25, (errs, rate)


def test_curved_elements_are_rejected():
    from paper_2205_07824_b300.ldg import LDGError
    mesh = synth.warped_box(3, amp=0.05, pg=2)
    _, g = pair(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN)
    with pytest.raises(LDGError):
        g.project(0.0)
