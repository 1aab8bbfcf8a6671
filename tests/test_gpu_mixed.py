"""Mixed precision: the Krylov J.v in FP32 arithmetic (FP64 in memory), with the
FP64 Newton residual, Arnoldi process and final check. The FP32 J.v is not held
to the FP64 parity bar; its error against the FP64 oracle is measured and must
sit at FP32 round-off level, and the outer Newton iteration must still reach
the FP64 tolerance (inexact Newton)."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, cuda, host, pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mesh,p,model,case", [
    (lambda: synth.quad_box((8, 7), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2), 3, oracle.EULER,
     oracle.CASE_VORTEX),
    (lambda: synth.tri_square(8, affine=SHEAR2), 2, oracle.POISSON, oracle.CASE_SINSIN),
    (lambda: synth.hex_box((3, 3, 4), affine=SHEAR3), 4, oracle.CONVDIFF, oracle.CASE_EXPSIN),
])
def test_fp32_jvp_error_against_fp64_oracle(mesh, p, model, case, record_property):
    m = mesh()
    o, g = pair(m, p, model, case)
    u = synth.random_euler_state(m.n_elem, o.npe, 1) if model == oracle.EULER else synth.random_vector(o.ndof, 1)
    v = synth.random_vector(o.ndof, 2)
    ref = o.jvp(u, v)
    jv32 = host(g.jvp_prec(1, cuda(u), cuda(v)))
    err = np.linalg.norm(jv32 - ref) / np.linalg.norm(ref)
    record_property("fp32_jv_rel_err", err)
    print(f"FP32 J.v relative error vs FP64 oracle: {err:.2e}")
    assert 1e-10 < err < 2e-5


def test_newton_with_fp32_krylov_reaches_fp64_tolerance():
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3, krylov_precision=1)
    dt = 0.05
    un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
    o.set_time(2, dt, dt, un, unm1)
    g.set_time(2, dt, dt, cuda(un), cuda(unm1))
    u = cuda(un)
    rep = g.newton_gmres(u)
    assert rep["rfinal"] <= 1e-8 * rep["r0"]
    ug = host(u)
    # the FP64 oracle residual of the mixed-precision solution meets the same bar
    assert np.linalg.norm(o.residual(ug)) <= 1.5e-8 * rep["r0"]
    uo, rc, st = o.newton(un.copy(), m=30, newton_rtol=1e-11, gmres_rtol=1e-6)
    assert np.linalg.norm(ug - uo) <= 1e-7 * np.linalg.norm(uo)
