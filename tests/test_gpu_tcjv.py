"""The Euler J.v with its contractions on the tensor cores (tcgen05) against the FP64
CPU oracle.

Interpolation to the volume and face points, the weak volume integral, the face lift
and the mass matrix run as BF16 GEMMs with FP32 accumulation in tensor memory, batched
over 32 elements (128 rows) per CTA; the pointwise fluxes are FP32 dual numbers. Its
error against the FP64 oracle is measured and bounded (BF16 hi/lo splits: FP32-class;
one BF16 product: about 1e-2), on periodic, far-field and wall faces, with the BDF time
term, and on element counts with a ragged last CTA; inside Newton-GMRES the FP64
residual refines it back to the FP64 tolerance."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, cuda, host, pair

pytestmark = pytest.mark.gpu

BOUND = {3: 1e-4, 4: 5e-2}   # TC_BF16X3, TC_BF16: relative 2-norm error against the oracle


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _state(mesh, npe, seed):
    return synth.random_euler_state(mesh.n_elem, npe, seed)


def _walled(nx, ny):
    """A far-field box whose bottom faces are no-slip walls."""
    mesh = synth.quad_box((nx, ny), hi=(10.0, 10.0))
    bc = np.zeros((mesh.n_elem, 4), dtype=np.uint8)
    bc[:nx, 2] = 1          # face 2 = axis 1, side 0: y = 0
    mesh.bc = bc
    return mesh


@pytest.mark.parametrize("prec", [3, 4])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tc_jv_error_against_the_oracle(p, prec):
    """Sheared periodic vortex box, 9 x 7 = 63 elements (a full and a ragged CTA)."""
    mesh = synth.quad_box((9, 7), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    o, g = pair(mesh, p, oracle.EULER, oracle.CASE_VORTEX)
    u, v = _state(mesh, o.npe, 1), synth.random_vector(o.ndof, 2)
    ref = o.jvp(u, v)
    err = _rel(host(g.jvp_prec(prec, cuda(u), cuda(v))), ref)
    e32 = _rel(host(g.jvp_prec(1, cuda(u), cuda(v))), ref)
    print(f"p={p} tensor-core J.v ({'bf16x3' if prec == 3 else 'bf16'}) error {err:.2e}; FP32 SIMT {e32:.2e}")
    assert err <= BOUND[prec]
    assert "k_euler_jv_tc" in g.jv_kernels(prec)


@pytest.mark.parametrize("prec", [3, 4])
def test_tc_jv_far_field_walls_and_time_term(prec):
    mesh = _walled(9, 7)
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX)
    u, v = _state(mesh, o.npe, 3), synth.random_vector(o.ndof, 4)
    un, unm1 = _state(mesh, o.npe, 5), _state(mesh, o.npe, 6)
    ref0 = o.jvp(u, v)
    assert _rel(host(g.jvp_prec(prec, cuda(u), cuda(v))), ref0) <= BOUND[prec]
    o.set_time(2, 0.3, 0.05, un, unm1)
    g.set_time(2, 0.3, 0.05, cuda(un), cuda(unm1))
    ref = o.jvp(u, v)
    err = _rel(host(g.jvp_prec(prec, cuda(u), cuda(v))), ref)
    print(f"walls + far field + BDF2 mass term: error {err:.2e}")
    assert err <= BOUND[prec]


@pytest.mark.parametrize("n", [(3, 3), (8, 4), (11, 6)])
def test_tc_jv_element_counts(n):
    """9 elements (one partial CTA), 32 (one full CTA), 66 (two full, one of 2)."""
    mesh = synth.quad_box(n, hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 2, oracle.EULER, oracle.CASE_VORTEX)
    u, v = _state(mesh, o.npe, 7), synth.random_vector(o.ndof, 8)
    out = cuda(np.full(o.ndof, 7.0))
    g.jvp_prec(3, cuda(u), cuda(v), out=out)
    assert _rel(host(out), o.jvp(u, v)) <= BOUND[3]


def test_tc_jv_is_linear_in_v_and_zero_at_v_zero():
    mesh = synth.quad_box((6, 6), hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX)
    u, v = _state(mesh, o.npe, 9), synth.random_vector(o.ndof, 10)
    z = host(g.jvp_prec(3, cuda(u), cuda(np.zeros(o.ndof))))
    assert np.array_equal(z, np.zeros(o.ndof))
    a = host(g.jvp_prec(3, cuda(u), cuda(v)))
    b = host(g.jvp_prec(3, cuda(u), cuda(2.0 * v)))
    # scaling v by 2 scales every BF16 part exactly: the same products, doubled
    assert np.array_equal(b, 2.0 * a)


@pytest.mark.parametrize("prec", [3, 4])
def test_newton_gmres_with_tensor_core_jv_reaches_the_fp64_tolerance(prec):
    """One BDF2 step of the vortex (16 x 16, p = 3) with block-Jacobi GMRES on the
    tensor-core J.v: the FP64 Newton residual still falls to 1e-8 and the state equals
    the FP64 solve's to the Newton tolerance."""
    from paper_2205_07824_b300.ldg import LDG
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    out = {}
    for kp in (0, prec):
        g = LDG(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, (1.4,), newton_rtol=1e-8, gmres_rtol=1e-3, precond=1,
                krylov_precision=kp)
        un, unm1 = g.interpolate(0.0), g.interpolate(-dt)
        g.set_time(2, dt, dt, un, unm1)
        u = un.clone()
        rep = g.newton_gmres(u)
        assert rep["status"] == 0 and rep["rfinal"] <= 1e-8 * rep["r0"], rep
        out[kp] = (host(u), rep)
    d = _rel(out[prec][0], out[0][0])
    print(f"Newton {out[prec][1]['newton_iters']} / GMRES {out[prec][1]['gmres_iters']} iterations "
          f"(FP64: {out[0][1]['newton_iters']} / {out[0][1]['gmres_iters']}); state difference {d:.2e}")
    assert d <= 1e-7


def test_tensor_core_jv_is_refused_where_it_does_not_exist():
    from paper_2205_07824_b300.ldg import LDG, Batch
    mesh = synth.quad_box(4)
    g = LDG(mesh, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, (0.1, 1.0, 1.0, 0.5))
    n = g.n_dof
    with pytest.raises(RuntimeError):
        g.jvp_prec(3, cuda(np.zeros(n)), cuda(np.zeros(n)))
    assert g.jv_kernels(3) == ""
    with pytest.raises(RuntimeError):
        LDG(mesh, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, (0.1, 1.0, 1.0, 0.5), krylov_precision=3)
    vmesh = synth.quad_box(4, hi=(10.0, 10.0), periodic=(True, True))
    with pytest.raises(RuntimeError):
        LDG(vmesh, 3, oracle.EULER, oracle.CASE_VORTEX, (1.4,), nq1=4, krylov_precision=3)   # p + 1 points
    with pytest.raises(RuntimeError):
        Batch([vmesh], [3], oracle.EULER, oracle.CASE_VORTEX, [(1.4,)], krylov_precision=3)
