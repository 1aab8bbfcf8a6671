"""The wave model's DIRK step on the GPU against the oracle (Section 2.1's wave form of
Eq. 1a with the displacement ODE, Eq. 2; Section 2.2's DIRK schemes).

`ldg_wave_step` eliminates each stage's q: Q_i = Qh_i + a_ii dt Q(U_i), so the stage is the
context's Poisson-type implicit solve with kappa' = a_ii dt c^2 plus a constant term, and
q and w follow node by node. The oracle (`oracle/wave.py`) steps the coupled (u, q) system
itself, with the operator assembled column by column and a dense solve per stage. The two
share no code; their u, q and w agree to the stage solves' tolerance."""
import numpy as np
import pytest

import oracle
from oracle import wave
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, cuda, host, pair

pytestmark = pytest.mark.gpu

C2, TAU = 0.8, 0.5
SOLVE = dict(gmres_m=30, gmres_rtol=1e-8, newton_rtol=1e-13, max_newton=10, max_restarts=200, precond=1)

CASES = [
    ("quad_periodic_p3", lambda: synth.quad_box((5, 4), hi=(1.2, 1.0), periodic=(True, True), affine=SHEAR2), 3),
    ("quad_dirichlet_p2", lambda: synth.quad_box((4, 5), affine=SHEAR2), 2),
    ("hex_periodic_p2", lambda: synth.hex_box((3, 3, 3), periodic=(True, True, True), affine=SHEAR3), 2),
    ("tri_dirichlet_p2", lambda: synth.tri_square(4, affine=SHEAR2), 2),
    ("tet_dirichlet_p1", lambda: synth.tet_cube(2), 1),
]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("scheme", [1, 2, 3, 4])
@pytest.mark.parametrize("name,mk,p", CASES, ids=[c[0] for c in CASES])
def test_wave_step_matches_the_oracle(name, mk, p, scheme):
    mesh = mk()
    o, g = pair(mesh, p, oracle.POISSON, oracle.CASE_ZERO, mu=(C2, TAU), **SOLVE)
    L, _ = wave.wave_operator(o)
    n, nq = o.ndof, o.ndof * o.nd
    rng = np.random.default_rng(7)
    u, q, w = rng.standard_normal(n), rng.standard_normal(nq), rng.standard_normal(n)
    alpha, beta, dt = 1.0, 0.3, 0.05
    gu, gq, gw = cuda(u), cuda(q), cuda(w)
    for k in range(3):
        u, q, w = wave.wave_step(L, n, u, q, w, dt, scheme, alpha=alpha, beta=beta)
        rep = g.wave_step(gu, gq, gw, t=k * dt, dt=dt, scheme=scheme, alpha=alpha, beta=beta)
        assert rep["status"] == 0 and rep["gmres_iters"] > 0, rep
    for what, got, ref in (("u", gu, u), ("q", gq, q), ("w", gw, w)):
        assert _rel(host(got), ref) <= 1e-10, (name, scheme, what, _rel(host(got), ref))


def test_wave_step_leaves_the_operator_as_it_was_and_skips_w_when_absent():
    """The step changes kappa only for its stage solves: the context's residual and J.v are
    unchanged afterwards; without w only u and q advance (and match the oracle)."""
    mesh = synth.quad_box((4, 4), periodic=(True, True), affine=SHEAR2)
    o, g = pair(mesh, 2, oracle.POISSON, oracle.CASE_ZERO, mu=(C2, TAU), **SOLVE)
    L, _ = wave.wave_operator(o)
    n = o.ndof
    rng = np.random.default_rng(3)
    u, q, v = rng.standard_normal(n), rng.standard_normal(n * o.nd), rng.standard_normal(n)
    jv0 = host(g.jvp(cuda(v), cuda(v)))
    gu, gq = cuda(u), cuda(q)
    g.wave_step(gu, gq, None, dt=0.02, scheme=4)
    u1, q1, _ = wave.wave_step(L, n, u, q, None, 0.02, 4)
    assert _rel(host(gu), u1) <= 1e-10 and _rel(host(gq), q1) <= 1e-10
    assert np.array_equal(host(g.jvp(cuda(v), cuda(v))), jv0)
    assert _rel(host(g.jvp(cuda(v), cuda(v))), o.jvp(np.zeros(n), v)) <= 1e-12


def test_wave_step_rejects_other_models_and_cases():
    from paper_2205_07824_b300.ldg import LDG
    mesh = synth.quad_box(4)
    n = None
    for model, case, mu in ((oracle.CONVDIFF, oracle.CASE_ZERO, (0.1, 1.0, 1.0, 0.5)),
                            (oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0)), (oracle.EULER, oracle.CASE_VORTEX, (1.4,))):
        g = LDG(mesh, 2, model, case, mu)
        n = g.n_dof
        u, q = cuda(np.zeros(n)), cuda(np.zeros(n * g.dim))
        with pytest.raises(RuntimeError):
            g.wave_step(u, q, None, dt=0.1)


def test_wave_step_on_convection_diffusion_without_convection():
    """Convection-diffusion with beta = 0 is the same operator: its wave step equals the
    Poisson oracle's."""
    mesh = synth.quad_box((4, 4), periodic=(True, True), affine=SHEAR2)
    o, _ = pair(mesh, 2, oracle.POISSON, oracle.CASE_ZERO, mu=(C2, TAU))
    from paper_2205_07824_b300.ldg import LDG
    g = LDG(mesh, 2, oracle.CONVDIFF, oracle.CASE_ZERO, (C2, TAU, 0.0, 0.0), nq1=o.nq1, **SOLVE)
    L, _ = wave.wave_operator(o)
    n = o.ndof
    rng = np.random.default_rng(4)
    u, q = rng.standard_normal(n), rng.standard_normal(n * o.nd)
    gu, gq = cuda(u), cuda(q)
    g.wave_step(gu, gq, None, dt=0.03, scheme=2)
    u1, q1, _ = wave.wave_step(L, n, u, q, None, 0.03, 2)
    assert _rel(host(gu), u1) <= 1e-10 and _rel(host(gq), q1) <= 1e-10
