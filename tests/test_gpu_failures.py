"""Failure detection, by host-side fault injection only (a corrupted input, a
tolerance that cannot be met, a bad argument or mesh): every case returns its status
code through the C-ABI and the report, nothing waits without bound, the context stays
usable, and in a batch a failing instance does not stop the others."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import cuda, host

pytestmark = pytest.mark.gpu

NONFINITE, MAXIT, ERR_ARG, ERR_MESH = -4, -5, -1, -6


def _vortex(**kw):
    from paper_2205_07824_b300.ldg import LDG
    mesh = synth.quad_box(8, hi=(10.0, 10.0), periodic=(True, True))
    g = LDG(mesh, 2, oracle.EULER, oracle.CASE_VORTEX, (1.4,), **kw)
    un, unm1 = g.interpolate(0.0), g.interpolate(-0.05)
    g.set_time(2, 0.05, 0.05, un, unm1)
    return g, un


@pytest.mark.parametrize("precond", [0, 1])
def test_nonfinite_state_is_reported_and_the_context_recovers(precond):
    g, un = _vortex(precond=precond)
    u = un.clone()
    u[17] = float("nan")
    rep = g.newton_gmres(u, check=False)
    assert rep["status"] == NONFINITE, rep
    # the same context then solves a clean step
    u = un.clone()
    rep = g.newton_gmres(u)
    assert rep["status"] == 0 and rep["rfinal"] <= 1e-8 * rep["r0"]


def test_unreachable_tolerance_stops_at_the_newton_cap():
    g, un = _vortex(precond=1, newton_rtol=1e-30, max_newton=3)
    u = un.clone()
    rep = g.newton_gmres(u, check=False)
    assert rep["status"] == MAXIT and rep["newton_iters"] == 3, rep
    assert np.all(np.isfinite(host(u)))


def test_exhausted_restarts_still_update_and_newton_continues():
    """A linear solve that cannot meet its tolerance within its restarts still applies its
    update (inexact Newton); with enough Newton steps the solve still converges."""
    g, un = _vortex(precond=1, gmres_m=2, max_restarts=1, gmres_rtol=1e-12, max_newton=40, newton_rtol=1e-6)
    u = un.clone()
    rep = g.newton_gmres(u, check=False)
    assert rep["status"] == 0 and rep["newton_iters"] > 3, rep
    assert rep["rfinal"] <= 1e-6 * rep["r0"]


def test_batch_isolates_a_failing_instance():
    from paper_2205_07824_b300.ldg import Batch
    meshes = [synth.quad_box(4), synth.quad_box(5), synth.quad_box(6)]
    mus = [(0.05, 1.0, 1.0, 0.0), (0.02, 1.0, 0.6, 0.8), (0.03, 1.0, 0.0, 1.0)]
    b = Batch(meshes, [2, 2, 2], oracle.CONVDIFF, oracle.CASE_SINSIN, mus, precond=1)
    u = np.zeros(b.n_total)
    u[b.offsets[1] + 3] = np.nan
    du = cuda(u)
    reps, _ = b.solve(du, check=False)
    assert reps[1]["status"] == NONFINITE, reps[1]
    for i in (0, 2):
        assert reps[i]["status"] == 0 and reps[i]["rfinal"] <= 1e-8 * reps[i]["r0"], reps[i]
        o = oracle.Oracle(meshes[i], 2, oracle.CONVDIFF, oracle.CASE_SINSIN, mus[i])
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        assert np.linalg.norm(o.residual(host(du)[sl])) <= 2e-8 * np.linalg.norm(o.residual(np.zeros(o.ndof)))


def test_bad_arguments_and_meshes_are_rejected():
    from paper_2205_07824_b300.ldg import LDG, LDGError
    g, un = _vortex()
    v = cuda(np.ones(g.n_dof))
    with pytest.raises(LDGError) as e:
        g.jvp_fd(un, v, order=3)
    assert e.value.code == ERR_ARG
    with pytest.raises(LDGError) as e:
        g.dirk_step(un.clone(), 0.0, 0.1, scheme=9)
    assert e.value.code == ERR_ARG
    with pytest.raises(LDGError):
        g.set_tile(7)
    # a non-conforming mesh: the second quad's face on the shared edge is longer, so no
    # translation (a periodic seam) maps its face points onto the first quad's
    mesh = synth.quad_box((2, 1))
    mesh.xyz[1, 2, 1] += 0.1
    mesh.xyz[1, 3, 1] += 0.1
    with pytest.raises(LDGError) as e:
        LDG(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
    assert e.value.code == ERR_MESH
    # the first context is untouched by the failed creation
    rep = g.newton_gmres(un.clone())
    assert rep["status"] == 0
