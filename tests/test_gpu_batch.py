"""Batched parametrised problems and the tile autotuner.

Parity: the batch residual and J.v of every instance equal the oracle's for that
instance alone (per-element model parameters); every compiled tile gives the same
operator. Solve: each instance of the batched Newton-GMRES meets the Newton
tolerance when its residual is recomputed by the oracle, the graph-driven and the
host-driven loops give bitwise identical results, an instance that is already
solved drops out, and block-Jacobi cuts the Krylov iterations."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, assert_parity, cuda, host

pytestmark = pytest.mark.gpu


def _instances():
    """Mixed batch: orders 1-4, two models, uneven meshes, one sheared, one trivial."""
    rng = np.random.default_rng(7)
    spec = []
    for i, (side, p) in enumerate([(3, 2), (4, 3), (2, 4), (5, 2), (3, 1), (4, 4), (2, 3), (6, 2)]):
        k = float(10 ** rng.uniform(-2, -0.5))
        a = float(rng.uniform(0, 2 * np.pi))
        mesh = synth.quad_box(side, affine=SHEAR2 if i == 3 else None)
        spec.append(dict(mesh=mesh, p=p, mu=(k, 1.0, np.cos(a), np.sin(a)), case=oracle.CASE_SINSIN))
    return spec


def _batch(spec, model=oracle.CONVDIFF, **kw):
    from paper_2205_07824_b300.ldg import Batch
    return Batch([s["mesh"] for s in spec], [s["p"] for s in spec], model, [s["case"] for s in spec],
                 [s["mu"] for s in spec], **kw)


def _oracles(spec, model=oracle.CONVDIFF):
    return [oracle.Oracle(s["mesh"], s["p"], model, s["case"], s["mu"]) for s in spec]


def test_batch_layout():
    spec = _instances()
    b = _batch(spec)
    os_ = _oracles(spec)
    assert b.n_inst == len(spec)
    assert b.n_groups == len({s["p"] for s in spec})
    assert sum(b.n_dof) == b.n_total
    for i, o in enumerate(os_):
        assert b.n_dof[i] == o.ndof
    # the instance slices tile the batch vector exactly once
    cover = np.zeros(b.n_total, dtype=int)
    for i in range(b.n_inst):
        cover[b.offsets[i]:b.offsets[i] + b.n_dof[i]] += 1
    assert (cover == 1).all()


def test_batch_residual_and_jvp_match_oracle_per_instance():
    spec = _instances()
    b = _batch(spec)
    os_ = _oracles(spec)
    u = np.zeros(b.n_total)
    v = np.zeros(b.n_total)
    for i, o in enumerate(os_):
        u[b.offsets[i]:b.offsets[i] + b.n_dof[i]] = synth.random_vector(o.ndof, 100 + i)
        v[b.offsets[i]:b.offsets[i] + b.n_dof[i]] = synth.random_vector(o.ndof, 200 + i)
    r = host(b.residual(cuda(u)))
    jv = host(b.jvp(cuda(u), cuda(v)))
    jv32 = host(b.jvp(cuda(u), cuda(v), precision=1))
    for i, o in enumerate(os_):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        assert_parity(r[sl], o.residual(u[sl]), what=f"R instance {i}")
        ref = o.jvp(u[sl], v[sl])
        assert_parity(jv[sl], ref, what=f"Jv instance {i}")
        assert np.linalg.norm(jv32[sl] - ref) <= 1e-5 * np.linalg.norm(ref), i


@pytest.mark.parametrize("p,model", [(3, oracle.CONVDIFF), (2, oracle.POISSON), (3, oracle.EULER)])
def test_every_tile_matches_oracle(p, model):
    from paper_2205_07824_b300.ldg import LDG
    if model == oracle.EULER:
        mesh = synth.quad_box((5, 4), hi=(10.0, 10.0), periodic=(True, True))
        mu, case = (1.4,), oracle.CASE_VORTEX
    else:
        mesh = synth.quad_box((7, 5), affine=SHEAR2)
        mu, case = ((0.05, 0.3, 1.0, 0.5) if model == oracle.CONVDIFF else (1.0, 1.0)), oracle.CASE_SINSIN
    o = oracle.Oracle(mesh, p, model, case, mu)
    g = LDG(mesh, p, model, case, mu, nq1=o.nq1)
    if model == oracle.EULER:
        u = synth.random_euler_state(mesh.n_elem, o.npe, 3)
    else:
        u = synth.random_vector(o.ndof, 3)
    v = synth.random_vector(o.ndof, 4)
    r_ref, jv_ref = o.residual(u), o.jvp(u, v)
    seen = set()
    for t in range(4):
        g.set_tile(t)
        tile, ne_q, ne_r, ne_j = g.get_tile()
        assert tile == t and ne_r >= 1 and ne_j >= 1
        seen.add((ne_q, ne_r, ne_j))
        assert_parity(host(g.residual(cuda(u))), r_ref, what=f"R tile {t}")
        assert_parity(host(g.jvp(cuda(u), cuda(v))), jv_ref, what=f"Jv tile {t}")
    assert len(seen) >= 2          # the tiles really differ in elements per CTA
    tile, ms = g.autotune(force=True)
    assert 0 <= tile < 4 and ms > 0
    assert g.get_tile()[0] == tile
    tile2, ms2 = g.autotune()          # cached choice
    assert tile2 == tile and ms2 < 0


def _check_solution(b, spec, u, reps, rtol):
    os_ = _oracles(spec)
    for i, o in enumerate(os_):
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        r0 = np.linalg.norm(o.residual(np.zeros(o.ndof)))
        rf = np.linalg.norm(o.residual(u[sl]))
        assert reps[i]["status"] == 0, (i, reps[i])
        assert rf <= 2.0 * rtol * r0, (i, rf / r0, reps[i])
        assert reps[i]["rfinal"] <= rtol * reps[i]["r0"] * (1 + 1e-9)


@pytest.mark.parametrize("pc", [0, 1])
def test_batch_solve_graph_equals_eager_and_converges(pc):
    spec = _instances()
    b = _batch(spec, precond=pc, gmres_m=20, newton_rtol=1e-8, gmres_rtol=1e-3)
    ue = cuda(np.zeros(b.n_total))
    reps_e, _ = b.solve(ue, use_graph=False)
    ug = cuda(np.zeros(b.n_total))
    reps_g, ms = b.solve(ug, use_graph=True)
    assert ms > 0 and b.kernel_executions() > 0
    ue, ug = host(ue), host(ug)
    assert np.array_equal(ue, ug)           # same kernels in the same order
    for a, c in zip(reps_e, reps_g):
        assert a["gmres_iters"] == c["gmres_iters"] and a["newton_iters"] == c["newton_iters"]
    _check_solution(b, spec, ug, reps_g, 1e-8)
    # a second launch of the same graph reproduces the solve
    ug2 = cuda(np.zeros(b.n_total))
    reps_g2, _ = b.solve(ug2)
    assert np.array_equal(host(ug2), ug)
    assert [r["gmres_iters"] for r in reps_g2] == [r["gmres_iters"] for r in reps_g]


def test_batch_matches_single_instance_solves():
    from paper_2205_07824_b300.ldg import LDG
    spec = _instances()[:4]
    b = _batch(spec, precond=1, gmres_m=20)
    u = cuda(np.zeros(b.n_total))
    reps, _ = b.solve(u)
    u = host(u)
    for i, s in enumerate(spec):
        g = LDG(s["mesh"], s["p"], oracle.CONVDIFF, s["case"], s["mu"], gmres_m=20, precond=1)
        ui = cuda(np.zeros(g.n_dof))
        rep = g.newton_gmres(ui)
        ui = host(ui)
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        assert np.linalg.norm(u[sl] - ui) <= 1e-6 * np.linalg.norm(ui), i
        assert rep["newton_iters"] == reps[i]["newton_iters"], (rep, reps[i])
        assert abs(rep["gmres_iters"] - reps[i]["gmres_iters"]) <= max(2, rep["gmres_iters"] // 10)


def test_block_jacobi_reduces_iterations_and_solved_instance_drops_out():
    spec = _instances()
    # instance 0 becomes trivial: zero data, zero initial guess -> R(u0) = 0
    spec[0] = dict(spec[0], case=oracle.CASE_ZERO)
    its = {}
    for pc in (0, 1):
        b = _batch(spec, precond=pc, gmres_m=20)
        u = cuda(np.zeros(b.n_total))
        reps, _ = b.solve(u)
        its[pc] = [r["gmres_iters"] for r in reps]
        assert reps[0]["newton_iters"] == 0 and reps[0]["gmres_iters"] == 0 and reps[0]["r0"] == 0.0
        assert np.all(host(u)[b.offsets[0]:b.offsets[0] + b.n_dof[0]] == 0.0)
        _check_solution(b, spec, host(u), reps, 1e-8)
    assert sum(its[1]) < 0.7 * sum(its[0]), its


def test_batch_fp32_krylov_reaches_fp64_tolerance():
    spec = _instances()
    b = _batch(spec, precond=1, krylov_precision=1, gmres_m=20)
    u = cuda(np.zeros(b.n_total))
    reps, _ = b.solve(u)
    _check_solution(b, spec, host(u), reps, 1e-8)


def test_batch_bdf2_euler_matches_single_context():
    """Time-dependent batch: two BDF2 steps of the vortex (one instance, and the same
    vortex twice) against the single-context solver."""
    from paper_2205_07824_b300.ldg import LDG, Batch, BDF2
    mesh = synth.quad_box(8, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    for n_inst in (1, 2):
        b = Batch([mesh] * n_inst, [3] * n_inst, oracle.EULER, oracle.CASE_VORTEX, [(1.4,)] * n_inst, gmres_m=20,
                  precond=1, krylov_precision=1)
        g = LDG(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, (1.4,), gmres_m=20, precond=1, krylov_precision=1)
        un, unm1 = g.interpolate(0.0), g.interpolate(-dt)
        bun = cuda(np.tile(host(un), n_inst))
        bunm1 = cuda(np.tile(host(unm1), n_inst))
        for k in range(2):
            t1 = (k + 1) * dt
            g.set_time(BDF2, t1, dt, un, unm1)
            u = un.clone()
            rep = g.newton_gmres(u)
            unm1.copy_(un)
            un.copy_(u)
            b.set_time(BDF2, t1, dt, bun, bunm1)
            bu = bun.clone()
            reps, _ = b.solve(bu)
            bunm1.copy_(bun)
            bun.copy_(bu)
            ref = host(un)
            for i in range(n_inst):
                got = host(b.slice(bun, i))
                assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref), (n_inst, k, i)
                assert reps[i]["status"] == 0 and reps[i]["rfinal"] <= 1e-8 * reps[i]["r0"]
                assert reps[i]["newton_iters"] == rep["newton_iters"]


@pytest.mark.parametrize("pc", [0, 1])
def test_pair_basis_batch_matches_fp64_basis(pc):
    """krylov_basis = F32X2 (Gram-Schmidt on (hi, lo) float pairs, emulated FP64) on the
    mixed batch: graph and host-driven loops give the same bits, every instance meets the
    Newton tolerance against the oracle, and the solutions agree with the FP64-basis solve
    to the solve tolerance with about the same GMRES iterations."""
    from paper_2205_07824_b300.ldg import BASIS_F32X2
    spec = _instances()
    b64 = _batch(spec, precond=pc, gmres_m=20, newton_rtol=1e-8, gmres_rtol=1e-3)
    u64 = cuda(np.zeros(b64.n_total))
    reps64, _ = b64.solve(u64)
    bff = _batch(spec, precond=pc, gmres_m=20, newton_rtol=1e-8, gmres_rtol=1e-3, krylov_basis=BASIS_F32X2)
    ue = cuda(np.zeros(bff.n_total))
    reps_e, _ = bff.solve(ue, use_graph=False)
    ug = cuda(np.zeros(bff.n_total))
    reps_g, _ = bff.solve(ug)
    assert np.array_equal(host(ue), host(ug))
    _check_solution(bff, spec, host(ug), reps_g, 1e-8)
    a, c = host(u64), host(ug)
    for i in range(len(spec)):
        sl = slice(bff.offsets[i], bff.offsets[i] + bff.n_dof[i])
        assert np.linalg.norm(a[sl] - c[sl]) <= 1e-6 * np.linalg.norm(a[sl])
        assert abs(reps_g[i]["gmres_iters"] - reps64[i]["gmres_iters"]) <= max(2, reps64[i]["gmres_iters"] // 10)


def test_batch_forcing_last_step_per_instance():
    """newton_forcing = LAST on the mixed batch: each instance's linear tolerance follows
    its own ||R0|| / ||Rk||, every instance still meets the Newton tolerance against the
    oracle, and no instance needs more GMRES iterations than with the fixed forcing term."""
    from paper_2205_07824_b300.ldg import FORCING_LAST
    spec = _instances()
    reps = {}
    for forcing in (0, FORCING_LAST):
        b = _batch(spec, precond=1, gmres_m=20, newton_rtol=1e-8, gmres_rtol=1e-3, newton_forcing=forcing)
        u = cuda(np.zeros(b.n_total))
        reps[forcing], _ = b.solve(u)
        _check_solution(b, spec, host(u), reps[forcing], 1e-8)
    assert sum(r["gmres_iters"] for r in reps[FORCING_LAST]) <= sum(r["gmres_iters"] for r in reps[0])


def test_batch_block_jacobi_reuse_across_solves():
    """pc_reuse = 2 on the mixed batch: the blocks are built by the first of two solve calls
    and reused by the second (pc_setups 1 then 0), which still converges."""
    spec = _instances()
    b = _batch(spec, precond=1, gmres_m=20, newton_rtol=1e-8, gmres_rtol=1e-3, pc_reuse=2)
    setups = []
    for _ in range(3):
        u = cuda(np.zeros(b.n_total))
        reps, _ = b.solve(u)
        setups.append(reps[0]["pc_setups"])
        _check_solution(b, spec, host(u), reps, 1e-8)
    assert setups == [1, 0, 1]
