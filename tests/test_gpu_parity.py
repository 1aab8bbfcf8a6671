"""Parity of the CUDA LDG kernels with the FP64 CPU oracle (Section 2.2, Eq. 1a-1b;
Section 3.3), element by element, on seeded inputs. Sizes span several CTA tiles
with a ragged last tile; meshes are sheared so that every geometric factor is
exercised."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, assert_parity, cuda, host, pair, state

pytestmark = pytest.mark.gpu


def _run_r_jv(mesh, p, model, case, seed=1):
    o, g = pair(mesh, p, model, case)
    u = state(o, mesh, seed)
    v = synth.random_vector(o.ndof, seed + 100)
    r = host(g.residual(cuda(u)))
    assert_parity(r, o.residual(u), what="R")
    jv = host(g.jvp(cuda(u), cuda(v)))
    assert_parity(jv, o.jvp(u, v), what="J.v")
    return o, g


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("model,case", [(oracle.POISSON, oracle.CASE_SINSIN), (oracle.CONVDIFF, oracle.CASE_EXPSIN)])
def test_triangles(p, model, case):
    _run_r_jv(synth.tri_square(7, affine=SHEAR2), p, model, case)


@pytest.mark.parametrize("kind,p", [("tri", 1), ("tri", 3), ("tri", 6), ("tet", 1), ("tet", 3)])
@pytest.mark.parametrize("model,case", [(oracle.POISSON, oracle.CASE_SINSIN), (oracle.CONVDIFF, oracle.CASE_EXPSIN)])
def test_unstructured_simplices(kind, p, model, case):
    """R and J.v on unstructured simplex meshes (random diagonals, jittered vertices,
    rotated local numbering, shuffled elements; several tiles with a ragged last one)."""
    mesh = synth.tri_unstructured(9, seed=7) if kind == "tri" else synth.tet_unstructured(3, seed=4)
    _run_r_jv(mesh, p, model, case)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("model,case", [(oracle.POISSON, oracle.CASE_SINSIN), (oracle.CONVDIFF, oracle.CASE_EXPSIN)])
def test_quads_dirichlet(p, model, case):
    _run_r_jv(synth.quad_box((7, 5), affine=SHEAR2), p, model, case)


def test_quads_periodic_convdiff():
    _run_r_jv(synth.quad_box((6, 5), hi=(2.0, 1.5), periodic=(True, True), affine=SHEAR2), 2,
              oracle.CONVDIFF, oracle.CASE_ZERO)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_euler_periodic(p):
    mesh = synth.quad_box((7, 6), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    _run_r_jv(mesh, p, oracle.EULER, oracle.CASE_VORTEX)


def test_euler_far_field_boundary():
    mesh = synth.quad_box((5, 4), hi=(10.0, 10.0))
    _run_r_jv(mesh, 2, oracle.EULER, oracle.CASE_VORTEX)


def test_euler_walls_on_affine_quadrilaterals():
    """Periodic in x, no-slip walls at y = 0 and y = 10 (wall marks on affine elements)."""
    mesh = synth.quad_box((6, 5), hi=(10.0, 10.0), periodic=(True, False))
    bc = np.zeros((mesh.n_elem, 4), dtype=np.uint8)
    bc[:6, 2] = 1
    bc[-6:, 3] = 1
    mesh.bc = bc
    _run_r_jv(mesh, 3, oracle.EULER, oracle.CASE_VORTEX)


@pytest.mark.parametrize("p,n", [(1, (3, 4, 5)), (2, (3, 4, 5)), (3, (3, 3, 4)), (4, (3, 3, 3)), (5, (2, 2, 3)),
                                 (6, (2, 2, 2))])
def test_hexes_convdiff(p, n):
    _run_r_jv(synth.hex_box(n, affine=SHEAR3), p, oracle.CONVDIFF, oracle.CASE_EXPSIN)


@pytest.mark.parametrize("p", [1, 2])
def test_hexes_poisson(p):
    _run_r_jv(synth.hex_box((3, 4, 3), affine=SHEAR3), p, oracle.POISSON, oracle.CASE_SINSIN)


@pytest.mark.parametrize("etype,p", [(0, 2), (1, 3), (2, 2)])
def test_q_stage(etype, p):
    mesh = {0: synth.tri_square(5, affine=SHEAR2), 1: synth.quad_box((5, 4), affine=SHEAR2),
            2: synth.hex_box((3, 3, 2), affine=SHEAR3)}[etype]
    o, g = pair(mesh, p, oracle.POISSON, oracle.CASE_SINSIN)
    u = synth.random_vector(o.ndof, 7)
    assert_parity(host(g.q(cuda(u))), o.q(u), what="q")


def test_interpolation_matches_oracle():
    mesh = synth.quad_box((6, 6), hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX)
    assert_parity(host(g.interpolate(0.3)), o.interpolate(0.3), what="interp")


@pytest.mark.parametrize("scheme", [1, 2])
def test_bdf_time_terms(scheme):
    mesh = synth.quad_box((5, 6), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    o, g = pair(mesh, 2, oracle.EULER, oracle.CASE_VORTEX)
    u, un, unm1 = (synth.random_euler_state(mesh.n_elem, o.npe, s) for s in (1, 2, 3))
    v = synth.random_vector(o.ndof, 4)
    o.set_time(scheme, 0.1, 0.05, un, unm1)
    g.set_time(scheme, 0.1, 0.05, cuda(un), cuda(unm1))
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R bdf")
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="Jv bdf")
    mesh = synth.hex_box((3, 2, 2), affine=SHEAR3)
    o, g = pair(mesh, 2, oracle.CONVDIFF, oracle.CASE_EXPSIN)
    u, un, unm1 = (synth.random_vector(o.ndof, s) for s in (1, 2, 3))
    o.set_time(scheme, 0.0, 0.1, un, unm1)
    g.set_time(scheme, 0.0, 0.1, cuda(un), cuda(unm1))
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R bdf cd")
    assert_parity(host(g.jvp(cuda(u), cuda(v[: o.ndof]))), o.jvp(u, v[: o.ndof]), what="Jv bdf cd")


def test_bitwise_reproducible():
    mesh = synth.quad_box((9, 7), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX)
    u = cuda(state(o, mesh, 5))
    v = cuda(synth.random_vector(o.ndof, 6))
    a = host(g.jvp(u, v))
    b = host(g.jvp(u, v))
    assert np.array_equal(a, b)


# ------------------------------------------------------------ full workloads
def test_full_poisson_512_triangles_p2():
    """2-D Poisson, p = 2 on 16 x 16 squares split into 512 triangles."""
    _run_r_jv(synth.tri_square(16), 2, oracle.POISSON, oracle.CASE_SINSIN)


def test_full_euler_vortex_64x64_p3():
    """Isentropic vortex, periodic [0,10]^2, 64 x 64 quadrilaterals, p = 3, BDF2 step."""
    mesh = synth.quad_box(64, hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX)
    un = o.interpolate(0.0)
    unm1 = o.interpolate(-0.05)
    o.set_time(2, 0.05, 0.05, un, unm1)
    g.set_time(2, 0.05, 0.05, cuda(un), cuda(unm1))
    # a perturbed state: at the interpolated exact solution R is a near-cancellation
    u = o.interpolate(0.05) + 1e-2 * synth.random_vector(o.ndof, 4)
    v = synth.random_vector(o.ndof, 3)
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what="R vortex 64x64")
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="Jv vortex 64x64")


def test_full_convdiff_hex48_p4_sampled():
    """3-D convection-diffusion on 48^3 hexahedra, p = 4 (13.8 M DOF): the kernel runs
    on the full mesh; the oracle evaluates a sample of elements (corners, faces, interior)."""
    n = 48
    mesh = synth.hex_box(n)
    o, g = pair(mesh, 4, oracle.CONVDIFF, oracle.CASE_EXPSIN, mu=(1e-2, 1e-2, 1.0, 0.5, 0.25), gmres_m=2)
    u = synth.random_vector(o.ndof, 0)
    v = synth.random_vector(o.ndof, 1)
    rng = np.random.default_rng(0)
    el = np.unique(np.concatenate([[0, n - 1, n * n - 1, mesh.n_elem - 1, mesh.n_elem // 2],
                                   rng.integers(0, mesh.n_elem, 40)]))
    npe = o.npe
    r = host(g.residual(cuda(u))).reshape(-1, 1, npe)[el]
    assert_parity(r, o.residual_some(u, el), what="R hex 48^3")
    jv = host(g.jvp(cuda(u), cuda(v))).reshape(-1, 1, npe)[el]
    ref = o.jvp_some(u, v, el)
    assert_parity(jv, ref, what="Jv hex 48^3")
    # the (hi, lo) float-pair J.v of the same operator, held to the FP64 bar
    jvff = host(g.jvp_prec(2, cuda(u), cuda(v))).reshape(-1, 1, npe)[el]
    assert_parity(jvff, ref, what="float-pair Jv hex 48^3")


# ------------------------------------------------------------------- solvers
def test_gmres_matches_oracle_solve():
    mesh = synth.quad_box((6, 6), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    o, g = pair(mesh, 2, oracle.EULER, oracle.CASE_VORTEX, gmres_rtol=1e-11, gmres_m=30, max_restarts=200)
    u = o.interpolate(0.0)
    o.set_time(1, 0.0, 0.2, u, u)
    g.set_time(1, 0.0, 0.2, cuda(u), cuda(u))
    b = synth.random_vector(o.ndof, 2)
    x, rep = g.gmres(cuda(u), cuda(b))
    x = host(x)
    xo, its, rc, _ = o.gmres(u, b, m=30, rtol=1e-12, maxit=5000)
    assert rc == 0
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo), rep
    assert rep["lin_resid"] <= 1e-11 * 1.01


def test_newton_poisson_512_triangles_one_step():
    """2-D Poisson on 512 triangles, p = 2: one Newton step from u = 0 with unpreconditioned GMRES to 1e-10."""
    mesh = synth.tri_square(16)
    o, g = pair(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN, gmres_m=30, gmres_rtol=1e-10,
                max_restarts=400, newton_rtol=1e-9, max_newton=1)
    u = cuda(np.zeros(o.ndof))
    rep = g.newton_gmres(u)
    uo, rc, st = o.newton(np.zeros(o.ndof), m=200, newton_rtol=1e-9, gmres_rtol=1e-11, max_newton=3)
    assert rep["newton_iters"] == 1 and rep["rfinal"] <= 1e-9 * rep["r0"]
    ug = host(u)
    assert np.linalg.norm(ug - uo) <= 1e-8 * np.linalg.norm(uo)
    eu, _ = o.l2_error(ug)
    euo, _ = o.l2_error(uo)
    assert abs(eu - euo) <= 1e-6 * euo


def test_newton_vortex_bdf2_step_16x16():
    """One BDF2 step of the vortex by Newton-GMRES to 1e-8 on a 16 x 16 mesh, p = 3."""
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-4)
    dt = 0.05
    un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
    o.set_time(2, dt, dt, un, unm1)
    g.set_time(2, dt, dt, cuda(un), cuda(unm1))
    u = cuda(un)
    rep = g.newton_gmres(u)
    assert rep["rfinal"] <= 1e-8 * rep["r0"]
    uo, rc, st = o.newton(un.copy(), m=30, newton_rtol=1e-10, gmres_rtol=1e-6)
    assert rc == 0
    ug = host(u)
    # both satisfy ||R|| <= 1e-8 ||R0||; the solutions agree to the solve tolerance
    assert np.linalg.norm(ug - uo) <= 1e-7 * np.linalg.norm(uo)
    assert np.linalg.norm(o.residual(ug)) <= 1.5e-8 * st["r0"]


@pytest.mark.parametrize("kprec,pc", [(0, 0), (1, 1)])
def test_newton_forcing_last_step(kprec, pc):
    """newton_forcing = LAST loosens only the linear tolerance that the Newton test does
    not need (at least half of newton_rtol ||R0|| / ||Rk||): the BDF2 vortex step still
    reaches ||R|| <= 1e-8 ||R0||, with no more GMRES iterations than the fixed forcing
    term, and both solutions agree with the oracle's tight solve."""
    from paper_2205_07824_b300.ldg import FORCING_FIXED, FORCING_LAST
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    reps, sols = {}, {}
    for forcing in (FORCING_FIXED, FORCING_LAST):
        o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3,
                    krylov_precision=kprec, precond=pc, newton_forcing=forcing)
        un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
        g.set_time(2, dt, dt, cuda(un), cuda(unm1))
        u = cuda(un)
        reps[forcing] = g.newton_gmres(u)
        sols[forcing] = host(u)
    o.set_time(2, dt, dt, un, unm1)
    uo, rc, st = o.newton(un.copy(), m=30, newton_rtol=1e-10, gmres_rtol=1e-6)
    assert rc == 0
    print({f: (r["newton_iters"], r["gmres_iters"], r["rfinal"] / r["r0"]) for f, r in reps.items()})
    for forcing, rep in reps.items():
        assert rep["rfinal"] <= 1e-8 * rep["r0"]
        assert np.linalg.norm(sols[forcing] - uo) <= 1e-7 * np.linalg.norm(uo)
        assert np.linalg.norm(o.residual(sols[forcing])) <= 1.5e-8 * st["r0"]
    assert reps[FORCING_LAST]["gmres_iters"] <= reps[FORCING_FIXED]["gmres_iters"]
    assert reps[FORCING_LAST]["newton_iters"] == reps[FORCING_FIXED]["newton_iters"]


def test_block_jacobi_reuse_over_time_steps():
    """pc_reuse = 3: the block-Jacobi blocks are built at the first of every three solve
    calls and reused in between (reported pc_setups 1, 0, 0, 1), a change of dt rebuilds
    them, and every step still reaches the Newton tolerance with a solution that agrees
    with the one rebuilt every step."""
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    sols, setups = {}, {}
    for reuse in (1, 3):
        o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3,
                    krylov_precision=1, precond=1, pc_reuse=reuse)
        um1, u0 = o.interpolate(-dt), o.interpolate(0.0)
        prev, cur = cuda(um1), cuda(u0)
        setups[reuse], sols[reuse] = [], []
        for step in range(4):
            g.set_time(2, (step + 1) * dt, dt, cur, prev)
            u = cur.clone()
            rep = g.newton_gmres(u)
            assert rep["rfinal"] <= 1e-8 * rep["r0"]
            setups[reuse].append(rep["pc_setups"])
            sols[reuse].append(host(u))
            prev, cur = cur, u
        # a new dt changes the BDF mass coefficient: the blocks are rebuilt at once
        g.set_time(2, 5 * dt, 0.5 * dt, cur, prev)
        setups[reuse].append(g.newton_gmres(cur.clone())["pc_setups"])
    assert setups[1] == [1, 1, 1, 1, 1]
    assert setups[3] == [1, 0, 0, 1, 1]
    for a, b in zip(sols[1], sols[3]):
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(a)


@pytest.mark.parametrize("kprec,pc", [(0, 0), (1, 1)])
def test_pair_basis_vortex_step(kprec, pc):
    """The BDF2 vortex step with the Gram-Schmidt sweeps on (hi, lo) float pairs reaches
    the Newton tolerance, agrees with the oracle's tight solve like the FP64-basis solve,
    and needs about the same GMRES iterations."""
    from paper_2205_07824_b300.ldg import BASIS_FP64, BASIS_F32X2
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    reps, sols = {}, {}
    for basis in (BASIS_FP64, BASIS_F32X2):
        o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3,
                    krylov_precision=kprec, precond=pc, krylov_basis=basis)
        un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
        g.set_time(2, dt, dt, cuda(un), cuda(unm1))
        u = cuda(un)
        reps[basis] = g.newton_gmres(u)
        sols[basis] = host(u)
    o.set_time(2, dt, dt, un, unm1)
    uo, rc, st = o.newton(un.copy(), m=30, newton_rtol=1e-10, gmres_rtol=1e-6)
    assert rc == 0
    print({b: (r["newton_iters"], r["gmres_iters"]) for b, r in reps.items()})
    for basis, rep in reps.items():
        assert rep["rfinal"] <= 1e-8 * rep["r0"]
        assert np.linalg.norm(sols[basis] - uo) <= 1e-7 * np.linalg.norm(uo)
    n64, nff = reps[BASIS_FP64]["gmres_iters"], reps[BASIS_F32X2]["gmres_iters"]
    assert abs(nff - n64) <= max(2, n64 // 10)


def test_host_buffer_solve_equals_device_solve():
    """ldg_newton_gmres_host (state in host memory, copied in and out by the library)
    gives the bits and the report of ldg_newton_gmres on a device buffer."""
    mesh = synth.quad_box(8, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3,
                krylov_precision=1, precond=1)
    un, unm1 = o.interpolate(0.0), o.interpolate(-dt)
    g.set_time(2, dt, dt, cuda(un), cuda(unm1))
    ud = cuda(un)
    rd = g.newton_gmres(ud)
    uh = np.ascontiguousarray(un.copy())
    rh = g.newton_gmres_host(uh)
    assert np.array_equal(uh, host(ud))
    assert (rh["newton_iters"], rh["gmres_iters"], rh["status"]) == (rd["newton_iters"], rd["gmres_iters"], 0)


@pytest.mark.parametrize("model,prec", [(oracle.EULER, 0), (oracle.NS, 1), (oracle.CONVDIFF, 0), (oracle.CONVDIFF, 2)])
def test_host_many_jvp_equals_device_jvp(model, prec):
    """ldg_jvp_host_many (directions in pinned host memory, copies overlapped with the J.v
    of the neighbouring directions through two device slots) gives, for each of five
    directions, the bits of ldg_jvp_prec on device buffers; outputs that share one host
    buffer keep the last direction's result; the FP64 result meets the oracle."""
    import torch
    if model == oracle.CONVDIFF:
        mesh, p, case = synth.hex_box((3, 4, 3)), 3, oracle.CASE_EXPSIN
    else:
        mesh, p, case = synth.quad_box((6, 5), hi=(10.0, 10.0), periodic=(True, True)), 3, oracle.CASE_VORTEX
    o, g = pair(mesh, p, model, case, gmres_m=2)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 21) if model in (oracle.EULER, oracle.NS) else \
        synth.random_vector(o.ndof, 21)
    vs = [torch.from_numpy(synth.random_vector(o.ndof, 30 + i)).pin_memory() for i in range(5)]
    outs = [torch.full((o.ndof,), float("nan"), dtype=torch.float64).pin_memory() for _ in range(4)]
    uh = None if model == oracle.CONVDIFF else torch.from_numpy(u).pin_memory()
    g.jvp_host_many(prec, uh, vs, outs + [outs[0]])    # the fifth result overwrites the first
    for i, v in enumerate(vs):
        ref = host(g.jvp_prec(prec, cuda(u), cuda(v.numpy())))
        got = outs[0].numpy() if i in (0, 4) else outs[i].numpy()
        if i == 0:
            continue
        assert np.array_equal(got, ref), (i, np.abs(got - ref).max())
        if prec == 0:
            assert_parity(got, o.jvp(u, v.numpy()), what=f"host-many J.v direction {i}")
    with pytest.raises(RuntimeError):
        g.jvp_host_many(prec, uh, vs[:0] + [vs[0]], [None])


@pytest.mark.parametrize("model", [oracle.EULER, oracle.NS, oracle.CONVDIFF])
def test_finite_difference_jvp(model):
    """The FD variant against the exact J.v: the forward difference is off by O(eps),
    the central one by O(eps^2) plus rounding of order 2^-52 ||R|| / eps, below the
    forward one; for the linear model both reproduce R(v) - R(0) up to rounding / eps."""
    mesh = synth.quad_box((5, 4), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    mu = {oracle.EULER: (1.4,), oracle.NS: (1.4, 10.0, 0.72), oracle.CONVDIFF: (0.05, 0.3, 1.0, 0.5)}[model]
    o, g = pair(mesh, 3, model, oracle.CASE_VORTEX if model != oracle.CONVDIFF else oracle.CASE_SINSIN, mu=mu)
    u, v = state(o, mesh, 3), synth.random_vector(o.ndof, 4)
    ref = o.jvp(u, v)
    nrm = np.linalg.norm(ref)
    e1 = np.linalg.norm(host(g.jvp_fd(cuda(u), cuda(v), 1)) - ref) / nrm
    e2 = np.linalg.norm(host(g.jvp_fd(cuda(u), cuda(v), 2)) - ref) / nrm
    print(f"FD J.v relative error, model {model}: forward {e1:.2e}, central {e2:.2e}")
    assert e1 < 1e-5 and e2 < 1e-6
    if model != oracle.CONVDIFF:
        assert e2 < e1           # central: O(eps^2), here already down to rounding / eps
    assert np.all(host(g.jvp_fd(cuda(u), cuda(np.zeros(o.ndof)), 2)) == 0.0)


@pytest.mark.parametrize("scheme", [1, 2, 3, 4])
def test_dirk_step_matches_oracle(scheme):
    """One DIRK step of the vortex (Euler) and of the viscous vortex (Navier-Stokes)
    against the oracle's DIRK step, both solved to a tight Newton tolerance."""
    for model, mu in ((oracle.EULER, (1.4,)), (oracle.NS, (1.4, 100.0, 0.72))):
        mesh = synth.quad_box(6, hi=(10.0, 10.0), periodic=(True, True))
        o, g = pair(mesh, 2, model, oracle.CASE_VORTEX, mu=mu, newton_rtol=1e-11, gmres_rtol=1e-8,
                    max_restarts=200, precond=1)
        u0 = o.interpolate(0.0)
        ref, _ = o.dirk_step(u0, 0.0, 0.2, scheme, newton_rtol=1e-12, gmres_rtol=1e-10, m=30, max_gmres=20000)
        u = cuda(u0)
        rep = g.dirk_step(u, 0.0, 0.2, scheme)
        assert rep["status"] == 0 and rep["newton_iters"] >= 1
        got = host(u)
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref), (model, np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_dirk_temporal_order_on_gpu():
    """GPU DIRK steps on the linear semi-discrete problem of the oracle pin converge to
    the exact solution (matrix exponential computed from the oracle's operators) at the
    schemes' orders."""
    import scipy.linalg as sl
    mesh = synth.quad_box(3, hi=(2.0, 2.0), periodic=(True, True))
    mu = (0.02, 0.3, 1.0, 0.5)
    o, g = pair(mesh, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, mu=mu, newton_rtol=1e-12, gmres_rtol=1e-12,
                max_restarts=200)
    n = o.ndof
    A = o.jacobian_cs(np.zeros(n))
    r0 = o.residual(np.zeros(n))
    M = np.stack([o.mass(e) for e in np.eye(n)], 1)
    ustar = -np.linalg.solve(A, r0)
    u0 = o.interpolate()
    T = 0.25
    yT = ustar + sl.expm(-T * np.linalg.solve(M, A)) @ (u0 - ustar)
    for scheme, order in ((1, 1), (2, 2), (3, 3), (4, 4)):
        errs = []
        for N in (16, 32):
            u, t = cuda(u0), 0.0
            for _ in range(N):
                g.dirk_step(u, t, T / N, scheme)
                t += T / N
            errs.append(np.linalg.norm(host(u) - yT) / np.linalg.norm(yT))
        assert np.log2(errs[0] / errs[1]) > order - 0.3, (scheme, errs)

