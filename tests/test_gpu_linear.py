"""The nodal J.v kernels of the linear models on affine quadrilaterals, hexahedra,
triangles and tetrahedra (the same operator as the quadrature-point stage kernels, in
exact nodal form) against the FP64 oracle and against the stage kernels: rotated local
frames (non-trivial face orientations), unstructured simplex meshes, periodic seams,
Dirichlet faces, the BDF mass term, ragged CTA tiles, per-instance parameters of a
batch, the FP32-arithmetic form's error, and the (hi, lo) float-pair form (emulated FP64)
held to the FP64 bar."""
import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu

# vertex orders of a local frame turned by 90 degrees about the last axis (the
# lexicographic order of the rotated frame; the Jacobian keeps its sign)
ROT_QUAD = [1, 3, 0, 2]
ROT_HEX = [1, 3, 0, 2, 5, 7, 4, 6]


def _rotate_some(mesh, every=3):
    """Turns the local frame of every `every`-th element (so faces between turned and
    unturned elements carry non-identity orientations)."""
    perm = ROT_QUAD if mesh.etype == synth.QUAD else ROT_HEX
    m = synth.Mesh(mesh.etype, mesh.xyz.copy(), mesh.vid.copy(), mesh.name)
    for e in range(0, m.n_elem, every):
        m.xyz[e] = mesh.xyz[e][perm]
        m.vid[e] = mesh.vid[e][perm]
    return m


# the nodal J.v kernels of each element type (hexahedra: one thread per node in FP64, one
# per line in FP32 and float pairs)
KNAME = {synth.QUAD: "k_lin_q + k_lin_r", synth.HEX: "k_lin_q + k_lin_r", synth.TRI: "k_sim_q + k_sim_r",
         synth.TET: "k_sim_q + k_sim_r"}
KNAME_LOW = {**KNAME, synth.HEX: "k_hex_q + k_hex_r"}

MESHES = [
    ("quad_rot_p1", lambda: _rotate_some(synth.quad_box((7, 5), affine=SHEAR2)), 1, oracle.POISSON),
    ("quad_rot_p3", lambda: _rotate_some(synth.quad_box((7, 5), affine=SHEAR2)), 3, oracle.CONVDIFF),
    ("quad_per_p4", lambda: _rotate_some(synth.quad_box((6, 5), hi=(2.0, 1.5), periodic=(True, True))), 4,
     oracle.CONVDIFF),
    ("hex_rot_p2", lambda: _rotate_some(synth.hex_box((3, 4, 3), affine=SHEAR3), 2), 2, oracle.CONVDIFF),
    ("hex_per_p4", lambda: _rotate_some(synth.hex_box((3, 3, 3), hi=(1.5, 1.5, 1.5), periodic=(True, True, True),
                                                      affine=SHEAR3)), 4, oracle.CONVDIFF),
    ("hex_p6", lambda: synth.hex_box((2, 2, 3), affine=SHEAR3), 6, oracle.CONVDIFF),
    ("hex_poisson_p1", lambda: _rotate_some(synth.hex_box((4, 3, 3))), 1, oracle.POISSON),
    ("tri_p1", lambda: synth.tri_square(6, affine=SHEAR2), 1, oracle.POISSON),
    ("tri_unstr_p3", lambda: synth.tri_unstructured(7, seed=5), 3, oracle.CONVDIFF),
    ("tri_per_p6", lambda: synth.tri_square(4, hi=(2.0, 2.0), periodic=(True, True), affine=SHEAR2), 6,
     oracle.CONVDIFF),
    ("tet_p2", lambda: synth.tet_cube(2, affine=SHEAR3), 2, oracle.POISSON),
    ("tet_unstr_p3", lambda: synth.tet_unstructured(3, seed=2), 3, oracle.CONVDIFF),
    ("tet_per_p4", lambda: synth.tet_cube(3, hi=(1.5, 1.5, 1.5), periodic=(True, True, True)), 4, oracle.CONVDIFF),
    ("tet_p1", lambda: synth.tet_cube(3, affine=SHEAR3), 1, oracle.CONVDIFF),
]


@pytest.mark.parametrize("name,mk,p,model", MESHES, ids=[m[0] for m in MESHES])
def test_nodal_jv_matches_oracle_and_stage_form(name, mk, p, model):
    from paper_2205_07824_b300.ldg import JV_STAGE
    mesh = mk()
    o, g = pair(mesh, p, model, oracle.CASE_EXPSIN)
    simplex = mesh.etype in (synth.TRI, synth.TET)
    assert g.jv_kernels(0).startswith(KNAME[mesh.etype]), g.jv_kernels(0)
    assert "cartesian" not in g.jv_kernels(0)   # sheared or turned by 90 degrees
    _, gs = pair(mesh, p, model, oracle.CASE_EXPSIN, jv_form=JV_STAGE)
    assert gs.jv_kernels(0).startswith("k_qstage + k_residual"), gs.jv_kernels(0)
    u, v = synth.random_vector(o.ndof, 1), synth.random_vector(o.ndof, 2)
    ref = o.jvp(u, v)
    jv = host(g.jvp(cuda(u), cuda(v)))
    assert_parity(jv, ref, what=f"{name} nodal J.v")
    assert_parity(host(g.residual(cuda(u))), o.residual(u), what=f"{name} R")
    assert_parity(jv, host(gs.jvp(cuda(u), cuda(v))), rtol2=1e-13, rtolmax=1e-12, what=f"{name} nodal vs stage")
    jv32 = host(g.jvp_prec(1, cuda(u), cuda(v)))
    e32 = np.linalg.norm(jv32 - ref) / np.linalg.norm(ref)
    assert e32 <= 2e-6, (name, e32)
    kff = g.jv_kernels(2)
    assert kff.startswith(KNAME_LOW[mesh.etype]) and "f32x2" in kff, kff
    assert g.jv_kernels(1).startswith(KNAME_LOW[mesh.etype]), g.jv_kernels(1)
    assert_parity(host(g.jvp_prec(2, cuda(u), cuda(v))), ref, what=f"{name} float-pair J.v")
    assert gs.jv_kernels(2) == ""
    with pytest.raises(RuntimeError):
        gs.jvp_prec(2, cuda(u), cuda(v))


# vertex orders of a local frame turned by 180 degrees about the last axis: J stays
# diagonal (two negative entries), and faces between turned and unturned elements meet
# with non-identity orientations
TURN_QUAD = [3, 2, 1, 0]
TURN_HEX = [3, 2, 1, 0, 7, 6, 5, 4]


def _turn_some(mesh, every=3):
    perm = TURN_QUAD if mesh.etype == synth.QUAD else TURN_HEX
    m = synth.Mesh(mesh.etype, mesh.xyz.copy(), mesh.vid.copy(), mesh.name)
    for e in range(0, m.n_elem, every):
        m.xyz[e] = mesh.xyz[e][perm]
        m.vid[e] = mesh.vid[e][perm]
    return m


CART_MESHES = [
    ("quad_box_p3", lambda: synth.quad_box((7, 5)), 3, oracle.CONVDIFF),
    ("quad_turned_per_p4", lambda: _turn_some(synth.quad_box((6, 5), hi=(2.0, 1.5), periodic=(True, True))), 4,
     oracle.CONVDIFF),
    ("quad_turned_p2", lambda: _turn_some(synth.quad_box((5, 6))), 2, oracle.POISSON),
    ("hex_box_p4", lambda: synth.hex_box((3, 4, 3)), 4, oracle.CONVDIFF),
    ("hex_turned_per_p2", lambda: _turn_some(synth.hex_box((3, 3, 3), hi=(1.5, 1.5, 1.5),
                                                          periodic=(True, True, True))), 2, oracle.POISSON),
    ("hex_turned_p3", lambda: _turn_some(synth.hex_box((3, 2, 4), hi=(1.0, 0.5, 2.0))), 3, oracle.CONVDIFF),
    ("hex_box_p6", lambda: synth.hex_box((2, 2, 3)), 6, oracle.CONVDIFF),
    # p = 1: every node lies on a face of every axis
    ("quad_turned_p1", lambda: _turn_some(synth.quad_box((5, 4), periodic=(True, False))), 1, oracle.CONVDIFF),
    ("hex_turned_p1", lambda: _turn_some(synth.hex_box((3, 3, 2), periodic=(False, True, False))), 1, oracle.CONVDIFF),
    ("hex_box_p5", lambda: synth.hex_box((2, 3, 2), hi=(1.0, 1.5, 0.5)), 5, oracle.CONVDIFF),
]


@pytest.mark.parametrize("name,mk,p,model", CART_MESHES, ids=[m[0] for m in CART_MESHES])
def test_cartesian_nodal_jv(name, mk, p, model):
    """Meshes of axis-aligned boxes take the nodal instances that leave out the zero
    entries of J^-1 and of the face normals; the result meets the same bars as the general
    instances (oracle, stage form, FP32 error, float pairs), with and without the BDF term."""
    from paper_2205_07824_b300.ldg import JV_STAGE
    mesh = mk()
    o, g = pair(mesh, p, model, oracle.CASE_EXPSIN)
    assert "cartesian" in g.jv_kernels(0), g.jv_kernels(0)
    _, gs = pair(mesh, p, model, oracle.CASE_EXPSIN, jv_form=JV_STAGE)
    u, v = synth.random_vector(o.ndof, 11), synth.random_vector(o.ndof, 12)
    ref = o.jvp(u, v)
    jv = host(g.jvp(cuda(u), cuda(v)))
    assert_parity(jv, ref, what=f"{name} Cartesian nodal J.v")
    assert_parity(jv, host(gs.jvp(cuda(u), cuda(v))), rtol2=1e-13, rtolmax=1e-12, what=f"{name} nodal vs stage")
    e32 = np.linalg.norm(host(g.jvp_prec(1, cuda(u), cuda(v))) - ref) / np.linalg.norm(ref)
    assert e32 <= 2e-6, (name, e32)
    assert_parity(host(g.jvp_prec(2, cuda(u), cuda(v))), ref, what=f"{name} float-pair J.v")
    un, unm1 = synth.random_vector(o.ndof, 13), synth.random_vector(o.ndof, 14)
    o.set_time(2, 0.0, 0.05, un, unm1)
    g.set_time(2, 0.0, 0.05, cuda(un), cuda(unm1))
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what=f"{name} Cartesian nodal J.v, BDF2")


@pytest.mark.parametrize("scheme", [1, 2])
def test_nodal_jv_with_bdf_mass_term(scheme):
    mesh = _rotate_some(synth.hex_box((3, 2, 3), affine=SHEAR3))
    o, g = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN)
    u, un, unm1, v = (synth.random_vector(o.ndof, s) for s in (1, 2, 3, 4))
    o.set_time(scheme, 0.0, 0.07, un, unm1)
    g.set_time(scheme, 0.0, 0.07, cuda(un), cuda(unm1))
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="nodal J.v with the BDF term")
    assert_parity(host(g.jvp_prec(1, cuda(u), cuda(v))), o.jvp(u, v), rtol2=2e-6, rtolmax=2e-5,
                  what="FP32 nodal J.v with the BDF term")
    assert_parity(host(g.jvp_prec(2, cuda(u), cuda(v))), o.jvp(u, v), what="float-pair nodal J.v with the BDF term")


def test_nodal_jv_with_bdf_mass_term_on_tetrahedra():
    mesh = synth.tet_unstructured(2, seed=9)
    o, g = pair(mesh, 2, oracle.CONVDIFF, oracle.CASE_EXPSIN)
    u, un, v = (synth.random_vector(o.ndof, s) for s in (1, 2, 4))
    o.set_time(1, 0.0, 0.05, un, None)
    g.set_time(1, 0.0, 0.05, cuda(un), None)
    assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what="tet nodal J.v with the BDF1 term")
    assert_parity(host(g.jvp_prec(2, cuda(u), cuda(v))), o.jvp(u, v), what="tet float-pair J.v with the BDF1 term")


def test_nodal_jv_ragged_tiles():
    """Element counts that leave a partial last CTA (hex p = 2: 9 elements per CTA;
    quad p = 2: 28 per CTA; tet p = 3: 12; tri p = 2: 42)."""
    for mesh, p in ((synth.hex_box((5, 2, 1)), 2), (synth.quad_box((29, 1)), 2), (synth.tet_cube(2), 3),
                    (synth.tri_square(5), 2)):
        o, g = pair(mesh, p, oracle.CONVDIFF, oracle.CASE_EXPSIN)
        u, v = synth.random_vector(o.ndof, 5), synth.random_vector(o.ndof, 6)
        assert_parity(host(g.jvp(cuda(u), cuda(v))), o.jvp(u, v), what=f"ragged {mesh.etype} p={p}")
        assert_parity(host(g.jvp_prec(2, cuda(u), cuda(v))), o.jvp(u, v), what=f"float-pair ragged {mesh.etype} p={p}")


def test_nodal_jv_in_a_batch_uses_each_instance_parameters():
    """Batched groups look the model parameters up per element: the batch J.v of every
    instance equals its own oracle's."""
    import torch
    from paper_2205_07824_b300.ldg import Batch
    meshes = [synth.quad_box(5), synth.quad_box((4, 6)), synth.quad_box(3)]
    ps = [3, 3, 2]
    mus = [(0.05, 1.0, 1.0, 0.0), (0.002, 0.5, 0.6, -0.8), (0.1, 2.0, -1.0, 0.3)]
    b = Batch(meshes, ps, oracle.CONVDIFF, oracle.CASE_SINSIN, mus)
    u = torch.randn(b.n_total, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    v = torch.randn(b.n_total, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    jv = host(b.jvp(u, v, 0))
    jvff = host(b.jvp(u, v, 2))
    uh, vh = host(u), host(v)
    for i, (m, p, mu) in enumerate(zip(meshes, ps, mus)):
        o = oracle.Oracle(m, p, oracle.CONVDIFF, oracle.CASE_SINSIN, mu)
        sl = slice(b.offsets[i], b.offsets[i] + b.n_dof[i])
        ref = o.jvp(uh[sl], vh[sl])
        assert_parity(jv[sl], ref, what=f"batch instance {i}")
        assert_parity(jvff[sl], ref, what=f"float-pair batch instance {i}")


@pytest.mark.parametrize("scale", [1e-20, 1e-9, 1.0, 1e12, 1e25])
def test_float_pair_jv_is_homogeneous_over_the_float_range(scale):
    """J.v is linear: the float-pair form of J (c v) equals c times the FP64 J v to the
    FP64 bar for c across the magnitudes a pair carries at full precision (the FP64 to
    pair split takes its power of two in one or two factors on either side of 2^-74)."""
    mesh = _rotate_some(synth.hex_box((3, 2, 3), affine=SHEAR3))
    o, g = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN)
    v = synth.random_vector(o.ndof, 8)
    ref = host(g.jvp(cuda(v), cuda(v)))
    got = host(g.jvp_prec(2, cuda(v * scale), cuda(v * scale))) / scale
    assert_parity(got, ref, what=f"float-pair J.v at scale {scale:g}")


def test_float_pair_jv_of_zero_is_zero_and_nonfinite_propagates():
    mesh = synth.quad_box((5, 4), affine=SHEAR2)
    o, g = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN)
    z = np.zeros(o.ndof)
    assert not np.any(host(g.jvp_prec(2, cuda(z), cuda(z))))
    v = synth.random_vector(o.ndof, 3)
    for bad in (np.nan, np.inf):
        w = v.copy()
        w[7] = bad
        out = host(g.jvp_prec(2, cuda(w), cuda(w)))
        assert not np.all(np.isfinite(out)), bad


def test_float_pair_krylov_solve_reaches_the_fp64_solution():
    """Newton-GMRES with the float-pair Krylov J.v (krylov_precision = F32X2) on a hexahedral
    convection-diffusion problem: the same converged state as the FP64 solve, and a
    context whose J.v has no float-pair kernels (the stage-kernel form) refuses the option
    at creation."""
    from paper_2205_07824_b300.ldg import F32X2, LDG, PC_BJACOBI
    mesh = synth.hex_box((4, 3, 3), affine=SHEAR3)
    kw = dict(gmres_m=30, gmres_rtol=1e-10, newton_rtol=1e-10, max_restarts=100, precond=PC_BJACOBI)
    o, g64 = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN, **kw)
    _, gff = pair(mesh, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN, krylov_precision=F32X2, **kw)
    u64, uff = cuda(np.zeros(o.ndof)), cuda(np.zeros(o.ndof))
    r64, rff = g64.newton_gmres(u64), gff.newton_gmres(uff)
    assert r64["status"] == 0 and rff["status"] == 0, (r64, rff)
    assert np.linalg.norm(host(uff) - host(u64)) <= 1e-9 * np.linalg.norm(host(u64))
    assert abs(rff["gmres_iters"] - r64["gmres_iters"]) <= 2, (rff, r64)
    from paper_2205_07824_b300.ldg import JV_STAGE
    with pytest.raises(RuntimeError):
        LDG(mesh, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN, (0.05, 0.3, 1.0, 0.5, 0.25), krylov_precision=F32X2,
            jv_form=JV_STAGE)
