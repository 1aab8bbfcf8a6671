"""Pins of the FP64 CPU oracle against what the mathematics and the paper fix.

Each test targets a mistake that could hide in the oracle: a wrong quadrature
or basis (exactness, partition of unity), a dropped or mis-signed term
(patch test, conservation, free stream, symmetry and definiteness, upwind
dissipation, the Riemann-jump closed form), a wrong derivative (complex step),
and the convergence rates stated in Section 4.1 / Table 3.
"""
import json
import math
from fractions import Fraction
import os

import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SHEAR2 = np.array([[1.0, 0.3], [0.1, 0.9]])
SHEAR3 = np.array([[1.0, 0.2, 0.1], [0.0, 0.9, 0.15], [0.05, 0.0, 1.1]])


def _mesh(etype, n, **kw):
    return {0: synth.tri_square, 1: synth.quad_box, 2: synth.hex_box, 3: synth.tet_cube}[etype](n, **kw)


# ---------------------------------------------------------------- reference rules
def test_gauss_and_gll_closed_forms():
    o = oracle.Oracle(synth.quad_box(2), 2, oracle.POISSON, oracle.CASE_ZERO, nq1=3)
    nodes, qx, qw, fs, fw = o.ref_rules()
    # 3-point Gauss-Legendre: 0, +-sqrt(3/5); weights 8/9, 5/9
    assert np.allclose(np.sort(fs[:, 0]), [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(fw[np.argsort(fs[:, 0])], [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    # GLL with 3 points: -1, 0, 1
    assert np.allclose(np.unique(nodes[:, 0]), [-1, 0, 1], atol=1e-15)
    o = oracle.Oracle(synth.quad_box(2), 3, oracle.POISSON, oracle.CASE_ZERO)
    assert np.allclose(np.unique(o.ref_rules()[0][:, 0]), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1],
                       atol=1e-15)
    o = oracle.Oracle(synth.quad_box(2), 4, oracle.POISSON, oracle.CASE_ZERO)
    assert np.allclose(np.unique(o.ref_rules()[0][:, 0]),
                       [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)


def _tri_monomial_integral(a, b):
    # integral of xi^a eta^b over the triangle (-1,-1),(1,-1),(-1,1): with xi = 2s-1,
    # eta = 2t-1 on the unit triangle, and int s^m t^n = m! n! / (m+n+2)!; summed in
    # exact rationals (the alternating sum cancels badly in floating point at high degree)
    tot = Fraction(0)
    for m in range(a + 1):
        for n in range(b + 1):
            c = math.comb(a, m) * math.comb(b, n) * 2 ** (m + n) * (-1) ** (a - m + b - n)
            tot += Fraction(c * math.factorial(m) * math.factorial(n), math.factorial(m + n + 2))
    return float(4 * tot)


@pytest.mark.parametrize("nq1", [2, 3, 4, 5, 6, 7, 8])
def test_triangle_rule_exactness(nq1):
    o = oracle.Oracle(synth.tri_square(1), 1, oracle.POISSON, oracle.CASE_ZERO, nq1=nq1)
    _, qx, qw, _, _ = o.ref_rules()
    for a in range(2 * nq1 - 1):
        for b in range(2 * nq1 - 1 - a):
            got = np.sum(qw * qx[:, 0] ** a * qx[:, 1] ** b)
            assert abs(got - _tri_monomial_integral(a, b)) < 1e-13, (a, b)


def _tet_monomial_integral(a, b, c):
    # integral of xi^a eta^b zeta^c over the reference tetrahedron: with xi = 2s - 1 etc.
    # on the unit tetrahedron, int s^m t^n r^l = m! n! l! / (m + n + l + 3)!
    tot = Fraction(0)
    for m in range(a + 1):
        for n in range(b + 1):
            for l in range(c + 1):
                cf = (math.comb(a, m) * math.comb(b, n) * math.comb(c, l) * 2 ** (m + n + l)
                      * (-1) ** (a - m + b - n + c - l))
                tot += Fraction(cf * math.factorial(m) * math.factorial(n) * math.factorial(l),
                                math.factorial(m + n + l + 3))
    return float(8 * tot)


@pytest.mark.parametrize("nq1", [2, 3, 4, 5, 6])
def test_tetrahedron_rule_exactness(nq1):
    """The collapsed Gauss rule with nq1 points per direction is exact to total degree
    2 nq1 - 3 (its Jacobian factor (1-b)(1-c)^2 / 8 spends two degrees in c)."""
    o = oracle.Oracle(synth.tet_cube(1), 1, oracle.POISSON, oracle.CASE_ZERO, nq1=nq1)
    _, qx, qw, fs, fw = o.ref_rules()
    deg = 2 * nq1 - 3
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                got = np.sum(qw * qx[:, 0] ** a * qx[:, 1] ** b * qx[:, 2] ** c)
                assert abs(got - _tet_monomial_integral(a, b, c)) < 1e-13, (a, b, c)
    # faces: the collapsed triangle rule in the face parameters
    for a in range(2 * nq1 - 1):
        for b in range(2 * nq1 - 1 - a):
            got = np.sum(fw * fs[:, 0] ** a * fs[:, 1] ** b)
            assert abs(got - _tri_monomial_integral(a, b)) < 1e-13, (a, b)


@pytest.mark.parametrize("etype", [1, 2])
def test_tensor_rule_exactness(etype):
    nq1 = 3
    o = oracle.Oracle(_mesh(etype, 1), 1, oracle.POISSON, oracle.CASE_ZERO, nq1=nq1)
    _, qx, qw, _, _ = o.ref_rules()
    nd = 2 if etype == 1 else 3

    def exact1(a):
        return 0.0 if a % 2 else 2.0 / (a + 1)
    for a in range(2 * nq1):
        for b in range(2 * nq1):
            c = 1 if nd == 3 else 0
            got = np.sum(qw * qx[:, 0] ** a * qx[:, 1] ** b * (qx[:, 2] ** c if nd == 3 else 1))
            ref = exact1(a) * exact1(b) * (exact1(c) if nd == 3 else 1)
            assert abs(got - ref) < 1e-13


@pytest.mark.parametrize("etype,p", [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (0, 6), (1, 1), (1, 3), (1, 5), (2, 2),
                                     (2, 4), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_basis_partition_and_kronecker(etype, p):
    o = oracle.Oracle(_mesh(etype, 1), p, oracle.POISSON, oracle.CASE_ZERO)
    nodes = o.ref_rules()[0]
    phi, _ = o.basis(nodes)
    assert np.allclose(phi, np.eye(o.npe), atol=1e-12)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, (20, 3))
    if etype == 0:
        pts[:, :2] = np.where((pts[:, 0] + pts[:, 1] > 0)[:, None], -pts[:, :2], pts[:, :2])
    if etype == 3:
        # points of the reference tetrahedron: barycentric draws
        lam = rng.dirichlet(np.ones(4), 20)
        V = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
        pts = lam @ V
    phi, dphi = o.basis(pts)
    assert np.allclose(phi.sum(1), 1, atol=1e-12)
    assert np.allclose(dphi.sum(1), 0, atol=1e-11)


# ------------------------------------------------------------- discretisation
@pytest.mark.parametrize("etype,p,model,case", [
    (0, 1, oracle.POISSON, oracle.CASE_LINEAR), (0, 2, oracle.POISSON, oracle.CASE_POLY2),
    (0, 3, oracle.CONVDIFF, oracle.CASE_POLY2), (1, 1, oracle.CONVDIFF, oracle.CASE_LINEAR),
    (1, 2, oracle.POISSON, oracle.CASE_POLY2), (1, 3, oracle.CONVDIFF, oracle.CASE_POLY2),
    (2, 2, oracle.CONVDIFF, oracle.CASE_POLY2), (2, 1, oracle.POISSON, oracle.CASE_LINEAR),
    (3, 1, oracle.POISSON, oracle.CASE_LINEAR), (3, 2, oracle.CONVDIFF, oracle.CASE_POLY2),
    (3, 3, oracle.POISSON, oracle.CASE_POLY2), (0, 4, oracle.POISSON, oracle.CASE_POLY2),
    (0, 5, oracle.CONVDIFF, oracle.CASE_LINEAR), (0, 6, oracle.CONVDIFF, oracle.CASE_POLY2),
    (3, 4, oracle.CONVDIFF, oracle.CASE_POLY2)])
def test_patch_test(etype, p, model, case):
    """Consistency + uniqueness of LDG: a polynomial of degree <= p (with q = -grad u
    and the matching source/boundary data) has zero residual."""
    aff = SHEAR3 if etype >= 2 else SHEAR2
    mesh = _mesh(etype, 3 if etype < 2 else 2, affine=aff)
    mu = (0.7, 1.3) if model == oracle.POISSON else (0.05, 0.4, 1.0, -0.6, 0.3)
    o = oracle.Oracle(mesh, p, model, case, mu)
    u = o.interpolate()
    r = o.residual(u)
    assert np.abs(r).max() < 1e-12 * max(1.0, np.abs(o.residual(np.zeros_like(u))).max())


NS_MU = (1.4, 10.0, 0.72)          # gamma, Re, Pr (penalty tau = 1/Re)


@pytest.mark.parametrize("etype,model", [(0, oracle.POISSON), (1, oracle.CONVDIFF), (2, oracle.CONVDIFF),
                                         (1, oracle.EULER), (1, oracle.NS), (3, oracle.CONVDIFF)])
def test_conservation_periodic(etype, model):
    """Single-valued numerical fluxes and sum_i phi_i = 1: on a periodic mesh with no
    source, the sum of all element residuals vanishes for any state."""
    n = 3
    nd = 3 if etype in (2, 3) else 2
    mesh = _mesh(etype, n, hi=(2.0,) * nd, periodic=(True,) * nd)
    mu = {oracle.POISSON: (1.0, 1.0), oracle.CONVDIFF: (0.1, 0.2, 1.0, 0.5, 0.25), oracle.EULER: (1.4,),
          oracle.NS: NS_MU}[model]
    gas = model in (oracle.EULER, oracle.NS)
    o = oracle.Oracle(mesh, 2, model, oracle.CASE_CONST if gas else oracle.CASE_ZERO, mu)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 3) if gas else synth.random_vector(o.ndof, 3)
    r = o.residual(u).reshape(mesh.n_elem, o.ncu, o.npe)
    tot = r.sum(axis=(0, 2))
    assert np.all(np.abs(tot) <= 1e-13 * np.abs(r).sum())


def test_free_stream_euler():
    mesh = synth.quad_box(4, hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    o = oracle.Oracle(mesh, 3, oracle.EULER, oracle.CASE_CONST, (1.4,))
    assert np.abs(o.residual(o.interpolate())).max() < 1e-13


@pytest.mark.parametrize("periodic", [True, False])
def test_free_stream_navier_stokes(periodic):
    """A uniform state is an exact solution: R = 0, also against far-field boundaries."""
    mesh = synth.quad_box(4, hi=(10.0, 10.0), periodic=(periodic, periodic), affine=SHEAR2)
    o = oracle.Oracle(mesh, 3, oracle.NS, oracle.CASE_CONST, NS_MU)
    assert np.abs(o.residual(o.interpolate())).max() < 1e-13


def test_navier_stokes_inviscid_limit_is_euler():
    """With zero viscosity and zero penalty the NS residual is the Euler residual."""
    mesh = synth.quad_box(3, hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
    oe = oracle.Oracle(mesh, 2, oracle.EULER, oracle.CASE_VORTEX, (1.4,))
    on = oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_VORTEX, (1.4, 1e300, 0.72, 0.0))
    u = synth.random_euler_state(mesh.n_elem, oe.npe, 5)
    re, rn = oe.residual(u), on.residual(u)
    assert np.linalg.norm(rn - re) <= 1e-14 * np.linalg.norm(re)


def test_navier_stokes_viscous_terms_vanish_for_rigid_rotation():
    """A rigid rotation (zero strain rate) with variable density and uniform internal
    energy carries no viscous stress and no heat flux. Its state is cubic, so on Q3
    elements u_h and the LDG gradient are exact, and the NS residual must equal the
    Euler residual (viscous volume, face and penalty terms all zero). A missing
    transpose in the stress, or a heat flux built on grad E instead of grad e, would
    not vanish here; with a shear flow (the vortex) the two residuals do differ."""
    mesh = synth.quad_box(3, affine=SHEAR2)
    oe = oracle.Oracle(mesh, 3, oracle.EULER, oracle.CASE_ROTATION, (1.4,))
    on = oracle.Oracle(mesh, 3, oracle.NS, oracle.CASE_ROTATION, (1.4, 2.0, 0.72))
    u = on.interpolate()
    re, rn = oe.residual(u), on.residual(u)
    # the viscous terms cancel out of O(mu |grad v|) ~ 0.25 entries: rounding ~ 1e-12 relative
    assert np.linalg.norm(rn - re) <= 1e-10 * np.linalg.norm(re)
    oe2 = oracle.Oracle(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, (1.4,))
    on2 = oracle.Oracle(mesh, 3, oracle.NS, oracle.CASE_VORTEX, (1.4, 2.0, 0.72))
    u2 = on2.interpolate()
    assert np.linalg.norm(on2.residual(u2) - oe2.residual(u2)) > 1e-3 * np.linalg.norm(oe2.residual(u2))


def _quad_node_xy(o, mesh):
    """Physical positions [E][npe][2] of the nodes of parallelogram elements: the
    bilinear vertex map (vertices in lexicographic order) at the reference nodes."""
    s, t = o.ref_rules()[0][:, 0], o.ref_rules()[0][:, 1]
    N = np.stack([(1 - s) * (1 - t), (1 + s) * (1 - t), (1 - s) * (1 + t), (1 + s) * (1 + t)], 1) / 4
    return np.einsum("na,ead->end", N, mesh.xyz)


def _ns_viscous_sums(rho, m, rhoE, p=2, n=6, mu=(1.4, 5.0, 0.72)):
    """Per-element sums over test functions of R_NS - R_Euler, for a state given as
    nodal functions of position, on the elements of an n x n box that are at least two
    faces away from its boundary (their q and neighbour q see no boundary data)."""
    mesh = synth.quad_box(n)
    on = oracle.Oracle(mesh, p, oracle.NS, oracle.CASE_CONST, mu)
    oe = oracle.Oracle(mesh, p, oracle.EULER, oracle.CASE_CONST, mu[:1])
    X = _quad_node_xy(on, mesh)
    x, y = X[..., 0], X[..., 1]
    u = np.stack([rho(x, y), m(x, y)[0], m(x, y)[1], rhoE(x, y)], 1).ravel()
    d = (on.residual(u) - oe.residual(u)).reshape(mesh.n_elem, 4, on.npe).sum(-1)
    inner = [i + n * j for j in range(2, n - 2) for i in range(2, n - 2)]
    return d[inner], 1.0 / n ** 2


def test_navier_stokes_viscous_stress_closed_form():
    """Section 2.1's viscous flux pinned by a closed form. Constant density and internal
    energy with the uniform dilatation v = a (x, y): the Stokes stress is the constant
    (2/3) mu a I (bulk coefficient -2/3: 2a - (2/3)(2a)), so the momentum sums vanish and
    the energy flux v . tau = (2/3) mu a^2 (x, y) has divergence (4/3) mu a^2. The state is
    quadratic, exact in Q2, and continuous, so the LDG q is -grad u exactly and every face
    jump is zero: summed over the test functions, R_NS - R_Euler on an element K is
    -int_dK Fv . n = -(4/3) mu a^2 |K| in the energy and 0 elsewhere. A bulk coefficient of
    -1/3 gives -(8/3) mu a^2 |K|."""
    r0, a, e0, mu = 1.3, 0.4, 2.0, 1.0 / 5.0
    d, area = _ns_viscous_sums(lambda x, y: r0 + 0 * x, lambda x, y: (r0 * a * x, r0 * a * y),
                               lambda x, y: r0 * (e0 + 0.5 * a * a * (x * x + y * y)))
    want = np.array([0.0, 0.0, 0.0, -(4.0 / 3.0) * mu * a * a * area])
    assert np.abs(d - want).max() <= 1e-12, (d, want)


def test_navier_stokes_heat_flux_closed_form():
    """The Fourier heat flux (mu gamma / Pr) grad e pinned by a closed form: gas at rest
    with constant density and internal energy e = b x^2 has no stress and the energy flux
    (mu gamma / Pr)(2 b x, 0), so summed over the test functions R_NS - R_Euler on an
    element K is -(mu gamma / Pr) 2 b |K| in the energy and 0 elsewhere. A heat flux
    without gamma, or on grad E, fails it."""
    r0, b, mu, gam, pr = 1.3, 0.7, 1.0 / 5.0, 1.4, 0.72
    d, area = _ns_viscous_sums(lambda x, y: r0 + 0 * x, lambda x, y: (0 * x, 0 * x),
                               lambda x, y: r0 * b * x * x)
    want = np.array([0.0, 0.0, 0.0, -(mu * gam / pr) * 2.0 * b * area])
    assert np.abs(d - want).max() <= 1e-12, (d, want)


def test_poisson_jacobian_symmetric_positive_definite():
    o = oracle.Oracle(synth.tri_square(2, affine=SHEAR2), 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
    J = o.jacobian_cs(np.zeros(o.ndof))
    assert np.linalg.norm(J - J.T) <= 1e-13 * np.linalg.norm(J)
    assert np.linalg.eigvalsh(0.5 * (J + J.T)).min() > 0


@pytest.mark.parametrize("mesh_kind,p,model,case", [
    ("tri", 2, oracle.POISSON, oracle.CASE_POLY2), ("tri", 3, oracle.CONVDIFF, oracle.CASE_POLY2),
    ("tri", 5, oracle.POISSON, oracle.CASE_POLY2), ("tet", 2, oracle.CONVDIFF, oracle.CASE_POLY2),
    ("tet", 3, oracle.POISSON, oracle.CASE_POLY2)])
def test_patch_test_unstructured_simplices(mesh_kind, p, model, case):
    """The patch test on unstructured simplex meshes: random diagonals (vertex degrees 3
    to 8), jittered vertices, rotated local vertex numbering and shuffled elements; a
    polynomial of degree <= p still has zero residual, so faces are paired and oriented
    correctly under every local numbering."""
    mesh = synth.tri_unstructured(5, seed=11) if mesh_kind == "tri" else synth.tet_unstructured(2, seed=5)
    mu = (0.7, 1.3) if model == oracle.POISSON else ((0.05, 0.4, 1.0, -0.6) if mesh_kind == "tri"
                                                    else (0.05, 0.4, 1.0, -0.6, 0.3))
    o = oracle.Oracle(mesh, p, model, case, mu)
    u = o.interpolate()
    r = o.residual(u)
    assert np.abs(r).max() < 1e-12 * max(1.0, np.abs(o.residual(np.zeros_like(u))).max())


def test_poisson_jacobian_spd_on_unstructured_triangles():
    """The LDG Poisson operator (central traces with a jump penalty) is symmetric positive
    definite; so it stays on a random-diagonal, jittered mesh."""
    o = oracle.Oracle(synth.tri_unstructured(3, seed=2), 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
    J = o.jacobian_cs(np.zeros(o.ndof))
    assert np.linalg.norm(J - J.T) <= 1e-13 * np.linalg.norm(J)
    assert np.linalg.eigvalsh(0.5 * (J + J.T)).min() > 0


def test_upwind_dissipation():
    """Pure convection with the upwind flux on a periodic mesh: u^T R(u) =
    1/2 sum_faces int |beta.n| [u]^2 > 0; a constant state gives zero."""
    mesh = synth.quad_box(3, periodic=(True, True))
    o = oracle.Oracle(mesh, 2, oracle.CONVDIFF, oracle.CASE_ZERO, (0.0, 0.0, 1.0, 0.5))
    u = synth.random_vector(o.ndof, 5)
    assert u @ o.residual(u) > 0
    assert abs(np.ones(o.ndof) @ o.residual(np.ones(o.ndof))) < 1e-13


def test_euler_riemann_jump_closed_form():
    """Piecewise-constant Euler states U_L (x < 5) and U_R (x > 5) on the periodic
    square: element residual sums reduce to the Rusanov flux jump on the interface,
    sum_i R_{K,i} = |face| [ (F(U_R) - F(U_L)).n / 2 + lambda/2 (U_L - U_R) ],
    lambda = max(|v_L.n| + c_L, |v_R.n| + c_R) (local Lax-Friedrichs)."""
    g = 1.4

    def prim2cons(r, vx, vy, p):
        return np.array([r, r * vx, r * vy, p / (g - 1) + 0.5 * r * (vx * vx + vy * vy)])

    def fx(U):
        r, vx, vy = U[0], U[1] / U[0], U[2] / U[0]
        p = (g - 1) * (U[3] - 0.5 * r * (vx * vx + vy * vy))
        return np.array([r * vx, r * vx * vx + p, r * vx * vy, (U[3] + p) * vx]), abs(vx) + math.sqrt(g * p / r)
    UL, UR = prim2cons(1.0, 0.3, -0.2, 1.0), prim2cons(0.6, -0.1, 0.4, 0.7)
    n = 6
    mesh = synth.quad_box(n, hi=(10.0, 10.0), periodic=(True, True))
    o = oracle.Oracle(mesh, 2, oracle.EULER, oracle.CASE_CONST, (g,))
    u = np.empty((mesh.n_elem, 4, o.npe))
    for e in range(mesh.n_elem):
        u[e] = (UL if (e % n) < n // 2 else UR)[:, None]
    r = o.residual(u.ravel()).reshape(mesh.n_elem, 4, o.npe).sum(axis=2)
    FL, sL = fx(UL)
    FR, sR = fx(UR)
    lam = max(sL, sR)
    h = 10.0 / n
    # element just left of x = 5 (normal +x): interface flux minus its own flux
    exp_left = h * (0.5 * (FR - FL) + 0.5 * lam * (UL - UR))
    # element just right of x = 0 seen from the seam at x = 0/10 (normal -x, neighbour U_R)
    exp_seam = h * (-0.5 * (FR - FL) + 0.5 * lam * (UL - UR))
    assert np.allclose(r[n // 2 - 1], exp_left, atol=1e-13)
    assert np.allclose(r[0], exp_seam, atol=1e-13)
    assert np.allclose(r[1], 0, atol=1e-13)          # no jump on any of its faces


# ------------------------------------------------------------------- J.v pins
@pytest.mark.parametrize("etype,model", [(0, oracle.POISSON), (2, oracle.CONVDIFF), (1, oracle.EULER),
                                         (1, oracle.NS), (3, oracle.CONVDIFF)])
def test_jvp_matches_complex_step_jacobian(etype, model):
    if model in (oracle.EULER, oracle.NS):
        mesh = synth.quad_box(3, hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2)
        o = oracle.Oracle(mesh, 2, model, oracle.CASE_VORTEX, (1.4,) if model == oracle.EULER else NS_MU)
        u = synth.random_euler_state(mesh.n_elem, o.npe, 11)
    else:
        mesh = _mesh(etype, 2, affine=SHEAR3 if etype >= 2 else SHEAR2)
        o = oracle.Oracle(mesh, 1 if etype == 2 else 2, model, oracle.CASE_SINSIN,
                          (1.0, 1.0) if model == oracle.POISSON else (0.1, 0.3, 1.0, 0.5, 0.25))
        u = synth.random_vector(o.ndof, 11)
    J = o.jacobian_cs(u)
    v = synth.random_vector(o.ndof, 12)
    jv = o.jvp(u, v)
    assert np.linalg.norm(jv - J @ v) <= 1e-13 * np.linalg.norm(jv)
    # finite differences agree to O(eps)
    eps = 1e-7
    fd = (o.residual(u + eps * v) - o.residual(u - eps * v)) / (2 * eps)
    assert np.linalg.norm(fd - jv) <= 1e-6 * np.linalg.norm(jv)


@pytest.mark.parametrize("etype", [0, 1, 2])
def test_linear_jvp_is_residual_difference(etype):
    o = oracle.Oracle(_mesh(etype, 2), 2, oracle.CONVDIFF, oracle.CASE_EXPSIN, (0.05, 0.2, 1.0, 0.5, 0.25))
    u, v = synth.random_vector(o.ndof, 1), synth.random_vector(o.ndof, 2)
    jv = o.jvp(u, v)
    ref = o.residual(v) - o.residual(np.zeros(o.ndof))
    assert np.linalg.norm(jv - ref) <= 1e-12 * np.linalg.norm(jv)


def test_sampled_residual_matches_full():
    o = oracle.Oracle(synth.hex_box(3), 2, oracle.CONVDIFF, oracle.CASE_EXPSIN, (0.01, 0.01, 1.0, 0.5, 0.25))
    u, v = synth.random_vector(o.ndof, 3), synth.random_vector(o.ndof, 4)
    el = np.array([0, 13, 26, 5])
    full = o.residual(u).reshape(27, 1, -1)
    assert np.array_equal(o.residual_some(u, el), full[el])
    fullj = o.jvp(u, v).reshape(27, 1, -1)
    assert np.array_equal(o.jvp_some(u, v, el), fullj[el])


# ------------------------------------------------------------ solver pins
def test_gmres_matches_dense_solve():
    mesh = synth.quad_box(3, hi=(10.0, 10.0), periodic=(True, True))
    o = oracle.Oracle(mesh, 2, oracle.EULER, oracle.CASE_VORTEX, (1.4,))
    u = o.project(0.0)
    un = u.copy()
    o.set_time(1, 0.0, 0.5, un, un)
    J = o.jacobian_cs(u)
    b = synth.random_vector(o.ndof, 9)
    x, its, rc, hist = o.gmres(u, b, m=20, rtol=1e-12, maxit=2000)
    assert rc == 0
    xd = np.linalg.solve(J, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.all(np.diff(hist[: min(len(hist), 20)]) <= 1e-12 * hist[0])   # monotone within a cycle


def test_newton_linear_one_step():
    o = oracle.Oracle(synth.tri_square(4), 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
    u, rc, st = o.newton(np.zeros(o.ndof), m=200, newton_rtol=1e-9, gmres_rtol=1e-11, max_newton=3)
    assert rc == 0 and st["newton_iters"] == 1
    assert st["rfinal"] <= 1e-9 * st["r0"]


# ---------------------------------------------------------- convergence rates
def _solve_linear(o):
    u0 = np.zeros(o.ndof)
    x, its, rc, _ = o.gmres(u0, o.residual(u0), m=300, rtol=1e-10, maxit=4000)
    assert rc == 0
    return -x


@pytest.mark.parametrize("p,ns,q_tol", [(4, (4, 8), 0.3), (5, (2, 4), 0.3), (6, (2, 4), 1.0)])
def test_high_order_triangle_rates(p, ns, q_tol):
    """Triangles at p = 4..6 converge at p + 1 in u and p in q (Section 4.1's rates).
    At p = 6 the q rate of the coarse pair 2 -> 4 is still pre-asymptotic (5.35), so it
    is only held above p - 1."""
    errs = []
    for n in ns:
        o = oracle.Oracle(synth.tri_square(n), p, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
        errs.append(o.l2_error(_solve_linear(o)))
    e = np.array(errs)
    ru = np.log2(e[-2, 0] / e[-1, 0])
    rq = np.log2(e[-2, 1] / e[-1, 1])
    assert abs(ru - (p + 1)) < 0.3, ru
    assert abs(rq - p) < q_tol, rq


@pytest.mark.parametrize("p,ns", [(1, (4, 8, 16)), (2, (4, 8, 16)), (3, (4, 8))])
def test_simplex_convergence_rates_match_section_4_1(p, ns):
    """On simplices the method converges at p+1 in u and p in q, as Section 4.1 and
    Table 3 report for tetrahedra."""
    gold = json.load(open(os.path.join(GOLD, "table3_rates.json")))
    errs = []
    for n in ns:
        o = oracle.Oracle(synth.tri_square(n), p, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
        errs.append(o.l2_error(_solve_linear(o)))
    e = np.array(errs)
    ru = np.log2(e[-2, 0] / e[-1, 0])
    rq = np.log2(e[-2, 1] / e[-1, 1])
    assert abs(ru - (p + 1)) < 0.3 and abs(rq - p) < 0.3, (ru, rq)
    assert abs(ru - gold["u_rate_finest"][str(p)]) < 0.3
    assert abs(rq - gold["q_rate_finest"][str(p)]) < 0.3


@pytest.mark.parametrize("etype,p,ns", [(1, 1, (4, 8, 16)), (1, 2, (4, 8, 16)), (1, 3, (8, 16)), (2, 1, (2, 4, 8))])
def test_tensor_convergence_rates(etype, p, ns):
    """Uniform tensor meshes with central traces and an O(1) penalty: the LDG error
    estimates for that penalty scaling give u at order p and q at order p - 1/2; odd p
    shows rates close to those (even p is optimal, with q superconvergent)."""
    errs = []
    for n in ns:
        o = oracle.Oracle(_mesh(etype, n), p, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
        errs.append(o.l2_error(_solve_linear(o)))
    e = np.array(errs)
    ru = np.log2(e[-2, 0] / e[-1, 0])
    rq = np.log2(e[-2, 1] / e[-1, 1])
    assert ru > p and rq > p - 0.6, (ru, rq)


def test_euler_vortex_consistency_rate():
    """Truncation error of the spatial operator on the travelling vortex,
    R(P u(t)) + M d/dt P u(t) -> 0 at order >= p in h."""
    errs = []
    p = 2
    for n in (8, 16):
        mesh = synth.quad_box(n, hi=(10.0, 10.0), periodic=(True, True))
        o = oracle.Oracle(mesh, p, oracle.EULER, oracle.CASE_VORTEX, (1.4,))
        d = 1e-4
        dudt = (o.project(d) - o.project(-d)) / (2 * d)
        res = o.residual(o.project(0.0)) + o.mass(dudt)
        errs.append(np.linalg.norm(res) / np.linalg.norm(o.mass(dudt)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > p - 0.3, (errs, rate)


# ------------------------------------------------------------- MLP oracle
def test_mlp_backprop_matches_central_differences():
    """The chain-rule gradient of the MLP loss equals central finite differences."""
    from oracle import mlp
    rng = np.random.default_rng(0)
    n_in, h, n_out = 6, 5, 6
    nparam = sum(int(np.prod(s)) for s in mlp.shapes(n_in, h, n_out))
    theta = rng.standard_normal(nparam) * 0.5
    X = rng.standard_normal((9, n_in))
    X[3] = 0.0                                    # a masked (zero-norm) pair
    T = rng.standard_normal((9, n_out))
    for U in (None, rng.standard_normal((9, 3))):
        nin = n_in + (0 if U is None else 3)
        nparam = sum(int(np.prod(s)) for s in mlp.shapes(nin, h, n_out))
        theta = rng.standard_normal(nparam) * 0.5
        loss, g = mlp.loss_grad(theta, X, T, nin, h, n_out, U=U)
        eps = 1e-6
        fd = np.empty_like(theta)
        for i in range(nparam):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += eps
            tm[i] -= eps
            fd[i] = (mlp.loss_grad(tp, X, T, nin, h, n_out, U=U)[0] -
                     mlp.loss_grad(tm, X, T, nin, h, n_out, U=U)[0]) / (2 * eps)
        assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(g)


def test_mlp_apply_is_positively_homogeneous():
    from oracle import mlp
    rng = np.random.default_rng(1)
    n_in, h = 8, 7
    theta = rng.standard_normal(sum(int(np.prod(s)) for s in mlp.shapes(n_in, h, n_in)))
    V = rng.standard_normal((5, n_in))
    a = mlp.apply(theta, V, n_in, h, n_in)
    assert np.allclose(mlp.apply(theta, 3.7 * V, n_in, h, n_in), 3.7 * a, rtol=1e-12, atol=1e-12)
    assert np.allclose(mlp.apply(theta, 0 * V, n_in, h, n_in), 0.0)


def test_adam_reduces_a_quadratic():
    from oracle import mlp
    theta = np.array([3.0, -2.0])
    m, v = np.zeros(2), np.zeros(2)
    for t in range(1, 2001):
        mlp.adam_step(theta, 2 * theta, m, v, t, lr=0.05)
    assert np.abs(theta).max() < 1e-2


def test_adam_first_step_and_constant_gradient():
    """Adam (Kingma & Ba 2015) from zero moments: the bias corrections make the first
    step exactly lr g / (|g| + eps) for any g, and under a constant gradient every
    later step is the same (m_hat = g and v_hat = g^2 at every t). A missing bias
    correction scales the first step by (1 - b1) / sqrt(1 - b2) ~ 3.2."""
    from oracle import mlp
    rng = np.random.default_rng(7)
    g = rng.standard_normal(16) * np.exp(rng.uniform(-6, 6, 16))
    theta = rng.standard_normal(16)
    m, v = np.zeros(16), np.zeros(16)
    lr, eps = 0.01, 1e-8
    prev = theta.copy()
    for t in range(1, 6):
        mlp.adam_step(theta, g, m, v, t, lr=lr)
        step = theta - prev
        assert np.allclose(step, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0), t
        prev = theta.copy()


def test_adam_second_step_closed_forms():
    """Two Adam steps from zero moments in closed form, with the published defaults
    b1 = 0.9, b2 = 0.999 (eps negligible for |g| ~ 1):
    gradients (g, -g): m_hat_2 = -g (1 - b1)/(1 + b1), v_hat_2 = g^2, so the second step
    is +lr (1 - b1)/(1 + b1) sign(g) = lr / 19;
    gradients (g, 2g): m_hat_2 = g (b1 + 2)/(1 + b1), v_hat_2 = g^2 (b2 + 4)/(1 + b2), so
    the second step is -lr (2.9 / 1.9) / sqrt(4.999 / 1.999) sign(g). A wrong b1 fails the
    first, a wrong b2 the second."""
    from oracle import mlp
    lr = 0.01
    for g2f, want in ((-1.0, lr / 19.0), (2.0, -lr * (2.9 / 1.9) / math.sqrt(4.999 / 1.999))):
        g = np.array([1.0, -1.0])
        theta, m, v = np.zeros(2), np.zeros(2), np.zeros(2)
        mlp.adam_step(theta, g, m, v, 1, lr=lr)
        t1 = theta.copy()
        mlp.adam_step(theta, g2f * g, m, v, 2, lr=lr)
        assert np.allclose(theta - t1, want * np.sign(g), rtol=1e-7, atol=0), (g2f, theta - t1)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    """The oracle's BF16 rounding (storage precision of the tensor-core inference
    path) against torch's float32 -> bfloat16 conversion, plus the tie cases."""
    import torch
    from oracle import mlp as omlp
    x = np.random.default_rng(3).standard_normal(10000) * np.exp(np.random.default_rng(4).uniform(-20, 20, 10000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(omlp.round_bf16(x), ref)
    ulp = 2.0 ** -7
    assert omlp.round_bf16(1.0 + ulp / 2) == 1.0                  # tie -> even (1.0)
    assert omlp.round_bf16(1.0 + 3 * ulp / 2) == 1.0 + 2 * ulp    # tie -> even (1 + 2 ulp)
    assert omlp.round_bf16(1.0 + 0.6 * ulp) == 1.0 + ulp


# ------------------------------------------------------- curved quadrilaterals
def _as_curved(mesh, pg):
    """The same affine mesh described by degree-pg map points (equispaced, a fastest)."""
    t = np.linspace(-1.0, 1.0, pg + 1)
    a, b = np.tile(t, pg + 1), np.repeat(t, pg + 1)
    w = np.stack([(1 - a) * (1 - b), (1 + a) * (1 - b), (1 - a) * (1 + b), (1 + a) * (1 + b)], 1) / 4
    return synth.Mesh(mesh.etype, mesh.xyz, mesh.vid, mesh.name, pg=pg, xgeo=np.einsum("pv,evd->epd", w, mesh.xyz))


@pytest.mark.parametrize("model,pg", [(oracle.CONVDIFF, 1), (oracle.NS, 3)])
def test_curved_path_on_affine_elements_equals_affine_path(model, pg):
    """Map points placed by the affine map: per-point Jacobians, normals and the
    Newton inverse map give the affine path's residual."""
    mesh = synth.quad_box((4, 3), hi=(10.0, 10.0), periodic=(True, False), affine=SHEAR2)
    mu = (0.1, 0.2, 1.0, 0.5) if model == oracle.CONVDIFF else NS_MU
    case = oracle.CASE_SINSIN if model == oracle.CONVDIFF else oracle.CASE_VORTEX
    oa = oracle.Oracle(mesh, 2, model, case, mu)
    oc = oracle.Oracle(_as_curved(mesh, pg), 2, model, case, mu)
    u = (synth.random_euler_state(mesh.n_elem, oa.npe, 4) if model == oracle.NS
         else synth.random_vector(oa.ndof, 4))
    ra = oa.residual(u)
    assert np.linalg.norm(oc.residual(u) - ra) <= 1e-13 * np.linalg.norm(ra)


@pytest.mark.parametrize("pg", [1, 2, 3])
def test_curved_mass_integrates_the_area(pg):
    """sum_ij M_ij = integral of det J: the warped elements tile the box exactly (the
    displacement vanishes on its boundary and shared edges conform), so the total is
    the box area; per element it is positive."""
    mesh = synth.warped_box((5, 4), pg, hi=(3.0, 2.0), amp=0.15)
    o = oracle.Oracle(mesh, 3, oracle.POISSON, oracle.CASE_ZERO)
    m = o.mass(np.ones(o.ndof)).reshape(mesh.n_elem, o.npe)
    assert abs(m.sum() - 6.0) < 1e-12
    assert (m.sum(1) > 0).all()


@pytest.mark.parametrize("model", [oracle.EULER, oracle.NS])
@pytest.mark.parametrize("which", ["warped_periodic", "warped_farfield", "ogrid_farfield"])
def test_curved_free_stream(model, which):
    """A uniform state is preserved on curved isoparametric quadrilaterals: in 2-D the
    metric terms det J J^-1 have the map's degree, so the chosen quadrature integrates
    the discrete divergence theorem exactly."""
    if which == "ogrid_farfield":
        mesh = synth.o_grid(3, 12, 3, outer=("circle", 2.0), jitter=0.3, wall=False)
    else:
        mesh = synth.warped_box(4, 3, hi=(10.0, 10.0), periodic=(which == "warped_periodic",) * 2, amp=0.2)
    mu = (1.4,) if model == oracle.EULER else NS_MU
    o = oracle.Oracle(mesh, 3, model, oracle.CASE_CONST, mu)
    u = o.interpolate()
    assert np.abs(o.residual(u)).max() < 1e-12


def test_curved_conservation_periodic():
    mesh = synth.warped_box(3, 2, hi=(2.0, 2.0), periodic=(True, True), amp=0.2)
    for model, mu, case in ((oracle.CONVDIFF, (0.1, 0.2, 1.0, 0.5), oracle.CASE_ZERO),
                            (oracle.NS, NS_MU, oracle.CASE_CONST)):
        o = oracle.Oracle(mesh, 2, model, case, mu)
        u = (synth.random_euler_state(mesh.n_elem, o.npe, 3) if model == oracle.NS
             else synth.random_vector(o.ndof, 3))
        r = o.residual(u).reshape(mesh.n_elem, o.ncu, o.npe)
        assert np.all(np.abs(r.sum(axis=(0, 2))) <= 1e-13 * np.abs(r).sum())


@pytest.mark.parametrize("model", [oracle.EULER, oracle.NS])
def test_wall_gas_at_rest(model):
    """Gas at rest between two circular walls is an exact steady solution: the wall
    flux carries only the pressure, and the viscous and penalty terms vanish."""
    mesh = synth.o_grid(3, 12, 3, outer=("circle", 2.0), jitter=0.3, outer_wall=True)
    o = oracle.Oracle(mesh, 3, model, oracle.CASE_REST, (1.4,) if model == oracle.EULER else NS_MU)
    assert np.abs(o.residual(o.interpolate())).max() < 1e-12


def test_walls_conserve_mass_and_energy():
    """With walls all round, no mass or energy crosses the boundary: the density and
    energy residuals sum to zero for any state (momentum feels the wall pressure)."""
    mesh = synth.o_grid(3, 12, 2, outer=("circle", 2.0), jitter=0.3, outer_wall=True)
    o = oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_REST, NS_MU)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 8)
    r = o.residual(u).reshape(mesh.n_elem, 4, o.npe)
    tot = r.sum(axis=(0, 2))
    scale = np.abs(r).sum(axis=(0, 2))
    assert abs(tot[0]) <= 1e-13 * scale[0] and abs(tot[3]) <= 1e-13 * scale[3]
    assert abs(tot[1]) > 1e-6 * scale[1]


def test_curved_wall_jvp_matches_complex_step():
    """J.v through curved geometry, the wall trace and the wall flux."""
    mesh = synth.o_grid(2, 8, 3, outer=("circle", 2.0), jitter=0.3)
    o = oracle.Oracle(mesh, 2, oracle.NS, oracle.CASE_CYLINDER, NS_MU)
    u = synth.random_euler_state(mesh.n_elem, o.npe, 12)
    u = u.reshape(mesh.n_elem, 4, o.npe)
    u[:, 3] += 15.0                                 # pressure of the Mach 0.2 free stream
    u = u.ravel()
    v = synth.random_vector(o.ndof, 13)
    J = o.jacobian_cs(u)
    jv = o.jvp(u, v)
    assert np.linalg.norm(jv - J @ v) <= 1e-13 * np.linalg.norm(J @ v)


def test_curved_annulus_convergence():
    """Poisson on the annulus 0.5 < r < 1 with curved maps of degree p = 2: u converges
    at order p + 1 (even p; a wrong metric term would stall it)."""
    errs = []
    for n in (4, 8, 16):
        mesh = synth.o_grid(n, 4 * n, 2, outer=("circle", 1.0), wall=False)
        o = oracle.Oracle(mesh, 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
        errs.append(o.l2_error(_solve_linear(o)))
    e = np.array(errs)
    assert np.log2(e[-2, 0] / e[-1, 0]) > 2.7, e


def test_curved_annulus_area():
    """sum_ij M_ij on the annulus 0.5 < r < 2: straight-sided maps give exactly the area
    between the two inscribed regular polygons, (n/2) sin(2 pi / n) (R^2 - r0^2); cubic
    maps approach pi (R^2 - r0^2) at order >= 4 in the angular spacing."""
    def area(pg, n):
        mesh = synth.o_grid(2, n, pg, outer=("circle", 2.0), wall=False)
        o = oracle.Oracle(mesh, 3, oracle.POISSON, oracle.CASE_ZERO)
        return o.mass(np.ones(o.ndof)).sum()
    for n in (8, 12):
        assert abs(area(1, n) - n / 2 * np.sin(2 * np.pi / n) * 3.75) < 1e-12
    exact = np.pi * 3.75
    e1, e2 = abs(area(3, 8) - exact), abs(area(3, 16) - exact)
    assert e2 < e1 and np.log2(e1 / e2) > 3.8, (e1, e2)


# ------------------------------------------------------------------- DIRK time stepping
def test_dirk_tableaus_meet_their_order_conditions():
    """Butcher order conditions: row sums c_i = sum_j a_ij; order 1 (sum b = 1), 2
    (b.c = 1/2), 3 (b.c^2 = 1/3, b.A c = 1/6), 4 (b.c^3 = 1/4, b.(c A c) = 1/8,
    b.A c^2 = 1/12, b.A A c = 1/24), to each scheme's order; DIRK22/33 are stiffly
    accurate (b = last row of A)."""
    conds = [lambda A, b, c: b.sum() - 1,
             lambda A, b, c: b @ c - 1 / 2,
             lambda A, b, c: b @ c ** 2 - 1 / 3, lambda A, b, c: b @ A @ c - 1 / 6,
             lambda A, b, c: b @ c ** 3 - 1 / 4, lambda A, b, c: b @ (c * (A @ c)) - 1 / 8,
             lambda A, b, c: b @ A @ c ** 2 - 1 / 12, lambda A, b, c: b @ A @ A @ c - 1 / 24]
    n_conds = {1: 1, 2: 2, 3: 4, 4: 8}
    for sch, order in ((oracle.DIRK11, 1), (oracle.DIRK22, 2), (oracle.DIRK33, 3), (oracle.DIRK34, 4)):
        A, b, c = (np.array(x) for x in oracle.dirk_tableau(sch))
        assert np.allclose(A.sum(1), c, atol=1e-15)
        assert np.allclose(np.triu(A, 1), 0) and len(set(np.diag(A))) == 1    # singly diagonally implicit
        for k in range(n_conds[order]):
            assert abs(conds[k](A, b, c)) < 1e-14, (sch, k)
        if sch in (oracle.DIRK22, oracle.DIRK33):
            assert np.allclose(A[-1], b, atol=1e-15)


def test_dirk_temporal_order_against_matrix_exponential():
    """On a linear semi-discrete problem M u' = -(A u + r0) (convection-diffusion on a
    periodic mesh), DIRK steps converge to the exact solution
    u* + expm(-t M^-1 A)(u0 - u*) at the scheme's order."""
    import scipy.linalg as sl
    mesh = synth.quad_box(3, hi=(2.0, 2.0), periodic=(True, True))
    o = oracle.Oracle(mesh, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, (0.02, 0.3, 1.0, 0.5))
    n = o.ndof
    A = o.jacobian_cs(np.zeros(n))
    r0 = o.residual(np.zeros(n))
    M = np.stack([o.mass(e) for e in np.eye(n)], 1)
    ustar = -np.linalg.solve(A, r0)
    u0 = o.interpolate()
    T = 0.25
    yT = ustar + sl.expm(-T * np.linalg.solve(M, A)) @ (u0 - ustar)
    for sch, order in ((oracle.DIRK11, 1), (oracle.DIRK22, 2), (oracle.DIRK33, 3), (oracle.DIRK34, 4)):
        errs = []
        for N in (16, 32):
            u, t, dt = u0.copy(), 0.0, T / N
            for _ in range(N):
                u, _ = o.dirk_step(u, t, dt, sch, newton_rtol=1e-12, gmres_rtol=1e-12, m=30, max_gmres=5000)
                t += dt
            errs.append(np.linalg.norm(u - yT) / np.linalg.norm(yT))
        rate = np.log2(errs[0] / errs[1])
        assert rate > order - 0.3, (sch, errs, rate)


def test_bdf2_temporal_order_against_matrix_exponential():
    """BDF2 time term M (3 u^{n+1} - 4 u^n + u^{n-1}) / (2 dt) of the workloads' implicit
    steps, pinned by its temporal order: on the linear semi-discrete problem
    M u' = -(A u + r0) (convection-diffusion on a periodic mesh), started from the exact
    solution at t = 0 and t = dt, the error at T against u* + expm(-t M^-1 A)(u0 - u*)
    falls at order 2 over three halvings of dt. A wrong coefficient of u^{n-1} makes
    the scheme inconsistent; a missing 1/2 solves a different ODE."""
    import scipy.linalg as sl
    mesh = synth.quad_box(3, hi=(2.0, 2.0), periodic=(True, True))
    o = oracle.Oracle(mesh, 2, oracle.CONVDIFF, oracle.CASE_SINSIN, (0.02, 0.3, 1.0, 0.5))
    n = o.ndof
    A = o.jacobian_cs(np.zeros(n))
    r0 = o.residual(np.zeros(n))
    M = np.stack([o.mass(e) for e in np.eye(n)], 1)
    ustar = -np.linalg.solve(A, r0)
    u0 = o.interpolate()
    L = np.linalg.solve(M, A)
    exact = lambda t: ustar + sl.expm(-t * L) @ (u0 - ustar)
    T = 0.5
    errs = []
    for N in (16, 32, 64, 128):
        dt = T / N
        unm1, un = u0.copy(), exact(dt)
        for k in range(1, N):
            o.set_time(2, (k + 1) * dt, dt, un, unm1)
            u, rc, _ = o.newton(un, newton_rtol=1e-10, gmres_rtol=1e-12, m=30, max_gmres=5000)
            assert rc == 0
            unm1, un = un, u
        errs.append(np.linalg.norm(un - exact(T)) / np.linalg.norm(exact(T)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.2), (errs, rates)


@pytest.mark.parametrize("p", [1, 2])
def test_tetrahedral_rates_match_table3(p):
    """Section 4.1 / Table 3: Poisson with u = sin(pi x) sin(pi y) sin(pi z) on structured
    tetrahedral meshes of the unit cube. Between the table's first two refinements
    (1/n = 2, 4) the rates of u_h and q_h agree with the table's within 0.3 (the traces
    and penalty of the paper are not given, so the error values themselves differ), and
    they already exceed p + 1/2 and p - 1/3."""
    gold = json.load(open(os.path.join(GOLD, "table3_rates.json")))
    errs = []
    for n in (2, 4):
        o = oracle.Oracle(synth.tet_cube(n), p, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
        errs.append(o.l2_error(_solve_linear(o)))
    e = np.array(errs)
    ru, rq = np.log2(e[0, 0] / e[1, 0]), np.log2(e[0, 1] / e[1, 1])
    assert abs(ru - gold["u_rate_n2_to_n4"][str(p)]) < 0.3, ru
    assert abs(rq - gold["q_rate_n2_to_n4"][str(p)]) < 0.3, rq
    assert ru > p + 0.5 and rq > p - 1 / 3, (ru, rq)



# ---------------------------------------------------------------- wave model (Section 2.1)
def _wave(mesh, p, c2, tau):
    from oracle import wave
    o = oracle.Oracle(mesh, p, oracle.POISSON, oracle.CASE_ZERO, (c2, tau))
    L, M = wave.wave_operator(o)
    return o, L, M


def _energy_matrix(o, M, c2):
    """blockdiag(M, c^2 M per q component) in the [E][dim][n_pe] layout of q."""
    import scipy.linalg as sla
    n, nd = o.ndof, o.nd
    idx = np.arange(n * nd).reshape(o.mesh.n_elem, nd, o.npe)
    Mq = np.zeros((n * nd, n * nd))
    for d in range(nd):
        sel = idx[:, d, :].ravel()
        Mq[np.ix_(sel, sel)] = M
    return sla.block_diag(M, c2 * Mq)


@pytest.mark.parametrize("kind", ["quad_periodic", "quad_dirichlet", "tri_periodic", "hex_periodic"])
def test_wave_operator_conserves_energy_without_penalty_and_dissipates_with_it(kind):
    """E(u, q) = u.M u + c^2 q.M q is the wave's energy; d/dt E = 2 y.E L y. With central
    traces and tau = 0 the LDG q-equation and the q-term of Eq. 1b are adjoint, so E L is
    skew; with tau > 0 its symmetric part is negative semidefinite and not zero. A flipped
    sign or a transposed coupling in either map, or a missing c^2, breaks the first."""
    mesh = {"quad_periodic": lambda: synth.quad_box(3, periodic=(True, True), affine=np.array([[1.0, 0.3], [0.1, 0.9]])),
            "quad_dirichlet": lambda: synth.quad_box(3),
            "tri_periodic": lambda: synth.tri_square(3, periodic=(True, True)),
            "hex_periodic": lambda: synth.hex_box(3, periodic=(True, True, True))}[kind]()
    p = 1 if mesh.nd == 3 else 2
    c2 = 0.7
    o, L, M = _wave(mesh, p, c2, 0.0)
    S = _energy_matrix(o, M, c2) @ L
    assert np.linalg.norm(S + S.T) <= 1e-13 * np.linalg.norm(S), kind
    o, L, M = _wave(mesh, p, c2, 1.0)
    S = _energy_matrix(o, M, c2) @ L
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev.max() <= 1e-13 * np.linalg.norm(S) and ev.min() < -1e-3 * np.linalg.norm(S), kind


def _standing_wave(o, c):
    from oracle import wave
    X = wave.quad_node_coords(o)
    sx = (np.sin(2 * np.pi * X[..., 0]) * np.sin(2 * np.pi * X[..., 1])).ravel()
    return sx, c * 2 * np.pi * np.sqrt(2.0)


@pytest.mark.parametrize("scheme,order", [(1, 1), (2, 2), (3, 3), (4, 4)])
def test_wave_dirk_temporal_order_against_the_matrix_exponential(scheme, order):
    """The DIRK step of the coupled (u, q) system against exp(T L) y0 for a smooth start
    (a standing-wave displacement): the observed order of each scheme."""
    import scipy.linalg as sla
    from oracle import wave
    o, L, M = _wave(synth.quad_box(4, periodic=(True, True)), 3, 1.0, 0.5)
    n = o.ndof
    sx, _ = _standing_wave(o, 1.0)
    y0 = np.concatenate([np.zeros(n), o.q(sx)])
    T = 0.2
    ex = sla.expm(T * L) @ y0
    errs = []
    for N in (16, 32, 64):
        u, q = y0[:n].copy(), y0[n:].copy()
        for _ in range(N):
            u, q, _ = wave.wave_step(L, n, u, q, None, T / N, scheme)
        errs.append(np.linalg.norm(np.concatenate([u, q]) - ex) / np.linalg.norm(ex))
    rate = math.log2(errs[1] / errs[2])
    assert order - 0.3 < rate < order + 0.3, (scheme, errs)


@pytest.mark.parametrize("p,lo,hi", [(1, 1.5, 2.6), (2, 2.5, 4.2)])
def test_wave_displacement_converges_to_the_standing_wave(p, lo, hi):
    """w = sin(2 pi x) sin(2 pi y) cos(omega t), omega = 2 pi sqrt(2) c, on the periodic unit
    square, from w0, u0 = 0, q0 = Q(w0): the displacement the ODE (alpha = 1, beta = 0)
    recovers at T = 0.15 after 60 DIRK34 steps converges under refinement 4 -> 8."""
    import scipy.linalg as sla
    from oracle import wave
    c, T, N = 1.0, 0.15, 60
    errs = []
    for m in (4, 8):
        o, L, M = _wave(synth.quad_box(m, periodic=(True, True)), p, c * c, 1.0)
        n = o.ndof
        sx, om = _standing_wave(o, c)
        u, q, w = np.zeros(n), o.q(sx), sx.copy()
        dt = T / N
        A, b, cc = oracle.dirk_tableau(4)
        lu = sla.lu_factor(np.eye(L.shape[0]) - dt * A[0][0] * L)
        for _ in range(N):
            u, q, w = wave.wave_step(L, n, u, q, w, dt, 4, solve=lambda a, r: sla.lu_solve(lu, r))
        ex = sx * math.cos(om * T)
        errs.append(np.linalg.norm(w - ex) / np.linalg.norm(ex))
    rate = math.log2(errs[0] / errs[1])
    assert lo < rate < hi, (p, errs)


def test_wave_ode_closed_form_for_a_constant_velocity():
    """A constant u on a periodic mesh is a steady state of the (u, q) system (Q(const) = 0,
    R_s(const, 0) = 0); then alpha dw/dt + beta w = u has w(t) = u / beta + (w0 - u / beta)
    exp(-beta t / alpha), which DIRK34 reaches to its truncation error."""
    from oracle import wave
    o, L, M = _wave(synth.quad_box(3, periodic=(True, True)), 2, 1.0, 1.0)
    n = o.ndof
    U0, alpha, beta, T, N = 0.8, 2.0, 3.0, 0.5, 20
    u, q = np.full(n, U0), np.zeros(n * o.nd)
    w0 = np.linspace(-1.0, 1.0, n)
    w = w0.copy()
    for _ in range(N):
        u, q, w = wave.wave_step(L, n, u, q, w, T / N, 4, alpha=alpha, beta=beta)
    assert np.abs(u - U0).max() < 1e-12 and np.abs(q).max() < 1e-12
    ex = U0 / beta + (w0 - U0 / beta) * math.exp(-beta * T / alpha)
    assert np.abs(w - ex).max() < 1e-6 * np.abs(ex).max()


# --------------------------------------------- reduced-basis preconditioner (Section 3.3)
def _dense_jacobian(o):
    n = o.ndof
    u = synth.random_vector(n, 1)
    return np.stack([o.jvp(u, e) for e in np.eye(n)], axis=1)


def test_reduced_basis_preconditioner_is_exact_on_its_subspace():
    """P^{-1} J w = w for every w in span(V): the minimal-residual part solves J x = J w on
    the subspace exactly and the block-Jacobi part then sees a zero remainder. Dropping J
    from the remainder (r - C r) or restricting with V instead of J V fails it."""
    from oracle import rbpc
    o = oracle.Oracle(synth.quad_box((3, 3), affine=np.array([[1.0, 0.3], [0.1, 0.9]])), 2, oracle.CONVDIFF,
                      oracle.CASE_ZERO, (0.1, 1.0, 1.0, 0.5))
    J = _dense_jacobian(o)
    Binv = rbpc.block_jacobi_inverse(J, o.npe * o.ncu)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((o.ndof, 5))
    for _ in range(3):
        w = V @ rng.standard_normal(5)
        got = rbpc.rb_apply(J, Binv, V, J @ w)
        assert np.linalg.norm(got - w) <= 1e-11 * np.linalg.norm(w)
    # without a basis it is block-Jacobi
    x = rng.standard_normal(o.ndof)
    assert np.array_equal(rbpc.rb_apply(J, Binv, V[:, :0], x), Binv @ x)
    # J C is the orthogonal projector onto span(J V) (the minimal-residual reading; the
    # Galerkin C = V (V^T J V)^{-1} V^T gives an oblique one and fails), with C read off as
    # P^{-1} with no block-Jacobi part
    C = np.stack([rbpc.rb_apply(J, np.zeros_like(J), V, e) for e in np.eye(o.ndof)], axis=1)
    JC = J @ C
    assert np.linalg.norm(JC - JC.T) <= 1e-10 * np.linalg.norm(JC)
    assert np.linalg.norm(JC @ JC - JC) <= 1e-10 * np.linalg.norm(JC)
    # the coarse part does not depend on the basis chosen for the subspace
    T = rng.standard_normal((5, 5))
    assert np.linalg.norm(rbpc.rb_apply(J, Binv, V @ T, x) - rbpc.rb_apply(J, Binv, V, x)) <= 1e-10 * np.linalg.norm(x)


def test_reduced_basis_preconditioner_on_the_whole_space_is_the_inverse():
    """With a basis of the whole space (16 DOF) C = J^{-1} and P^{-1} = J^{-1}."""
    from oracle import rbpc
    o = oracle.Oracle(synth.quad_box((2, 2)), 1, oracle.CONVDIFF, oracle.CASE_ZERO, (0.1, 1.0, 1.0, 0.5))
    J = _dense_jacobian(o)
    assert o.ndof == 16
    Binv = rbpc.block_jacobi_inverse(J, o.npe * o.ncu)
    V = np.random.default_rng(2).standard_normal((16, 16))
    x = np.random.default_rng(3).standard_normal(16)
    assert np.linalg.norm(rbpc.rb_apply(J, Binv, V, x) - np.linalg.solve(J, x)) <= 1e-10 * np.linalg.norm(x)


# ---------------------------------------------------------- curved triangles (Section 4.2)
def test_curved_triangle_maps_reproduce_the_annulus_area():
    """sum_ij M_ij of the isoparametric triangles of the annulus 0.5 <= r <= 1: with
    straight sides (map degree 1) exactly the area of the inscribed polygonal annulus,
    n_t (r1^2 - r0^2) sin(2 pi / n_t) / 2; with degree 2 and 3 maps it approaches
    pi (r1^2 - r0^2) at order 4 (a map point out of order or a wrong map Jacobian breaks
    both)."""
    def area(n, pg):
        m = synth.tri_annulus(n, 4 * n, pg)
        o = oracle.Oracle(m, max(pg, 1), oracle.POISSON, oracle.CASE_LINEAR, (1.0, 1.0))
        return o.mass(np.ones(o.ndof)).sum()
    n = 4
    assert abs(area(n, 1) - 4 * n * 0.5 * 0.75 * math.sin(2 * math.pi / (4 * n))) < 1e-13
    ex = math.pi * 0.75
    for pg in (2, 3):
        e1, e2 = abs(area(4, pg) - ex), abs(area(8, pg) - ex)
        assert math.log2(e1 / e2) > 3.5, (pg, e1, e2)


@pytest.mark.parametrize("pg,p", [(1, 1), (2, 2), (2, 3), (3, 3)])
def test_curved_triangle_patch_test(pg, p):
    """A linear exact solution (no source) is reproduced on curved triangles whenever the
    map degree is at most p: the metric terms w det J dxi/dx and the face normals n sJ are
    polynomial in the reference coordinates and the quadrature integrates them exactly, so
    R(u) vanishes to rounding. A normal turned the wrong way or a transposed Jacobian fails it."""
    m = synth.tri_annulus(2, 8, pg)
    o = oracle.Oracle(m, p, oracle.POISSON, oracle.CASE_LINEAR, (1.0, 1.0), nq1=p + pg + 1)
    u = o.interpolate(0.0)
    assert np.abs(o.residual(u)).max() < 1e-12


def test_curved_triangle_poisson_converges_on_the_annulus():
    """Poisson with u = sin(pi x) sin(pi y) on the annulus, p = 2 with degree-2 maps: the
    L2 error of u falls at order about p + 1 under refinement (2 x 8 -> 4 x 16)."""
    errs = []
    for n in (2, 4):
        m = synth.tri_annulus(n, 4 * n, 2)
        o = oracle.Oracle(m, 2, oracle.POISSON, oracle.CASE_SINSIN, (1.0, 1.0))
        u, rc, _ = o.newton(np.zeros(o.ndof), newton_rtol=1e-12, gmres_rtol=1e-12, m=60, max_gmres=5000)
        assert rc == 0
        errs.append(o.l2_error(u)[0])
    assert math.log2(errs[0] / errs[1]) > 2.6, errs
