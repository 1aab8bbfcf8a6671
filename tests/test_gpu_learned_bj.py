"""The learned correction of block-Jacobi (LDG_PC_MLP_BJ): the neighbour-trace features
against a brute-force search over node positions, the learned apply against the FP64
network oracle, and the trained network against plain block-Jacobi in the Newton-GMRES
solve of the isentropic vortex, trained on the (residual, Newton update) pairs that the
block-Jacobi solver itself produced."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, cuda, host, pair

pytestmark = pytest.mark.gpu
H = 128


def _node_positions(o, mesh):
    """Physical node positions [E][npe][nd]: the multilinear vertex map (quadrilaterals,
    hexahedra; vertices in lexicographic order) or the barycentric affine map
    (triangles, tetrahedra) at the reference nodes."""
    xi = o.ref_rules()[0][:, :mesh.nd]
    if mesh.etype in (synth.TRI, synth.TET):
        lam = (1.0 + xi) / 2.0
        L = np.concatenate([1.0 - lam.sum(1, keepdims=True), lam], 1)
        return np.einsum("na,ead->end", L, mesh.xyz)
    corners = np.array(np.meshgrid(*([[-1.0, 1.0]] * mesh.nd), indexing="ij")).reshape(mesh.nd, -1).T[:, ::-1]
    N = np.prod([(1.0 + xi[:, None, d] * corners[None, :, d]) / 2.0 for d in range(mesh.nd)], axis=0)
    return np.einsum("na,ead->end", N, mesh.xyz)


def _halo_brute(o, mesh, z, period=None):
    """h[K][c][i]: the sum over K's face neighbours of their z at the node placed where
    node i of K is (positions compared modulo the period), divided by ||z_K||."""
    X = _node_positions(o, mesh)
    nb = o.neighbours()
    E, npe, ncu = mesh.n_elem, o.npe, o.ncu
    zz = z.reshape(E, ncu, npe)
    h = np.zeros_like(zz)
    for K in range(E):
        for f in range(nb.shape[1]):
            N = nb[K, f]
            if N < 0:
                continue
            d = X[K][:, None, :] - X[N][None, :, :]
            if period is not None:
                d -= np.round(d / period) * period
            hit = np.argwhere(np.linalg.norm(d, axis=2) < 1e-9)
            for i, m in hit:
                h[K, :, i] += zz[N, :, m]
        nrm = np.linalg.norm(zz[K])
        h[K] /= nrm
    return h.ravel()


CASES = [
    ("quad_euler_per", lambda: synth.quad_box((5, 4), hi=(10.0, 10.0), periodic=(True, True), affine=SHEAR2), 3,
     oracle.EULER, oracle.CASE_VORTEX, np.array([10.0, 10.0]) @ SHEAR2.T),
    ("hex_cd", lambda: synth.hex_box((3, 3, 2), affine=SHEAR3), 2, oracle.CONVDIFF, oracle.CASE_EXPSIN, None),
    ("tet_poisson", lambda: synth.tet_cube(2, affine=SHEAR3), 2, oracle.POISSON, oracle.CASE_SINSIN, None),
    ("tri_cd", lambda: synth.tri_unstructured(4, seed=2), 3, oracle.CONVDIFF, oracle.CASE_EXPSIN, None),
]


@pytest.mark.parametrize("name,mk,p,model,case,period", CASES, ids=[c[0] for c in CASES])
def test_halo_features_match_brute_force(name, mk, p, model, case, period):
    mesh = mk()
    o, g = pair(mesh, p, model, case, gmres_m=2)
    z = synth.random_vector(o.ndof, 3)
    h = host(g.halo_features(cuda(z)))
    if period is not None and mesh.etype == synth.QUAD:
        # the periodic box is sheared: compare modulo each lattice vector in turn
        per = np.array([[10.0, 0.0], [0.0, 10.0]]) @ SHEAR2.T
        ref = _halo_periodic(o, mesh, z, per)
    else:
        ref = _halo_brute(o, mesh, z)
    assert np.abs(h - ref).max() <= 1e-12 * np.abs(ref).max(), name


def _halo_periodic(o, mesh, z, lattice):
    """_halo_brute on a periodic mesh whose period lattice has the rows of `lattice`."""
    X = _node_positions(o, mesh)
    nb = o.neighbours()
    E, npe, ncu = mesh.n_elem, o.npe, o.ncu
    zz = z.reshape(E, ncu, npe)
    h = np.zeros_like(zz)
    shifts = [a * lattice[0] + b * lattice[1] for a in (-1, 0, 1) for b in (-1, 0, 1)]
    for K in range(E):
        for f in range(nb.shape[1]):
            N = nb[K, f]
            if N < 0:
                continue
            best = None
            for sh in shifts:
                d = np.linalg.norm(X[K][:, None, :] - X[N][None, :, :] - sh, axis=2)
                hit = np.argwhere(d < 1e-9)
                if len(hit):
                    best = hit
                    break
            for i, m in (best if best is not None else []):
                h[K, :, i] += zz[N, :, m]
        h[K] /= np.linalg.norm(zz[K])
    return h.ravel()


def _bf16_round(x):
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def test_learned_bj_apply_matches_oracle():
    """y = ||z_K|| net(z_K / ||z_K||, h_K) with z = BJ^{-1} x from the context's blocks."""
    mesh = synth.quad_box((6, 5), hi=(10.0, 10.0), periodic=(True, True))
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, gmres_m=4, precond=3)
    n = o.npe * o.ncu
    u = synth.random_euler_state(mesh.n_elem, o.npe, 6)
    g.precond_setup(cuda(u))
    g.mlp_init(seed=4)
    theta = g.mlp_params()
    x = synth.random_vector(o.ndof, 5)
    y = host(g.mlp_bj_apply(cuda(x)))
    z = host(g.precond_apply(cuda(x)))
    hh = host(g.halo_features(cuda(z)))
    th = _bf16_round(theta)
    off = 0
    for sh in omlp.shapes(2 * n, H, n):
        k = int(np.prod(sh))
        if len(sh) == 1:
            th[off:off + k] = np.float32(theta[off:off + k])
        off += k
    ref = omlp.apply(th, z.reshape(-1, n), 2 * n, H, n, U=np.float32(hh).astype(np.float64).reshape(-1, n),
                     act_round=omlp.round_bf16).ravel()
    assert np.linalg.norm(y - ref) <= 1e-3 * np.linalg.norm(ref)


def test_learned_bj_correction_against_block_jacobi():
    """Train on the plain block-Jacobi solver's (residual, update) pairs over a few BDF2
    steps of the 16 x 16 vortex: its Newton steps (R(u_k), delta_k) and its Arnoldi steps
    (J z_j, z_j). The next step with the learned correction reaches 1e-8 without falling
    back, in a GMRES iteration count within 1.5x of block-Jacobi's (measured 26 against 23;
    trained on the Newton pairs alone it took 45, and on a 32 x 32 mesh 1,352 against 32).
    Both counts are printed: the learned correction does not beat block-Jacobi here."""
    import torch
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3, precond=1)
    cap = 400
    X = torch.empty(cap * o.ndof, dtype=torch.float64, device="cuda")
    T = torch.empty_like(X)
    U = torch.empty_like(X)
    un, unm1 = g.interpolate(0.0), g.interpolate(-dt)
    used, t = 0, 0.0
    for _ in range(8):
        g.set_time(2, t + dt, dt, un, unm1)
        u = un.clone()
        c, _ = g.newton_collect_updates(u, X[used * o.ndof:], T[used * o.ndof:], U[used * o.ndof:], cap - used, 3)
        used += c
        unm1.copy_(un)
        un.copy_(u)
        t += dt
    assert used >= 100
    g.mlp_init(seed=1)
    nd = used * o.ndof
    rep = g.mlp_train(X[:nd], T[:nd], U[:nd], epochs=60, batch=4096, lr=1e-3)
    assert rep["loss_last"] <= rep["loss_first"], rep
    its = {}
    for pc in (1, 3):
        _, g2 = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3, precond=pc)
        if pc == 3:
            g2.mlp_init(seed=1)
            g2.mlp_params(g.mlp_params())
        g2.set_time(2, t + dt, dt, un, unm1)
        u = un.clone()
        r = g2.newton_gmres(u)
        assert r["rfinal"] <= 1e-8 * r["r0"], r
        its[pc] = r
    print("GMRES iterations: block-Jacobi", its[1]["gmres_iters"], "learned correction", its[3]["gmres_iters"],
          "fallbacks", its[3]["pc_fallbacks"], "train", rep, "pairs", used)
    assert its[3]["pc_fallbacks"] == 0
    assert its[3]["gmres_iters"] <= 1.5 * its[1]["gmres_iters"], its
