"""Learned per-element preconditioner: the GPU forward/backward kernels against the
FP64 oracle of the network, and what the trained network gains in the Newton-GMRES
solve of the isentropic vortex over the same solve without it. The network is
trained on triples (v, (block-Jacobi)^{-1} v, u) that the plain block-Jacobi solver
produces for its Arnoldi vectors."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2205_07824_b300 import synth
from gpu_util import cuda, host, pair

pytestmark = pytest.mark.gpu
H = 128


def _bf16_round(x):
    """Round FP64 values to the nearest BF16 (ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def _ctx():
    mesh = synth.quad_box((6, 5), hi=(10.0, 10.0), periodic=(True, True))
    return pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, gmres_m=4)


def test_mlp_loss_and_gradient_match_fp64_oracle():
    o, g = _ctx()
    n = o.npe * o.ncu
    g.mlp_init(seed=3)
    theta = g.mlp_params()
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, n))
    X[7] = 0.0                                  # zero-norm pair: masked out
    T = rng.standard_normal((300, n)) * 0.3
    U = synth.random_euler_state(300, o.npe, 2).reshape(300, n)
    loss, grad = g.mlp_loss_grad(cuda(X), cuda(T), cuda(U))
    # the oracle sees the FP32 master weights and FP32-rounded inputs the GPU trains on
    U32 = np.float32(U).astype(np.float64)
    lo, go = omlp.loss_grad(np.float32(theta).astype(np.float64), X, T, 2 * n, H, n, U=U32)
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.linalg.norm(grad - go) <= 2e-5 * np.linalg.norm(go)


def test_mlp_apply_matches_oracle_with_bf16_weights():
    o, g = _ctx()
    n = o.npe * o.ncu
    g.mlp_init(seed=4)
    theta = g.mlp_params()
    v = synth.random_vector(o.ndof, 5)
    u = synth.random_euler_state(o.mesh.n_elem, o.npe, 6)
    y = host(g.mlp_apply(cuda(u), cuda(v)))
    th = _bf16_round(theta)
    # biases stay FP32 in the kernel; only the weight matrices are BF16
    off = 0
    for sh in omlp.shapes(2 * n, H, n):
        k = int(np.prod(sh))
        if len(sh) == 1:
            th[off:off + k] = np.float32(theta[off:off + k])
        off += k
    # the tensor-core inference path also stores the input and the hidden activations in BF16
    ref = omlp.apply(th, v.reshape(-1, n), 2 * n, H, n, U=np.float32(u).astype(np.float64).reshape(-1, n),
                     act_round=omlp.round_bf16).ravel()
    # FP32 accumulation order differs (tensor cores vs FP64): a few activations round to the
    # neighbouring BF16 value (2^-8 relative), which bounds the output difference
    assert np.linalg.norm(y - ref) <= 1e-3 * np.linalg.norm(ref)
    ref_plain = omlp.apply(th, v.reshape(-1, n), 2 * n, H, n, U=np.float32(u).astype(np.float64).reshape(-1, n)).ravel()
    assert np.linalg.norm(y - ref_plain) <= 2e-2 * np.linalg.norm(ref_plain)
    # the SIMT path (FP32 activations) matches the unrounded reference much more tightly,
    # which shows the result above came from the tensor-core path
    import os
    os.environ["LDG_MLP_SIMT"] = "1"
    try:
        g.mlp_params(theta)                     # re-uploads the weights and re-selects the path
        y_simt = host(g.mlp_apply(cuda(u), cuda(v)))
    finally:
        del os.environ["LDG_MLP_SIMT"]
    assert np.linalg.norm(y_simt - ref_plain) <= 1e-4 * np.linalg.norm(ref_plain)
    assert np.linalg.norm(y - y_simt) > 1e-4 * np.linalg.norm(ref_plain)


def test_trained_mlp_preconditioner_beats_no_preconditioner():
    mesh = synth.quad_box(16, hi=(10.0, 10.0), periodic=(True, True))
    dt = 0.05
    o, g = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3, precond=1)
    import torch
    # training triples from the plain (block-Jacobi) solver over a few BDF2 steps
    cap = 200
    X = torch.empty(cap * o.ndof, dtype=torch.float64, device="cuda")
    T = torch.empty_like(X)
    U = torch.empty_like(X)
    un, unm1 = g.interpolate(0.0), g.interpolate(-dt)
    used = 0
    t = 0.0
    for _ in range(6):
        g.set_time(2, t + dt, dt, un, unm1)
        u = un.clone()
        c, _ = g.newton_gmres_collect(u, X[used * o.ndof:], T[used * o.ndof:], U[used * o.ndof:], cap - used)
        used += c
        unm1.copy_(un)
        un.copy_(u)
        t += dt
    assert used > 20
    g.mlp_init(seed=1)
    nd = used * o.ndof
    rep = g.mlp_train(X[:nd], T[:nd], U[:nd], epochs=60, batch=2048, lr=1e-3)
    # starting from the least-squares linear map, Adam lowers the loss further
    assert rep["loss_last"] <= rep["loss_first"], rep
    # next step: no preconditioner vs the trained network
    its = {}
    for pc in (0, 1, 2):
        o2, g2 = pair(mesh, 3, oracle.EULER, oracle.CASE_VORTEX, newton_rtol=1e-8, gmres_rtol=1e-3, precond=pc)
        if pc == 2:
            g2.mlp_init(seed=1)
            g2.mlp_params(g.mlp_params())
        g2.set_time(2, t + dt, dt, un, unm1)
        u = un.clone()
        r = g2.newton_gmres(u)
        assert r["rfinal"] <= 1e-8 * r["r0"]
        its[pc] = r
    print("GMRES iterations: none", its[0]["gmres_iters"], "block-Jacobi", its[1]["gmres_iters"],
          "learned", its[2]["gmres_iters"], "fallbacks", its[2]["pc_fallbacks"], "train", rep)
    assert its[2]["pc_fallbacks"] == 0
    # the learned preconditioner needs no per-step block extraction, and cuts the
    # Krylov iterations to within a small factor of the exact block-Jacobi one
    assert its[2]["gmres_iters"] * 2 < its[0]["gmres_iters"]
    assert its[2]["pc_setups"] == 0
