"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 CPU oracle)."""
import numpy as np

import oracle
from paper_2205_07824_b300 import synth

SHEAR2 = np.array([[1.0, 0.3], [0.1, 0.9]])
SHEAR3 = np.array([[1.0, 0.2, 0.1], [0.0, 0.9, 0.15], [0.05, 0.0, 1.1]])

# FP64 parity bar: relative 2-norm and scaled max-norm of the difference
RTOL_2 = 1e-12
RTOL_MAX = 1e-11


def assert_parity(gpu, ref, rtol2=RTOL_2, rtolmax=RTOL_MAX, what=""):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    d = gpu - ref
    n2 = np.linalg.norm(ref)
    e2 = np.linalg.norm(d) / max(n2, 1e-300)
    emax = np.abs(d).max() / max(np.abs(ref).max(), 1e-300)
    assert e2 <= rtol2 and emax <= rtolmax, f"{what}: rel2 {e2:.3e} relmax {emax:.3e}"
    return e2, emax


def mu_for(model, nd):
    if model == oracle.POISSON:
        return (1.0, 1.0)
    if model == oracle.CONVDIFF:
        return (0.05, 0.3, 1.0, 0.5, 0.25)[: 2 + nd]
    if model == oracle.NS:
        return (1.4, 10.0, 0.72)       # gamma, Re, Pr: Re = 10 makes the viscous terms large
    return (1.4,)


def pair(mesh, p, model, case, mu=None, **kw):
    """The oracle and the CUDA operator for the same problem."""
    from paper_2205_07824_b300.ldg import LDG
    mu = mu_for(model, mesh.nd) if mu is None else mu
    o = oracle.Oracle(mesh, p, model, case, mu)
    g = LDG(mesh, p, model, case, mu, nq1=o.nq1, **kw)
    assert g.n_dof == o.ndof
    return o, g


def state(o, mesh, seed):
    if o.model in (oracle.EULER, oracle.NS):
        return synth.random_euler_state(mesh.n_elem, o.npe, seed)
    return synth.random_vector(o.ndof, seed)


def cuda(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
