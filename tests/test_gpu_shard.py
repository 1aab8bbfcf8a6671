"""The library's element-sharded R, J.v and GMRES (ldg_shard_*) on one GPU: two ranks run
as two host threads, each with its own context on its local mesh (owned elements, then
ghosts) and stream, and an in-process transport that copies ghost blocks between the
two contexts and sums the dot products. No kernel waits on another: the ranks meet only
on the host, inside the transport, after each stream has drained. The owned parts equal
the single-rank oracle's R and J.v (1e-12) and its GMRES solution (1e-8)."""
import threading

import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, cuda, host

pytestmark = pytest.mark.gpu


class _Hub:
    def __init__(self):
        self.barrier = threading.Barrier(2, timeout=60)
        self.bufs = [None, None]


class _InProcess:
    """Transport of rank `rank` of two ranks in one process (the role NCCL plays
    between processes): ghosts copied from the peer's vector, dot products summed in
    rank order on both ranks."""

    def __init__(self, hub, shards, rank):
        import torch
        self.hub, self.rank, self.peer = hub, rank, 1 - rank
        me, other = shards[rank], shards[1 - rank]
        self.recv = torch.as_tensor(me.recv.get(self.peer, np.zeros(0, dtype=np.int64)), device="cuda")
        self.src = torch.as_tensor(other.send.get(rank, np.zeros(0, dtype=np.int64)), device="cuda")

    def exchange(self, x, block):
        import torch
        h = self.hub
        h.bufs[self.rank] = x
        h.barrier.wait()
        if len(self.recv):
            x.view(-1, block)[self.recv] = h.bufs[self.peer].view(-1, block)[self.src]
        torch.cuda.synchronize()
        h.barrier.wait()

    def allreduce_sum(self, buf):
        import torch
        h = self.hub
        h.bufs[self.rank] = buf.clone()
        h.barrier.wait()
        tot = h.bufs[0] + h.bufs[1]
        torch.cuda.synchronize()
        h.barrier.wait()
        buf.copy_(tot)
        torch.cuda.synchronize()


def _run_ranks(fn):
    errs = []

    def body(r):
        try:
            fn(r)
        except BaseException as e:      # surfaced after the join
            errs.append(e)

    th = [threading.Thread(target=body, args=(r,)) for r in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]


@pytest.mark.parametrize("kind", ["quad", "hex", "tet"])
def test_sharded_operators_and_gmres_on_one_gpu(kind):
    import torch
    from paper_2205_07824_b300 import shard as shd
    from paper_2205_07824_b300.ldg import LDG, CONVDIFF
    mesh = {"quad": lambda: synth.quad_box((7, 6), affine=SHEAR2), "hex": lambda: synth.hex_box((3, 3, 4)),
            "tet": lambda: synth.tet_cube(2)}[kind]()
    mu = (0.05, 0.3, 1.0, 0.5, 0.25)[: 2 + mesh.nd]
    p = 2
    nb = shd.face_neighbours(mesh)
    shards = [shd.partition(mesh, 2, r, nb) for r in (0, 1)]
    hub = _Hub()
    results = {}
    for case in (oracle.CASE_ZERO, oracle.CASE_EXPSIN):
        og = oracle.Oracle(mesh, p, oracle.CONVDIFF, case, mu)
        u = synth.random_vector(og.ndof, 3)
        b = synth.random_vector(og.ndof, 5)
        ctxs = [LDG(s.mesh, p, CONVDIFF, case, mu, nq1=og.nq1, gmres_m=30, gmres_rtol=1e-12, max_restarts=200,
                    stream=torch.cuda.Stream()) for s in shards]
        comms = [shd.make_comm(_InProcess(hub, shards, r), shards[r].n_local) for r in (0, 1)]
        nloc = ctxs[0].n_pe

        def full(vec, r):
            x = torch.full((shards[r].n_local * nloc,), float("nan"), dtype=torch.float64, device="cuda")
            x[: shards[r].n_owned * nloc] = cuda(shards[r].owned_of(vec, nloc))
            return x

        def rank(r):
            g, sh = ctxs[r], shards[r]
            g.shard_setup(sh.n_owned, comms[r])
            out = {"R": host(g.shard_residual(full(u, r)))[: sh.n_owned * nloc]}
            if case == oracle.CASE_ZERO:
                out["Jv"] = host(g.shard_jvp(full(u, r)))[: sh.n_owned * nloc]
                x, rep = g.shard_gmres(full(b, r))
                out["x"], out["rep"] = host(x)[: sh.n_owned * nloc], rep
            results[(case, r)] = out

        _run_ranks(rank)
        R = np.concatenate([results[(case, r)]["R"] for r in (0, 1)])
        ref = og.residual(u)
        assert np.linalg.norm(R - ref) <= 1e-12 * np.linalg.norm(ref), (kind, case)
        if case == oracle.CASE_ZERO:
            Jv = np.concatenate([results[(case, r)]["Jv"] for r in (0, 1)])
            assert np.linalg.norm(Jv - og.jvp(np.zeros(og.ndof), u)) <= 1e-12 * np.linalg.norm(Jv), kind
            x = np.concatenate([results[(case, r)]["x"] for r in (0, 1)])
            xo, _, _, _ = og.gmres(np.zeros(og.ndof), b, m=60, rtol=1e-12, maxit=3000)
            assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo), kind
            reps = [results[(case, r)]["rep"] for r in (0, 1)]
            assert reps[0]["gmres_iters"] == reps[1]["gmres_iters"] > 0
