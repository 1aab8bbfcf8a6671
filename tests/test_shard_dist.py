"""Element-sharded LDG operators over two gloo ranks on the CPU (Section 3.5's
partitioned solve): the partition, the ghost layer and the exchange of ``shard.py``
drive rank-local evaluations, and the sharded R, J.v and GMRES solution equal the
single-rank oracle's. The rank-local arithmetic here is the oracle's (q-stage and the
residual with the exchanged q), so these tests pin the host logic; the same partitions
drive the library's sharded calls on the GPU (tests/test_gpu_shard.py)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

MU = (0.05, 0.3, 1.0, 0.5)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _mesh(kind):
    from paper_2205_07824_b300 import synth
    sh2 = np.array([[1.0, 0.3], [0.1, 0.9]])
    if kind == "quad_periodic":
        return synth.quad_box((6, 5), hi=(2.0, 1.5), periodic=(True, True), affine=sh2)
    if kind == "quad_dirichlet":
        return synth.quad_box((7, 6), affine=sh2)
    if kind == "hex":
        return synth.hex_box((3, 3, 4))
    return synth.tet_cube(2)


def _worker(rank, world, port, kind, out):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2205_07824_b300 import shard as shd, synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mesh = _mesh(kind)
        p = 2
        mu = MU + ((0.25,) if mesh.nd == 3 else ())
        sh = shd.partition(mesh, world, rank)
        ex = shd.GhostExchange(sh)
        res = {}
        for case in (oracle.CASE_ZERO, oracle.CASE_EXPSIN):
            og = oracle.Oracle(mesh, p, oracle.CONVDIFF, case, mu)
            ol = oracle.Oracle(sh.mesh, p, oracle.CONVDIFF, case, mu)
            nloc, nq = ol.npe * ol.ncu, ol.npe * ol.ncu * ol.nd
            u = synth.random_vector(og.ndof, 7)

            def sharded_residual(x_owned):
                # owned blocks known, ghosts filled by the exchange, q of the owned
                # elements exchanged before the residual stage
                x = torch.full((sh.n_local * nloc,), float("nan"), dtype=torch.float64)
                x[: sh.n_owned * nloc] = torch.as_tensor(x_owned)
                ex.exchange(x, nloc)
                q = torch.as_tensor(ol.q(x.numpy()))
                ex.exchange(q, nq)
                return ol.residual_with_q(x.numpy(), q.numpy())[: sh.n_owned * nloc]

            r_loc = sharded_residual(sh.owned_of(u, nloc))
            res[case] = (r_loc, og.residual(u)[sh.owned[0] * nloc: (sh.owned[-1] + 1) * nloc])
        packed = {k: (np.asarray(a).tolist(), np.asarray(c).tolist()) for k, (a, c) in res.items()}
        packed["sizes"] = (sh.n_owned, len(sh.ghosts))
        if kind == "quad_periodic":
            # all-periodic convection-diffusion keeps the constants in J's null space: no solve
            out[rank] = packed
            return
        # GMRES(m) on J x = b over the two ranks (R of CASE_ZERO is J.v): classical
        # Gram-Schmidt, every dot product summed over the ranks
        og = oracle.Oracle(mesh, p, oracle.CONVDIFF, oracle.CASE_ZERO, mu)
        ol = oracle.Oracle(sh.mesh, p, oracle.CONVDIFF, oracle.CASE_ZERO, mu)
        nloc, nq = ol.npe * ol.ncu, ol.npe * ol.ncu * ol.nd
        b = synth.random_vector(og.ndof, 11)
        bl = sh.owned_of(b, nloc)

        def jv(x_owned):
            x = torch.full((sh.n_local * nloc,), float("nan"), dtype=torch.float64)
            x[: sh.n_owned * nloc] = torch.as_tensor(x_owned)
            ex.exchange(x, nloc)
            q = torch.as_tensor(ol.q(x.numpy()))
            ex.exchange(q, nq)
            return ol.residual_with_q(x.numpy(), q.numpy())[: sh.n_owned * nloc]

        def gdot(a, c):
            t = torch.tensor([float(a @ c)], dtype=torch.float64)
            ex.allreduce_sum(t)
            return float(t.item())

        m, x = 40, np.zeros_like(bl)
        bn = np.sqrt(gdot(bl, bl))
        r = bl.copy()
        for _ in range(20):
            beta = np.sqrt(gdot(r, r))
            if beta <= 1e-11 * bn:
                break
            V = [r / beta]
            H = np.zeros((m + 1, m))
            for j in range(m):
                w = jv(V[j])
                for _pass in range(2):
                    h = np.array([gdot(V[i], w) for i in range(j + 1)])
                    H[: j + 1, j] += h
                    w = w - sum(h[i] * V[i] for i in range(j + 1))
                H[j + 1, j] = np.sqrt(gdot(w, w))
                V.append(w / H[j + 1, j])
            e1 = np.zeros(m + 1)
            e1[0] = beta
            y = np.linalg.lstsq(H, e1, rcond=None)[0]
            x = x + sum(y[i] * V[i] for i in range(m))
            r = bl - jv(x)
        xo, _, rc, _ = og.gmres(np.zeros(og.ndof), b, m=60, rtol=1e-12, maxit=3000)
        packed["gmres"] = (x.tolist(), xo[sh.owned[0] * nloc: (sh.owned[-1] + 1) * nloc].tolist())
        out[rank] = packed
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["quad_periodic", "quad_dirichlet", "hex", "tet"])
def test_sharded_residual_jvp_gmres_equal_single_rank_oracle(kind):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, kind, out), nprocs=2, join=True, start_method="spawn")
    import oracle
    for rank in (0, 1):
        res = out[rank]
        n_owned, n_ghost = res["sizes"]
        assert n_owned > 0 and n_ghost > 0
        for case in (oracle.CASE_ZERO, oracle.CASE_EXPSIN):
            got, ref = (np.array(a) for a in res[case])
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), (kind, rank, case)
        if kind != "quad_periodic":
            got, ref = (np.array(a) for a in res["gmres"])
            assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), (kind, rank)


def test_partition_covers_every_element_once_with_consistent_exchange_lists():
    from paper_2205_07824_b300 import shard as shd, synth
    mesh = synth.quad_box((7, 5), periodic=(True, False))
    nb = shd.face_neighbours(mesh)
    parts = [shd.partition(mesh, 3, r, nb) for r in range(3)]
    owned = np.concatenate([p.owned for p in parts])
    assert np.array_equal(np.sort(owned), np.arange(mesh.n_elem))
    for p in parts:
        # ghosts are exactly the off-rank face neighbours of owned elements
        want = set(nb[p.owned].ravel()) - set(p.owned.tolist()) - {-1}
        assert set(p.ghosts.tolist()) == want
        local = np.concatenate([p.owned, p.ghosts])
        for peer, idx in p.recv.items():
            q = parts[peer]
            qlocal = np.concatenate([q.owned, q.ghosts])
            # what the peer sends is, element for element, what this rank receives
            assert np.array_equal(local[idx], qlocal[q.send[p.rank]])
