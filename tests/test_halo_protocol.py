"""The halo exchange between processes (Sec. 6.5), on CPU with gloo ranks:
each rank takes its block of a global field, packs its faces in the order
the library's face map gives (mg_halo_face_sites), sends them to the ranks
the library's plan names (mg_halo_plan) and checks that what it received
are exactly the global neighbours of its boundary sites; the GCR inner
products of a decomposed vector are the allreduce of the ranks' partial
sums.  No GPU is used: the plan and the face map are host code."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_07873_gb300 as gb
    return gb


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, dims, procs, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1612_07873_gb300 as gb
    import synthetic as syn
    from oracle import lattice as lat
    n = 3
    L = np.array(dims)
    P = np.array(procs)
    ld = tuple(int(v) for v in L // P)
    rc = np.array([(rank // int(np.prod(P[:m]))) % P[m] for m in range(4)])
    x = syn.gaussian_field((lat.volume(dims), n), 5)          # same global field everywhere
    lc = lat.coords(ld)
    gsite = lat.index(dims, lc + rc * np.array(ld))
    xl = x[gsite]
    plan = gb.mg_halo_plan(dims, procs, rank)
    ok = True
    reqs, bufs = [], {}
    for f in range(8):
        if plan["face_sites"][f] == 0:
            continue
        mu, side = f // 2, f % 2
        sites = gb.mg_halo_face_sites(ld, mu, side)
        ok &= len(sites) == plan["face_sites"][f]
        send = torch.from_numpy(np.ascontiguousarray(xl[sites]).view(np.float64).copy())
        recv = torch.empty_like(send)
        bufs[f] = recv
        reqs.append(dist.isend(send, plan["send_to"][f], tag=f))
        reqs.append(dist.irecv(recv, plan["recv_from"][f], tag=f))
    for q in reqs:
        q.wait()
    for f, recv in bufs.items():
        mu, side = f // 2, f % 2
        e = np.eye(4, dtype=np.int64)[mu]
        # recv 2mu: +mu partners of the sites at x_mu = l - 1; 2mu+1: -mu
        # partners of the sites at x_mu = 0
        sites = gb.mg_halo_face_sites(ld, mu, 1 - side)
        partner = lc[sites] + rc * np.array(ld) + (e if side == 0 else -e)
        want = x[lat.index(dims, partner)]
        got = recv.numpy().view(np.complex128).reshape(want.shape)
        ok &= bool(np.array_equal(got, want))
    # GCR inner product of decomposed vectors: allreduce of partial sums
    b = syn.gaussian_field((lat.volume(dims), n), 6)
    part = np.vdot(xl, b[gsite])
    t = torch.tensor([part.real, part.imag], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    full = np.vdot(x, b)
    ok &= abs(complex(t[0].item(), t[1].item()) - full) <= 1e-12 * np.sum(np.abs(x) * np.abs(b))
    out[rank] = bool(ok)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dims,procs", [((4, 6, 4, 4), (2, 1, 1, 1)),
                                        ((2, 4, 2, 6), (1, 1, 1, 2)),
                                        ((4, 4, 6, 4), (1, 2, 1, 1))])
def test_halo_exchange_protocol_gloo(lib, dims, procs):
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, dims, procs, out))
          for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert out[0] and out[1]


def test_halo_plan_and_face_map(lib):
    """The plan of a 2 x 1 x 3 x 2 split: neighbours wrap periodically, an
    undivided direction has no faces, and face maps list the boundary sites
    with the other coordinates in lexicographic order."""
    import paper_1612_07873_gb300 as gb
    from oracle import lattice as lat
    dims, procs = (4, 2, 6, 4), (2, 1, 3, 2)
    P = np.array(procs)
    for r in range(int(np.prod(P))):
        rc = [(r // int(np.prod(P[:m]))) % P[m] for m in range(4)]
        plan = gb.mg_halo_plan(dims, procs, r)
        for mu in range(4):
            for s in (0, 1):
                f = 2 * mu + s
                if procs[mu] == 1:
                    assert plan["face_sites"][f] == 0 and plan["send_to"][f] == -1
                    continue
                dn, up = list(rc), list(rc)
                dn[mu] = (rc[mu] - 1) % procs[mu]
                up[mu] = (rc[mu] + 1) % procs[mu]
                rid = lambda c: int(sum(c[m] * int(np.prod(P[:m])) for m in range(4)))  # noqa: E731
                assert plan["send_to"][f] == (rid(up) if s else rid(dn))
                assert plan["recv_from"][f] == (rid(dn) if s else rid(up))
        offs = [o for o, n in zip(plan["face_offset"], plan["face_sites"]) if n]
        assert offs == sorted(offs) and offs[0] == 0
    ld = (2, 2, 2, 2)
    c = lat.coords(ld)
    for mu in range(4):
        for s in (0, 1):
            sites = gb.mg_halo_face_sites(ld, mu, s)
            want = [i for i in range(16) if c[i, mu] == (ld[mu] - 1 if s else 0)]
            assert sites == want
    with pytest.raises(gb.MGError):
        gb.mg_halo_plan((4, 4, 4, 4), (3, 1, 1, 1), 0)
    with pytest.raises(gb.MGError):
        gb.mg_halo_plan((4, 4, 4, 4), (2, 1, 1, 1), 2)
