"""Domain-decomposed coarse apply with a one-site halo (Sec. 6.5), every
sub-domain emulated on this GPU: scatter the global vector to the ranks,
pack all faces of each rank in one kernel, exchange into the receivers'
halo buffers, apply Eq. (3) per rank and gather.  The result must equal
the oracle's undecomposed apply on the whole lattice."""
import numpy as np
import pytest
import torch

import synthetic as syn
from gpu_helpers import make_ctx, rel_l2, to_dev, to_np
from oracle import dirac, lattice as lat

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}

CASES = [
    # fine lattice, aggregates, Nv, ranks per direction -> local coarse extents
    ((8, 8, 8, 8), (2, 2, 2, 2), 8, (2, 1, 1, 2)),      # local 2x4x4x2 (extent 2)
    ((12, 8, 8, 12), (2, 2, 2, 2), 8, (2, 2, 1, 2)),    # local 3x2x4x3 (extents 3 and 2)
    ((12, 8, 8, 12), (2, 2, 2, 2), 24, (1, 2, 2, 3)),   # n = 48, 12 ranks, local 6x2x2x2
    ((8, 8, 8, 8), (2, 2, 2, 2), 8, (4, 1, 1, 1)),      # local extent 1: both faces one slab
    ((8, 8, 8, 16), (2, 2, 2, 2), 16, (2, 2, 2, 2)),    # n = 32, 16 ranks, local 2x2x2x4
]


def _decomposed_apply(gb, mg, procs, x, dt):
    H = gb.Halo(mg.ctx, 1, procs)
    lvol = int(np.prod(H.local_dims))
    n = x.shape[1]
    xg = to_dev(x, dt)
    lx = [torch.empty((lvol, n), dtype=dt, device="cuda") for _ in range(H.nranks)]
    ly = [torch.empty_like(v) for v in lx]
    for r in range(H.nranks):
        H.scatter(r, lx[r], xg)
    for r in range(H.nranks):
        H.pack(r, lx[r])
    H.exchange()
    for r in range(H.nranks):
        H.apply(r, ly[r], lx[r])
    yg = torch.full_like(xg, float("nan"))
    for r in range(H.nranks):
        H.gather(r, yg, ly[r])
    torch.cuda.synchronize()
    launches = H.launch_count()
    H.close()
    return to_np(yg), launches


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dims,block,nv,procs", CASES)
def test_decomposed_apply_matches_undecomposed_oracle(gpu_lib, dims, block, nv, procs, prec):
    gb = gpu_lib
    mg, _ = make_ctx(gb, dims, [block], [nv], prec_fine=min(prec, 1), prec_coarse=prec)
    cd = lat.coarse_dims(dims, block)
    n, V = 2 * nv, lat.volume(cd)
    links = syn.gaussian_field((V, 9, n, n), 7 + nv)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = syn.gaussian_field((V, n), 8 + nv)
    want = dirac.StencilOp(cd, links).apply(x)
    dt = torch.complex128 if prec == 0 else torch.complex64
    got, launches = _decomposed_apply(gb, mg, procs, x, dt)
    err = rel_l2(got, want)
    assert err < TOL[prec], err
    nranks = int(np.prod(procs))
    assert launches >= 4 * nranks  # link split, scatter, pack, apply per rank (+ gather)
    mg.close()


def test_single_rank_equals_plain_apply(gpu_lib):
    """procs = 1 everywhere: no faces, the halo apply is the plain apply."""
    gb = gpu_lib
    dims, block, nv = (8, 8, 8, 8), (2, 2, 2, 2), 8
    mg, _ = make_ctx(gb, dims, [block], [nv])
    cd = lat.coarse_dims(dims, block)
    n, V = 2 * nv, lat.volume(cd)
    links = syn.gaussian_field((V, 9, n, n), 3)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = syn.gaussian_field((V, n), 4)
    got, _ = _decomposed_apply(gb, mg, (1, 1, 1, 1), x, torch.complex128)
    y = torch.empty((V, n), dtype=torch.complex128, device="cuda")
    gb.mg_coarse_apply(mg.ctx, 1, y, to_dev(x))
    torch.cuda.synchronize()
    assert rel_l2(got, to_np(y)) < 1e-14
    mg.close()


def test_halo_rejects_bad_splits(gpu_lib):
    gb = gpu_lib
    mg, _ = make_ctx(gb, (8, 8, 8, 8), [(2, 2, 2, 2)], [8])
    with pytest.raises(gb.MGError):      # operator not built yet
        gb.Halo(mg.ctx, 1, (2, 1, 1, 1))
    V = 256
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(syn.gaussian_field((V, 9, 16, 16), 1)))
    with pytest.raises(gb.MGError):      # 4 is not a multiple of 3
        gb.Halo(mg.ctx, 1, (3, 1, 1, 1))
    with pytest.raises(gb.MGError):      # the fine level has no coarse operator
        gb.Halo(mg.ctx, 0, (2, 1, 1, 1))
    mg.close()
