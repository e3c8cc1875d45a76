"""Five-block coarse-link storage: only X and the forward links are stored,
the backward links are rebuilt from the neighbour's forward link with the
gamma5 relation.  Galerkin-built links satisfy that relation, so the apply
must match the oracle's nine-block stencil apply."""
import numpy as np
import pytest
import torch

import synthetic as syn
from gpu_helpers import make_ctx, oracle_fine, rel_l2, to_dev, to_np
from oracle import lattice as lat, multigrid as mgo

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3, 3: 5e-3, 4: 5e-3}


def _ctx5(gb, dims, block, nv, prec, U=None, **kw):
    p = gb.default_params(dims=dims, block=[block], nvec=[nv], mass=-0.2, csw=1.0, nlevels=2,
                          prec_fine=0 if prec == 0 else 1, prec_coarse=prec, link_slots=5, **kw)
    if U is None:
        U = syn.gauge_field(dims, 0.3, 1)
    return gb.Multigrid(p, to_dev(U)), U


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dims,block,nv", [((8, 8, 8, 8), (2, 2, 2, 2), 24),
                                           ((8, 4, 4, 8), (2, 2, 2, 2), 16),
                                           ((6, 4, 4, 4), (2, 2, 2, 2), 24)])
def test_five_block_apply_matches_oracle(gpu_lib, prec, dims, block, nv):
    gb = gpu_lib
    mg, U = _ctx5(gb, dims, block, nv, prec)
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 61)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    gb.mg_build_coarse(mg.ctx, 0)
    cop = mgo.galerkin(oracle_fine(U, dims), mgo.block_orthonormalise(v, dims, block), block)
    x = syn.gaussian_field((cop.vol, cop.nd), 62)
    dt = torch.complex128 if prec == 0 else torch.complex64
    y = torch.empty((cop.vol, cop.nd), dtype=dt, device="cuda")
    gb.mg_coarse_apply(mg.ctx, 1, y, to_dev(x, dt))
    torch.cuda.synchronize()
    err = rel_l2(to_np(y), cop.apply(x))
    assert err < TOL[prec], err
    mg.close()


def test_five_block_three_level_solve(gpu_lib):
    gb = gpu_lib
    dims = (8, 8, 8, 16)
    U = syn.gauge_field(dims, 0.4, 3)
    p = gb.default_params(dims=dims, block=[(2, 2, 2, 2), (2, 2, 2, 2)], nvec=[12, 16],
                          mass=-0.3, csw=1.0, nlevels=3, prec_fine=1, prec_coarse=2,
                          link_slots=5)
    mg = gb.Multigrid(p, to_dev(U))
    for l in (0, 1):
        gb.mg_setup_nullvecs(mg.ctx, l, None)
        gb.mg_build_coarse(mg.ctx, l)
    b = syn.gaussian_field((lat.volume(dims), 12), 63)
    x = torch.zeros((lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    st = gb.mg_gcr_solve(mg.ctx, x, to_dev(b), 1e-10, 300)
    r = b - oracle_fine(U, dims, -0.3, 1.0).apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-10
    mg.close()
