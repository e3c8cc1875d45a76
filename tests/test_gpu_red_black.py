"""Red-black (Schur complement) preconditioning on the GPU against the
oracle (Secs. 3.3, 7.1): the Schur operator S = A_o - H_oe A_e^-1 H_eo of
the fine and of coarse levels, and MG solves whose smoothers and coarsest
solve work on S.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac, lattice as lat, schur as rb, solvers
from gpu_helpers import make_ctx, oracle_fine, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3}
CDT = {0: torch.complex128, 1: torch.complex64, 2: torch.complex64}


@pytest.mark.parametrize("antiperiodic", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
def test_schur_apply_fine(gpu_lib, prec, antiperiodic):
    gb = gpu_lib
    dims = (4, 4, 2, 6)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=prec, prec_coarse=prec,
                     antiperiodic=antiperiodic, eps=0.5, red_black=1)
    S = rb.SchurOp(dirac.wilson_clover_op(U, dims, -0.2, 1.0, bool(antiperiodic)))
    nr = 2
    x = syn.gaussian_field((nr, lat.volume(dims) // 2, 12), 91)
    y = torch.empty(x.shape, dtype=CDT[prec], device="cuda")
    gb.mg_schur_apply(mg.ctx, 0, y, to_dev(x, CDT[prec]), nrhs=nr)
    want = np.stack([S.apply(v) for v in x])
    assert rel_l2(to_np(y), want) < TOL[prec]
    mg.close()


@pytest.mark.parametrize("cdims,nv", [((4, 2, 2, 4), 8), ((2, 2, 4, 2), 24), ((2, 4, 2, 2), 32)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_schur_apply_coarse(gpu_lib, cdims, nv, prec):
    """Random coarse links with a dominant site block (X + 3 I); n = 16, 48, 64."""
    gb = gpu_lib
    dims = tuple(2 * c for c in cdims)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], prec_fine=0 if prec == 0 else 1,
                     prec_coarse=prec, red_black=1)
    n, vol = 2 * nv, lat.volume(cdims)
    links = syn.gaussian_field((vol, 9, n, n), 92) / np.sqrt(n)
    links[:, 0] += 3.0 * np.eye(n)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    S = rb.SchurOp(dirac.StencilOp(cdims, links))
    x = syn.gaussian_field((vol // 2, n), 93)
    y = torch.empty(x.shape, dtype=CDT[prec], device="cuda")
    gb.mg_schur_apply(mg.ctx, 1, y, to_dev(x, CDT[prec]))
    assert rel_l2(to_np(y), S.apply(x)) < TOL[prec]
    mg.close()


def test_red_black_two_level_solve_matches_oracle_fp64(gpu_lib):
    """The small 2-level FP64 workload with red-black smoothing and coarsest
    solve: same outer iteration count and history as the oracle's."""
    gb = gpu_lib
    w = syn.WORKLOADS["c1_8^4_2lvl_fp64"]
    dims, block, nv = w["dims"], w["block"][0], w["nvec"][0]
    mg, U = make_ctx(gb, dims, [block], [nv], mass=w["mass"], csw=w["csw"], eps=w["eps"],
                     seed=w["seed"], sweeps=w["sweeps"], red_black=1)
    vol = lat.volume(dims)
    x0 = syn.gaussian_field((nv, vol, 12), w["seed"], stream=10)
    gb.mg_setup_nullvecs(mg.ctx, 0, to_dev(x0))
    gb.mg_build_coarse(mg.ctx, 0)
    b = syn.gaussian_field((vol, 12), w["seed"], stream=99)
    x = torch.zeros((vol, 12), dtype=torch.complex128, device="cuda")
    st = gb.mg_gcr_solve(mg.ctx, x, to_dev(b), 1e-10, 100)
    op = oracle_fine(U, dims, w["mass"], w["csw"])
    plain = solvers.MultigridHierarchy.build(op, [x0], w["sweeps"], [block])
    hier = solvers.MultigridHierarchy(plain.ops, plain.Qs, plain.blocks,
                                      solvers.MGParams(schur=True))
    ref = hier.solve(b, 1e-10, 100)
    assert st["iters"] == ref.iters
    h = np.array(st["history"])
    assert np.abs(h - np.array(ref.history)).max() / np.array(ref.history).min() < 1e-6
    assert st["true_residual"] <= 1e-10
    assert rel_l2(to_np(x), ref.x) < 1e-9
    mg.close()


def _three_level(gb, red_black, prec_coarse=1):
    dims = (8, 8, 8, 8)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2), (2, 2, 2, 2)], [16, 16], prec_fine=1,
                     prec_coarse=prec_coarse, eps=0.4, mass=-0.3, sweeps=8, red_black=red_black)
    for l in range(2):
        gb.mg_setup_nullvecs(mg.ctx, l, None)
        gb.mg_build_coarse(mg.ctx, l)
    return mg, U, dims


@pytest.mark.parametrize("prec_coarse", [1, 2])
def test_red_black_three_level_fewer_iterations(gpu_lib, prec_coarse):
    gb = gpu_lib
    b = to_dev(syn.gaussian_field((8 ** 4, 12), 94))
    its = {}
    for red_black in (0, 1):
        mg, U, dims = _three_level(gb, red_black, prec_coarse)
        x = torch.zeros_like(b)
        st = gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 300)
        assert st["true_residual"] <= 1e-10
        res = np.linalg.norm(to_np(b) - oracle_fine(U, dims, -0.3).apply(to_np(x)))
        assert res / np.linalg.norm(to_np(b)) <= 1.05e-10
        its[red_black] = (st["iters"], st["level_iters"])
        mg.close()
    assert its[1][0] <= its[0][0], its


def test_red_black_multi_rhs_matches_single(gpu_lib):
    gb = gpu_lib
    mg, U, dims = _three_level(gb, 1)
    nr = 4
    b = syn.gaussian_field((nr, 8 ** 4, 12), 95)
    bd = to_dev(b)
    x = torch.zeros_like(bd)
    multi = gb.mg_gcr_solve_multi(mg.ctx, x, bd, nr, 1e-10, 300)
    for v in range(nr):
        xv = torch.zeros_like(bd[v])
        single = gb.mg_gcr_solve(mg.ctx, xv, bd[v].contiguous(), 1e-10, 300)
        assert multi[v]["true_residual"] <= 1.05e-10
        assert abs(multi[v]["iters"] - single["iters"]) <= 1
        assert rel_l2(to_np(x[v]), to_np(xv)) < 1e-6
    mg.close()


def test_odd_extent_level_has_no_red_black_form(gpu_lib):
    """Coarse extent 3: that level keeps the plain smoother/solver (no
    checkerboard with periodic wrap); the solve still converges."""
    gb = gpu_lib
    dims = (6, 4, 4, 4)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [8], red_black=1, sweeps=6)
    gb.mg_setup_nullvecs(mg.ctx, 0, None)
    gb.mg_build_coarse(mg.ctx, 0)
    x = torch.zeros((lat.volume((3, 2, 2, 2)) // 2, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.MGError) as e:
        gb.mg_schur_apply(mg.ctx, 1, torch.empty_like(x), x)
    assert e.value.status == gb.MG_ERR_STATE
    b = to_dev(syn.gaussian_field((lat.volume(dims), 12), 96))
    xs = torch.zeros_like(b)
    st = gb.mg_gcr_solve(mg.ctx, xs, b, 1e-10, 200)
    assert st["true_residual"] <= 1e-10
    mg.close()
