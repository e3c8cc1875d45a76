"""Multi-RHS MG-GCR solve (mg_gcr_solve_multi): nrhs right-hand sides per
call, every step batched over them.  Each right-hand side must reach the
tolerance on its own (true residual recomputed here with the FP64 oracle
operator), take the same number of outer steps as its single-RHS solve
(within one) and return the same solution.

Paths covered: FP32 levels (batched Wilson, per-aggregate batched
transfers, the FP32 multi-RHS coarse stream), BF16 levels (tensor-core
coarse apply through the interleaved layout), FP64 levels (per-vector coarse
applies), a zero right-hand side, and right-hand sides of very different
norms.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import lattice as lat
from gpu_helpers import make_ctx, oracle_fine, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _hierarchy(gb, dims, blocks, nvecs, pf, pc, mass=-0.2, eps=0.3, sweeps=6):
    mg, U = make_ctx(gb, dims, blocks, nvecs, prec_fine=pf, prec_coarse=pc, mass=mass, eps=eps,
                     sweeps=sweeps)
    for l in range(len(blocks)):
        gb.mg_setup_nullvecs(mg.ctx, l, None)
        gb.mg_build_coarse(mg.ctx, l)
    return mg, U


def _rhs(nr, vol, seed):
    b = syn.gaussian_field((nr, vol, 12), seed)
    b[-1] *= 1e3  # per-RHS tolerances are relative to each |b_v|
    return b


def _check_against_single(gb, mg, U, dims, b, tol=1e-10, mass=-0.2):
    nr, vol = b.shape[0], b.shape[1]
    bd = to_dev(b)
    x = torch.zeros_like(bd)
    multi = gb.mg_gcr_solve_multi(mg.ctx, x, bd, nr, tol=tol, maxiter=300)
    torch.cuda.synchronize()
    op = oracle_fine(U, dims, mass=mass)
    xs = to_np(x)
    for v in range(nr):
        xv = torch.zeros((vol, 12), dtype=torch.complex128, device="cuda")
        single = gb.mg_gcr_solve(mg.ctx, xv, bd[v].contiguous(), tol=tol, maxiter=300)
        torch.cuda.synchronize()
        if not np.any(b[v]):
            assert multi[v]["iters"] == 0 and not np.any(xs[v])
            continue
        res = np.linalg.norm(b[v] - op.apply(xs[v])) / np.linalg.norm(b[v])
        assert res <= 1.05 * tol, (v, res)
        assert multi[v]["true_residual"] <= 1.05 * tol
        assert abs(multi[v]["iters"] - single["iters"]) <= 1, (v, multi[v]["iters"],
                                                                 single["iters"])
        assert rel_l2(xs[v], to_np(xv)) < 1e-6
    return multi


@pytest.mark.parametrize("nr", [4, 3])
def test_multi_rhs_fp32_three_level(gpu_lib, nr):
    gb = gpu_lib
    dims = (8, 8, 8, 8)
    mg, U = _hierarchy(gb, dims, [(2, 2, 2, 2), (2, 2, 2, 2)], [16, 16], 1, 1)
    b = _rhs(nr, lat.volume(dims), 61)
    multi = _check_against_single(gb, mg, U, dims, b)
    assert multi[0]["level_iters"][2] > 0  # the coarsest level ran
    mg.close()


def test_multi_rhs_bf16_tensor_cores(gpu_lib):
    gb = gpu_lib
    dims = (8, 8, 8, 8)
    mg, U = _hierarchy(gb, dims, [(2, 2, 2, 2), (2, 2, 2, 2)], [16, 16], 1, 2)
    _check_against_single(gb, mg, U, dims, _rhs(4, lat.volume(dims), 62))
    mg.close()


def test_multi_rhs_fp64_two_level_with_zero_rhs(gpu_lib):
    gb = gpu_lib
    dims = (4, 4, 4, 8)
    mg, U = _hierarchy(gb, dims, [(2, 2, 2, 2)], [8], 0, 0)
    b = _rhs(3, lat.volume(dims), 63)
    b[1] = 0.0
    _check_against_single(gb, mg, U, dims, b)
    mg.close()


def test_multi_rhs_argument_errors(gpu_lib):
    gb = gpu_lib
    dims = (4, 4, 4, 4)
    mg, U = _hierarchy(gb, dims, [(2, 2, 2, 2)], [4], 1, 1)
    b = to_dev(_rhs(2, lat.volume(dims), 64))
    x = torch.zeros_like(b)
    for nr in (0, 33):
        with pytest.raises(gb.MGError) as e:
            gb.mg_gcr_solve_multi(mg.ctx, x, b, nr)
        assert e.value.status == gb.MG_ERR_ARG
    mg.close()
