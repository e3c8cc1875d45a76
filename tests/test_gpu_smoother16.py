"""16-bit fine-level smoother (params.prec_smoother = MG_BF16; Sec. 7.1 runs
the finest level's MR smoother in half precision): the BF16 operator copy
against the FP64 oracle at the 16-bit tolerance, and MG solves whose fine
smoother works in BF16 reaching 1e-10 (the outer FP64 GCR keeps the
solution exact) in about as many outer iterations as the FP32 smoother.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import lattice as lat
from gpu_helpers import make_ctx, oracle_fine, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

MG_BF16 = 2


def _ctx(gb, dims, blocks, nvecs, U=None, **kw):
    if U is None:
        U = syn.gauge_field(dims, kw.pop("eps", 0.4), 3)
    p = gb.default_params(dims=dims, block=blocks, nvec=nvecs, mass=kw.get("mass", -0.2),
                          csw=1.0, nlevels=len(blocks) + 1, prec_fine=1, prec_coarse=1,
                          setup_sweeps=kw.get("sweeps", 6), prec_smoother=kw.get("ps", MG_BF16))
    return gb.Multigrid(p, to_dev(U)), U


@pytest.mark.parametrize("policy", [0, 3, 4, 6])
@pytest.mark.parametrize("unitary", [True, False])
def test_bf16_operator(gpu_lib, unitary, policy):
    """Two-row links for an SU(3) field, all nine entries otherwise; every
    register-budget policy of the kernel pinned in turn (minimum CTAs per
    SM 0, 3, 4, 6)."""
    gb = gpu_lib
    dims = (4, 4, 4, 6)
    U = syn.gauge_field(dims, 0.5, 5) * (1.0 if unitary else 1.05)
    mg, _ = _ctx(gb, dims, [(2, 2, 2, 2)], [2], U=U)
    nr = 2
    psi = syn.gaussian_field((nr, lat.volume(dims), 12), 111)
    xin = torch.from_numpy(np.stack([psi.real, psi.imag], -1)).to("cuda", torch.bfloat16)
    out = torch.empty_like(xin)
    key = f"wilson16/v{lat.volume(dims)}/n{nr}/c{int(unitary)}"
    gb.mg_tune_set(key, policy)
    try:
        gb.mg_wilson_clover_apply_bf16(mg.ctx, out, xin, nr)
        assert gb.mg_tune_get(key) == policy
    finally:
        gb.mg_tune_set(key, -1)
    o = out.float().cpu().numpy()
    got = o[..., 0] + 1j * o[..., 1]
    op = oracle_fine(U, dims)
    want = np.stack([op.apply(p) for p in psi])
    assert rel_l2(got, want) < 5e-3
    mg.close()


def test_bf16_smoother_solve(gpu_lib):
    gb = gpu_lib
    dims = (8, 8, 8, 8)
    U = syn.gauge_field(dims, 0.4, 3)
    b = to_dev(syn.gaussian_field((8 ** 4, 12), 112))
    its = {}
    for ps in (1, MG_BF16):
        mg, _ = _ctx(gb, dims, [(2, 2, 2, 2), (2, 2, 2, 2)], [16, 16], U=U, ps=ps, mass=-0.3,
                     sweeps=8)
        for l in range(2):
            gb.mg_setup_nullvecs(mg.ctx, l, None)
            gb.mg_build_coarse(mg.ctx, l)
        x = torch.zeros_like(b)
        st = gb.mg_gcr_solve(mg.ctx, x, b, 1e-10, 300)
        res = np.linalg.norm(to_np(b) - oracle_fine(U, dims, -0.3).apply(to_np(x)))
        assert res / np.linalg.norm(to_np(b)) <= 1.05e-10
        its[ps] = st["iters"]
        mg.close()
    assert its[MG_BF16] <= its[1] + 2, its


def test_bf16_smoother_needs_fp32_fine_level(gpu_lib):
    gb = gpu_lib
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, 0.3, 1)
    p = gb.default_params(dims=dims, block=[(2, 2, 2, 2)], nvec=[4], prec_fine=0,
                          prec_smoother=MG_BF16)
    with pytest.raises(gb.MGError) as e:
        gb.Multigrid(p, to_dev(U))
    assert e.value.status == gb.MG_ERR_ARG


@pytest.mark.parametrize("nv", [24, 8])
def test_bf16_prolongator_transfers(gpu_lib, nv):
    """With the 16-bit smoother the fine-level restrict / prolong read a BF16
    copy of the prolongator (the Galerkin build keeps FP32)."""
    from oracle import multigrid as mgo
    gb = gpu_lib
    dims, block = (8, 4, 4, 8), (4, 4, 4, 4)
    U = syn.gauge_field(dims, 0.4, 6)
    mg, _ = _ctx(gb, dims, [block], [nv], U=U)
    vol = lat.volume(dims)
    v = syn.gaussian_field((nv, vol, 12), 113)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    Q = mgo.block_orthonormalise(v, dims, block)
    cd = lat.coarse_dims(dims, block)
    r = syn.gaussian_field((vol, 12), 114)
    rc = torch.empty((lat.volume(cd), 2 * nv), dtype=torch.complex64, device="cuda")
    gb.mg_restrict(mg.ctx, 0, rc, to_dev(r, torch.complex64))
    ec = syn.gaussian_field((lat.volume(cd), 2 * nv), 115)
    e = torch.empty((vol, 12), dtype=torch.complex64, device="cuda")
    gb.mg_prolong(mg.ctx, 0, e, to_dev(ec, torch.complex64))
    torch.cuda.synchronize()
    assert rel_l2(to_np(rc), mgo.restrict(Q, r, dims, block)) < 5e-3
    assert rel_l2(to_np(e), mgo.prolong(Q, ec, dims, block)) < 5e-3
    mg.close()
