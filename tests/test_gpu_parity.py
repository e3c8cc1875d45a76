"""GPU parity: every kernel of the hot path against the FP64 CPU oracle on
the same seeded inputs, through the C ABI.

Tolerances (relative L2 error against the FP64 oracle): 1e-12 for FP64
kernels, 1e-5 for FP32, 5e-3 for 16-bit link storage.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac, lattice as lat, multigrid as mgo, solvers
from gpu_helpers import make_ctx, oracle_fine, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 5e-3, 3: 5e-3, 4: 5e-3}


# ------------------------------------------------------------------ Eq. (2)
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("prec", [0, 1])
def test_wilson_clover_apply(gpu_lib, dims, prec):
    gb = gpu_lib
    blk = tuple(2 if d % 2 == 0 else 1 for d in dims)
    mg, U = make_ctx(gb, dims, [blk], [2], prec_fine=prec, prec_coarse=prec, csw=1.3,
                     mass=-0.15, eps=0.4)
    op = oracle_fine(U, dims, -0.15, 1.3)
    psi = syn.gaussian_field((lat.volume(dims), 12), 5)
    dt = torch.complex128 if prec == 0 else torch.complex64
    out = torch.empty((lat.volume(dims), 12), dtype=dt, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, to_dev(psi, dt))
    torch.cuda.synchronize()
    err = rel_l2(to_np(out), op.apply(psi))
    assert err < TOL[prec], err
    mg.close()


def test_wilson_clover_periodic_boundary(gpu_lib):
    gb = gpu_lib
    dims = (4, 2, 2, 4)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], antiperiodic=0, mass=0.1)
    op = dirac.wilson_clover_op(U, dims, 0.1, 1.0, antiperiodic=False)
    psi = syn.gaussian_field((lat.volume(dims), 12), 6)
    out = torch.empty((lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, to_dev(psi))
    torch.cuda.synchronize()
    assert rel_l2(to_np(out), op.apply(psi)) < 1e-12
    mg.close()


# ------------------------------------------------------------------ Eq. (3)
def _random_links(vol, n, seed):
    return syn.gaussian_field((vol, 9, n, n), seed) / np.sqrt(n)


@pytest.mark.parametrize("cdims,nv", [((2, 2, 2, 2), 8), ((4, 4, 4, 4), 24), ((2, 4, 2, 4), 32),
                                      ((3, 2, 2, 2), 3), ((2, 2, 2, 2), 5), ((4, 2, 2, 2), 16)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_coarse_apply_random_links(gpu_lib, cdims, nv, prec):
    """Coarse links set from the host (random), y = sum_slot L x(nbr) against
    the oracle stencil apply.  Covers the streaming kernel (n = 16, 48, 64)
    and the generic kernel (n = 6, 10, 32-with-odd-extent)."""
    gb = gpu_lib
    if prec >= 2 and (2 * nv) % 4:
        pytest.skip("16-bit links need n % 4 == 0")
    dims = tuple(c * 2 for c in cdims)
    prec_fine = 0 if prec == 0 else 1
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], prec_fine=prec_fine, prec_coarse=prec)
    n = 2 * nv
    vol = lat.volume(cdims)
    links = _random_links(vol, n, 11)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    cop = dirac.StencilOp(cdims, links)
    x = syn.gaussian_field((vol, n), 12)
    dt = torch.complex128 if prec == 0 else torch.complex64
    y = torch.empty((vol, n), dtype=dt, device="cuda")
    gb.mg_coarse_apply(mg.ctx, 1, y, to_dev(x, dt))
    torch.cuda.synchronize()
    err = rel_l2(to_np(y), cop.apply(x))
    assert err < TOL[prec], err
    # round trip of the link store
    back = torch.empty((vol, 9, n, n), dtype=torch.complex128, device="cuda")
    gb.mg_get_coarse_links(mg.ctx, 1, back)
    torch.cuda.synchronize()
    assert rel_l2(to_np(back), links) < (1e-15 if prec == 0 else TOL[prec])
    mg.close()


@pytest.mark.parametrize("cdims,nv,nrhs", [
    ((2, 2, 4, 2), 24, 2), ((2, 2, 4, 2), 24, 8), ((2, 2, 4, 2), 24, 12),  # NR 2, 8, 4 x 3
    ((3, 2, 2, 4), 16, 16), ((2, 2, 2, 2), 32, 6), ((2, 2, 2, 2), 8, 4),    # n 32, 64, 16
    ((2, 2, 4, 2), 24, 3)])                                                 # odd: generic
def test_coarse_apply_multi_rhs(gpu_lib, cdims, nv, nrhs):
    """FP32 multi-RHS apply, [site][n][nrhs] layout: the FP32 multi-RHS stream
    for even nrhs (chunks of 8, 4 or 2 right-hand sides per CTA), the generic
    kernel for odd nrhs."""
    gb = gpu_lib
    dims = tuple(c * 2 for c in cdims)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], prec_fine=1, prec_coarse=1)
    n, vol = 2 * nv, lat.volume(cdims)
    links = _random_links(vol, n, 13)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = syn.gaussian_field((vol, n, nrhs), 14)
    y = torch.empty((vol, n, nrhs), dtype=torch.complex64, device="cuda")
    gb.mg_coarse_apply(mg.ctx, 1, y, to_dev(x, torch.complex64), nrhs=nrhs)
    torch.cuda.synchronize()
    cop = dirac.StencilOp(cdims, links)
    want = np.stack([cop.apply(x[:, :, k]) for k in range(nrhs)], axis=-1)
    assert rel_l2(to_np(y), want) < 1e-5
    mg.close()


@pytest.mark.parametrize("cdims,nv,nrhs", [((4, 4, 2, 4), 24, 8), ((2, 2, 4, 2), 16, 16),
                                           ((2, 4, 2, 2), 32, 8)])
def test_coarse_apply_multi_rhs_every_load_batch(gpu_lib, cdims, nv, nrhs):
    """The FP32 multi-RHS stream at 8 right-hand sides per link read, every
    load batch the autotuner offers pinned in turn (choice = the cap on the
    16-byte link loads a thread keeps in flight)."""
    gb = gpu_lib
    dims = tuple(c * 2 for c in cdims)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], prec_fine=1, prec_coarse=1)
    n, vol = 2 * nv, lat.volume(cdims)
    links = _random_links(vol, n, 15)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = syn.gaussian_field((vol, n, nrhs), 16)
    xd = to_dev(x, torch.complex64)
    y = torch.empty((vol, n, nrhs), dtype=torch.complex64, device="cuda")
    cop = dirac.StencilOp(cdims, links)
    want = np.stack([cop.apply(x[:, :, k]) for k in range(nrhs)], axis=-1)
    key = f"stream_mr/p1/n{n}/v{vol}/r{nrhs}/b0"
    gb.mg_tune_set(key, -1)
    gb.mg_coarse_apply(mg.ctx, 1, y, xd, nrhs=nrhs)  # tunes: times every candidate
    choices = [c for c, _ in gb.mg_tune_report(key)]
    assert 4 in choices and len(choices) >= 2, choices
    for choice in choices:
        gb.mg_tune_set(key, choice)
        y.fill_(float("nan"))
        gb.mg_coarse_apply(mg.ctx, 1, y, xd, nrhs=nrhs)
        torch.cuda.synchronize()
        assert gb.mg_tune_get(key) == choice
        assert rel_l2(to_np(y), want) < 1e-5, choice
    gb.mg_tune_set(key, -1)
    mg.close()


# ------------------------------------------------------------------ setup
@pytest.mark.parametrize("dims,block,nv", [((4, 4, 4, 4), (2, 2, 2, 2), 6),
                                           ((4, 2, 4, 6), (2, 1, 2, 3), 4)])
def test_block_orthonormalise(gpu_lib, dims, block, nv):
    gb = gpu_lib
    mg, U = make_ctx(gb, dims, [block], [nv])
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 21)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    out = torch.empty((nv, lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, out, kind=1)
    torch.cuda.synchronize()
    assert rel_l2(to_np(out), mgo.block_orthonormalise(v, dims, block)) < 1e-12
    mg.close()


def test_block_orthonormalise_nearly_parallel_columns(gpu_lib):
    """Columns that differ by 1e-3 relative: the first projection removes
    almost all of their norm, so the second pass runs (and must)."""
    gb = gpu_lib
    dims, block, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    mg, U = make_ctx(gb, dims, [block], [nv])
    base = syn.gaussian_field((1, lat.volume(dims), 12), 28)
    v = base + 1e-3 * syn.gaussian_field((nv, lat.volume(dims), 12), 29)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    out = torch.empty((nv, lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, out, kind=1)
    torch.cuda.synchronize()
    assert rel_l2(to_np(out), mgo.block_orthonormalise(v, dims, block)) < 1e-12
    mg.close()


def test_rank_deficient_block_is_reported(gpu_lib):
    gb = gpu_lib
    dims, nv = (4, 4, 4, 4), 3
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv])
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 22)
    v[2] = 0.5 * v[0] - 2j * v[1]
    with pytest.raises(gb.MGError) as e:
        gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    assert e.value.status == gb.MG_ERR_RANK
    mg.close()


def test_setup_sweeps_fp64(gpu_lib):
    gb = gpu_lib
    dims, nv, sweeps = (4, 4, 4, 4), 4, 5
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], sweeps=sweeps)
    x0 = syn.gaussian_field((nv, lat.volume(dims), 12), 23)
    gb.mg_setup_nullvecs(mg.ctx, 0, to_dev(x0))
    raw = torch.empty((nv, lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, raw, kind=0)
    torch.cuda.synchronize()
    want = mgo.null_vectors(oracle_fine(U, dims), x0, sweeps)
    assert rel_l2(to_np(raw), want) < 1e-12
    mg.close()


@pytest.mark.parametrize("nv", [4, 6])
def test_setup_sweeps_fp32(gpu_lib, nv):
    """FP32 fine-level sweeps run the batched Wilson kernel (NB = 4, 2 or 1
    vectors per thread, as the autotuner picks) on all vectors at once."""
    gb = gpu_lib
    dims, sweeps = (4, 4, 4, 8), 3
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], sweeps=sweeps, prec_fine=1, prec_coarse=1)
    x0 = syn.gaussian_field((nv, lat.volume(dims), 12), 27)
    gb.mg_setup_nullvecs(mg.ctx, 0, to_dev(x0))
    raw = torch.empty((nv, lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, raw, kind=0)
    torch.cuda.synchronize()
    want = mgo.null_vectors(oracle_fine(U, dims), x0, sweeps)
    err = rel_l2(to_np(raw), want)
    assert err < 1e-5, err
    mg.close()


@pytest.mark.parametrize("nv2", [8, 6])
def test_setup_sweeps_coarse_fp32(gpu_lib, nv2):
    """FP32 coarse-level sweeps apply the level-1 operator to all vectors at
    once through the FP32 multi-RHS stream; checked against the oracle's sweeps
    on the same (GPU-built, exported) coarse operator."""
    gb = gpu_lib
    dims, b1, b2, nv1, sweeps = (8, 4, 4, 8), (2, 2, 2, 2), (2, 1, 1, 2), 16, 3
    mg, U = make_ctx(gb, dims, [b1, b2], [nv1, nv2], prec_fine=1, prec_coarse=1, sweeps=sweeps)
    v1 = syn.gaussian_field((nv1, lat.volume(dims), 12), 43)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v1))
    gb.mg_build_coarse(mg.ctx, 0)
    cd1 = lat.coarse_dims(dims, b1)
    n1, vol1 = 2 * nv1, lat.volume(cd1)
    links = torch.empty((vol1, 9, n1, n1), dtype=torch.complex128, device="cuda")
    gb.mg_get_coarse_links(mg.ctx, 1, links)
    x0 = syn.gaussian_field((nv2, vol1, n1), 44)
    gb.mg_setup_nullvecs(mg.ctx, 1, to_dev(x0))
    raw = torch.empty((nv2, vol1, n1), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 1, raw, kind=0)
    torch.cuda.synchronize()
    want = mgo.null_vectors(dirac.StencilOp(cd1, to_np(links)), x0, sweeps)
    err = rel_l2(to_np(raw), want)
    assert err < 1e-5, err
    mg.close()


# ------------------------------------------------------------------ transfer
@pytest.mark.parametrize("dims,block,nv", [((4, 4, 2, 6), (2, 2, 2, 3), 5),
                                           ((4, 4, 4, 4), (2, 2, 2, 2), 8),
                                           ((8, 4, 4, 8), (4, 4, 4, 4), 24)])
@pytest.mark.parametrize("prec", [0, 1])
def test_restrict_prolong(gpu_lib, dims, block, nv, prec):
    """Fine-level transfers: per-aggregate vector kernels (even Nv in FP32,
    any Nv in FP64 restrict) and the generic ones (odd Nv)."""
    gb = gpu_lib
    mg, U = make_ctx(gb, dims, [block], [nv], prec_fine=prec, prec_coarse=prec)
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 24)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    Q = mgo.block_orthonormalise(v, dims, block)
    cd = lat.coarse_dims(dims, block)
    dt = torch.complex128 if prec == 0 else torch.complex64
    r = syn.gaussian_field((lat.volume(dims), 12), 25)
    rc = torch.empty((lat.volume(cd), 2 * nv), dtype=dt, device="cuda")
    gb.mg_restrict(mg.ctx, 0, rc, to_dev(r, dt))
    ec = syn.gaussian_field((lat.volume(cd), 2 * nv), 26)
    e = torch.empty((lat.volume(dims), 12), dtype=dt, device="cuda")
    gb.mg_prolong(mg.ctx, 0, e, to_dev(ec, dt))
    torch.cuda.synchronize()
    assert rel_l2(to_np(rc), mgo.restrict(Q, r, dims, block)) < TOL[prec]
    assert rel_l2(to_np(e), mgo.prolong(Q, ec, dims, block)) < TOL[prec]
    mg.close()


# ------------------------------------------------------------------ Galerkin
@pytest.mark.parametrize("dims,block,nv,prec", [
    ((4, 4, 4, 4), (2, 2, 2, 2), 6, 0),     # coarse extent 2: +mu and -mu partners coincide
    ((6, 4, 2, 4), (2, 2, 2, 2), 4, 0),     # coarse extent 3 and 1
    ((8, 8, 8, 8), (2, 2, 2, 2), 24, 0),    # the small 2-level workload shape
    ((8, 8, 8, 8), (2, 2, 2, 2), 24, 1),
    ((8, 4, 4, 8), (4, 4, 4, 4), 8, 1),     # 4^4 aggregates
])
def test_galerkin_fine_to_coarse(gpu_lib, dims, block, nv, prec):
    gb = gpu_lib
    mg, U = make_ctx(gb, dims, [block], [nv], prec_fine=prec, prec_coarse=prec)
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 31)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    gb.mg_build_coarse(mg.ctx, 0)
    cd = lat.coarse_dims(dims, block)
    n = 2 * nv
    got = torch.empty((lat.volume(cd), 9, n, n), dtype=torch.complex128, device="cuda")
    gb.mg_get_coarse_links(mg.ctx, 1, got)
    torch.cuda.synchronize()
    Q = mgo.block_orthonormalise(v, dims, block)
    want = mgo.galerkin(oracle_fine(U, dims), Q, block).blocks
    err = rel_l2(to_np(got), want)
    assert err < TOL[prec], err
    mg.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nv1,nv2,b2", [
    (6, 8, (2, 1, 1, 2)),    # n2 = 16: one fine site per pass
    (6, 16, (2, 1, 1, 2)),   # n2 = 32: chunked, T products in 4 x 4 register tiles
    (6, 24, (2, 2, 2, 2)),   # n2 = 48
    (6, 32, (2, 2, 2, 2)),   # n2 = 64 (the shape of the 3-level workload's level 2)
    (5, 16, (2, 1, 1, 2)),   # chunked, 10 dof per coarse site: one T entry per thread
])
def test_galerkin_coarse_to_coarser(gpu_lib, prec, nv1, nv2, b2):
    """Level 1 -> 2: the Galerkin product of a coarse operator (dense links).
    The GPU's level-2 links are P2^dag (A1 + dA1) P2 + R2, with dA1 the
    level-1 error (at most TOL |A1|, the bound of the fine-to-coarse test)
    and R2 the level-2 build's own rounding; P2 has orthonormal columns, so
    |dA2| / |A2| <= TOL (1 + |A1| / |A2|) in the Frobenius norm of the link
    blocks (the ratio is 1.74 for the first case)."""
    gb = gpu_lib
    dims, b1 = (8, 4, 4, 8), (2, 2, 2, 2)
    mg, U = make_ctx(gb, dims, [b1, b2], [nv1, nv2], prec_fine=prec, prec_coarse=prec)
    v1 = syn.gaussian_field((nv1, lat.volume(dims), 12), 41)
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v1))
    gb.mg_build_coarse(mg.ctx, 0)
    cd1 = lat.coarse_dims(dims, b1)
    v2 = syn.gaussian_field((nv2, lat.volume(cd1), 2 * nv1), 42)
    gb.mg_set_nullvecs(mg.ctx, 1, to_dev(v2))
    gb.mg_build_coarse(mg.ctx, 1)
    cd2 = lat.coarse_dims(cd1, b2)
    n2 = 2 * nv2
    got = torch.empty((lat.volume(cd2), 9, n2, n2), dtype=torch.complex128, device="cuda")
    gb.mg_get_coarse_links(mg.ctx, 2, got)
    torch.cuda.synchronize()
    op1 = mgo.galerkin(oracle_fine(U, dims), mgo.block_orthonormalise(v1, dims, b1), b1)
    want = mgo.galerkin(op1, mgo.block_orthonormalise(v2, cd1, b2), b2).blocks
    err = rel_l2(to_np(got), want)
    bound = TOL[prec] * (1.0 + np.linalg.norm(op1.blocks) / np.linalg.norm(want))
    assert err < bound, (err, bound)
    mg.close()


# ------------------------------------------------------------------ solver
@pytest.mark.slow
def test_two_level_solve_matches_oracle_fp64(gpu_lib):
    """Small 2-level FP64 workload: identical outer iteration count and
    residual history within 1e-6 relative (the GPU orthogonalises by block
    Gram-Schmidt and reuses the smoother's residual, the oracle by modified
    Gram-Schmidt with a recomputed residual), true residual <= 1e-10."""
    gb = gpu_lib
    w = syn.WORKLOADS["c1_8^4_2lvl_fp64"]
    dims, block, nv = w["dims"], w["block"][0], w["nvec"][0]
    mg, U = make_ctx(gb, dims, [block], [nv], mass=w["mass"], csw=w["csw"], eps=w["eps"],
                     seed=w["seed"], sweeps=w["sweeps"])
    vol = lat.volume(dims)
    x0 = syn.gaussian_field((nv, vol, 12), w["seed"], stream=10)
    gb.mg_setup_nullvecs(mg.ctx, 0, to_dev(x0))
    gb.mg_build_coarse(mg.ctx, 0)
    b = syn.gaussian_field((vol, 12), w["seed"], stream=99)
    x = torch.zeros((vol, 12), dtype=torch.complex128, device="cuda")
    st = gb.mg_gcr_solve(mg.ctx, x, to_dev(b), 1e-10, 100)
    op = oracle_fine(U, dims, w["mass"], w["csw"])
    hier = solvers.MultigridHierarchy.build(op, [x0], w["sweeps"], [block])
    ref = hier.solve(b, 1e-10, 100)
    assert st["iters"] == ref.iters
    h = np.array(st["history"])
    assert np.abs(h - np.array(ref.history)).max() / np.array(ref.history).min() < 1e-6
    assert st["true_residual"] <= 1e-10
    assert rel_l2(to_np(x), ref.x) < 1e-9
    mg.close()


def test_three_level_solve_fp32_converges(gpu_lib):
    gb = gpu_lib
    dims = (8, 8, 8, 16)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], prec_fine=1,
                     prec_coarse=1, eps=0.4, mass=-0.3, sweeps=10)
    vol = lat.volume(dims)
    gb.mg_setup_nullvecs(mg.ctx, 0, None)
    gb.mg_build_coarse(mg.ctx, 0)
    gb.mg_setup_nullvecs(mg.ctx, 1, None)
    gb.mg_build_coarse(mg.ctx, 1)
    b = syn.gaussian_field((vol, 12), 77)
    x = torch.zeros((vol, 12), dtype=torch.complex128, device="cuda")
    st = gb.mg_gcr_solve(mg.ctx, x, to_dev(b), 1e-10, 200)
    assert st["true_residual"] <= 1e-10
    # independent check of the returned solution with the oracle operator
    r = b - oracle_fine(U, dims, -0.3, 1.0).apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-10
    mg.close()


def test_solver_reports_maxiter(gpu_lib):
    gb = gpu_lib
    dims = (4, 4, 4, 4)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [4])
    gb.mg_setup_nullvecs(mg.ctx, 0, None)
    gb.mg_build_coarse(mg.ctx, 0)
    b = to_dev(syn.gaussian_field((lat.volume(dims), 12), 78))
    x = torch.zeros_like(b)
    st = gb.mg_gcr_solve(mg.ctx, x, b, 1e-14, 2, check=False)
    assert st["status"] == gb.MG_ERR_NOT_CONVERGED and st["iters"] == 2
    mg.close()


def test_call_order_and_argument_errors(gpu_lib):
    gb = gpu_lib
    dims = (4, 4, 4, 4)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [4])
    y = torch.zeros((16, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.MGError) as e:
        gb.mg_coarse_apply(mg.ctx, 1, y, y.clone())
    assert e.value.status == gb.MG_ERR_STATE
    with pytest.raises(gb.MGError) as e:
        gb.mg_coarse_apply(mg.ctx, 1, y, y)
    assert e.value.status == gb.MG_ERR_ARG
    with pytest.raises(gb.MGError) as e:
        gb.mg_build_coarse(mg.ctx, 0)
    assert e.value.status == gb.MG_ERR_STATE
    mg.close()
    p = gb.default_params(dims=(6, 4, 4, 4), block=[(4, 2, 2, 2)], nvec=[4])
    with pytest.raises(gb.MGError) as e:
        gb.mg_create(p, to_dev(syn.gauge_field((6, 4, 4, 4), 0.1, 1)))
    assert e.value.status == gb.MG_ERR_ARG
