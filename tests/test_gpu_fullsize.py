"""Parity at the production-shaped size (32^3x64 fine lattice, 3 levels, FP32)
in the launch configuration the bench times, on outputs the oracle computes
site by site.

* fine Wilson-clover apply (autotuned policy) on sampled sites, both time
  boundaries included;
* the Galerkin-built level-1 operator (8^3x16, n = 48): its apply on sampled
  coarse sites, and Y_{-mu}(x) = g5hat Y_{+mu}(x - mu)^dag g5hat there;
* the 3-level solve: the residual b - M x recomputed by the oracle on
  sampled sites.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac, lattice as lat, multigrid as mgo

pytestmark = pytest.mark.gpu

W = syn.WORKLOADS["c2_32^3x64_3lvl_fp32"]
DIMS = tuple(W["dims"])


def _sample_sites(dims, n, seed):
    rng = np.random.default_rng(seed)
    vol = lat.volume(dims)
    sites = set(rng.integers(0, vol, n).tolist())
    stride_t = vol // dims[3]
    sites |= {0, stride_t - 1, vol - 1, vol - stride_t}  # t = 0 and t = Lt - 1 slices
    return np.array(sorted(sites))


@pytest.fixture(scope="module")
def hierarchy(gpu_lib):
    gb = gpu_lib
    U = syn.gauge_field(DIMS, W["eps"], W["seed"])
    p = gb.default_params(dims=DIMS, block=W["block"], nvec=W["nvec"], mass=W["mass"],
                          csw=W["csw"], nlevels=3, prec_fine=1, prec_coarse=1,
                          setup_sweeps=W["sweeps"], t_antiperiodic=W["antiperiodic"],
                          seed=W["seed"])
    mg = gb.Multigrid(p, torch.from_numpy(U).cuda())
    for l in range(2):
        gb.mg_setup_nullvecs(mg.ctx, l, None)
        gb.mg_build_coarse(mg.ctx, l)
    torch.cuda.synchronize()
    yield gb, mg, U
    mg.close()


def test_fine_apply_sampled(hierarchy):
    gb, mg, U = hierarchy
    vol = lat.volume(DIMS)
    psi = syn.gaussian_field((vol, 12), 101)
    out = torch.empty((vol, 12), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, torch.from_numpy(psi).to("cuda", torch.complex64))
    got = out.cpu().numpy().astype(np.complex128)
    sites = _sample_sites(DIMS, 200, 102)
    blocks = dirac.wilson_clover_blocks(U, DIMS, W["mass"], W["csw"], bool(W["antiperiodic"]),
                                        sites=sites)
    want = dirac.apply_at(blocks, psi, DIMS, sites)
    err = np.linalg.norm(got[sites] - want) / np.linalg.norm(want)
    assert err < 1e-5, err


@pytest.mark.parametrize("policy", [4, 10])
def test_fine_apply_compressed_links_sampled(hierarchy, policy):
    """Two-row (policy 4) and 8-real (policy 10) links at full size; the
    sample includes the 16 sites whose forward links are closest to a
    diagonal matrix (smallest 1 - |U_00|^2, where the 8-real rebuild divides)
    and their backward partners."""
    gb, mg, U = hierarchy
    vol = lat.volume(DIMS)
    info = gb.mg_gauge_compression(mg.ctx)
    assert info["two_row"] and info["eight_real"], info
    key = f"wilson/v{vol}/n1/c1"
    gb.mg_tune_set(key, policy)
    psi = syn.gaussian_field((vol, 12), 105)
    out = torch.empty((vol, 12), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, torch.from_numpy(psi).to("cuda", torch.complex64))
    got = out.cpu().numpy().astype(np.complex128)
    assert gb.mg_tune_get(key) == policy
    gb.mg_tune_set(key, -1)
    nrm = 1.0 - np.abs(U[:, :, 0, 0]) ** 2            # [mu][site]
    worst = np.argsort(nrm.ravel())[:16]
    mu, site = np.unravel_index(worst, nrm.shape)
    c = lat.coords(DIMS)[site]
    partner = lat.index(DIMS, c + np.eye(4, dtype=np.int64)[mu])
    sites = np.unique(np.concatenate([_sample_sites(DIMS, 100, 106), site, partner]))
    blocks = dirac.wilson_clover_blocks(U, DIMS, W["mass"], W["csw"], bool(W["antiperiodic"]),
                                        sites=sites)
    want = dirac.apply_at(blocks, psi, DIMS, sites)
    err = np.linalg.norm(got[sites] - want) / np.linalg.norm(want)
    assert err < 1e-5, (policy, err, info)


def test_level1_apply_and_backward_links_sampled(hierarchy):
    gb, mg, U = hierarchy
    lv = mg.levels[1]
    cdims, n, vol = tuple(lv["dims"]), lv["ndof"], lv["volume"]
    assert cdims == (8, 8, 8, 16) and n == 48
    links = torch.empty((vol, 9, n, n), dtype=torch.complex128, device="cuda")
    gb.mg_get_coarse_links(mg.ctx, 1, links)
    L = links.cpu().numpy()
    del links
    x = syn.gaussian_field((vol, n), 103)
    y = torch.empty((vol, n), dtype=torch.complex64, device="cuda")
    gb.mg_coarse_apply(mg.ctx, 1, y, torch.from_numpy(x).to("cuda", torch.complex64))
    got = y.cpu().numpy().astype(np.complex128)
    sites = _sample_sites(cdims, 96, 104)
    want = dirac.apply_at(L[sites], x, cdims, sites)
    err = np.linalg.norm(got[sites] - want) / np.linalg.norm(want)
    assert err < 1e-5, err
    # Eq. (3) backward blocks from the forward ones of the -mu neighbour
    g5 = mgo.gamma5_hat(n)
    c = lat.coords(cdims)[sites]
    for mu in range(4):
        back = lat.index(cdims, c - np.eye(4, dtype=int)[mu])
        yp = L[back, 1 + 2 * mu]
        rel = g5[None, :, None] * np.conj(np.swapaxes(yp, 1, 2)) * g5[None, None, :]
        d = np.abs(L[sites, 2 + 2 * mu] - rel).max() / np.abs(rel).max()
        assert d < 1e-5, (mu, d)


def test_solve_residual_sampled(hierarchy):
    gb, mg, U = hierarchy
    vol = lat.volume(DIMS)
    b = syn.gaussian_field((vol, 12), W["seed"], stream=99)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st = gb.mg_gcr_solve(mg.ctx, x, bd, 1e-10, 500)
    assert st["true_residual"] <= 1e-10
    xs = x.cpu().numpy()
    sites = _sample_sites(DIMS, 400, 105)
    blocks = dirac.wilson_clover_blocks(U, DIMS, W["mass"], W["csw"], bool(W["antiperiodic"]),
                                        sites=sites)
    r = b[sites] - dirac.apply_at(blocks, xs, DIMS, sites)
    assert np.linalg.norm(r) / np.linalg.norm(b[sites]) < 1e-9


def _exact_dot(a, b):
    """sum conj(a) b for vectors whose parts are FP32 values: every product
    is exact in float64, and numpy's pairwise float64 sum adds an error of
    about log2(N) 2^-53 of sum |terms|.  Returns the value and, per part,
    sum |terms| (the scale any summation error is measured against)."""
    ar, ai = a.real.astype(np.float64).ravel(), a.imag.astype(np.float64).ravel()
    br, bi = b.real.astype(np.float64).ravel(), b.imag.astype(np.float64).ravel()
    re = np.concatenate([ar * br, ai * bi])
    im = np.concatenate([ar * bi, -(ai * br)])
    return complex(np.sum(re), np.sum(im)), np.sum(np.abs(re)), np.sum(np.abs(im))


def test_outer_inner_products_are_fp64_accurate(hierarchy):
    """The outer GCR's inner products (Sec. 7.1) on FP32 vectors of the full
    fine lattice (25.2 M complex numbers, the bench's launch configuration):
    within 1e-12 of sum |terms| of the exact value, a bound that products
    rounded to FP32 (about 2^-24 / sqrt(N) of it) would miss; b is x's
    complement so that the result cancels to ~1e-4 of the scale.  The same
    holds for FP64 vectors with FP32-representable parts, and the inner
    levels' FP32 form stays within 1e-5."""
    gb, mg, U = hierarchy
    vol = lat.volume(DIMS)
    rng = np.random.default_rng(106)
    x = (rng.standard_normal((vol, 12)) + 1j * rng.standard_normal((vol, 12))).astype(np.complex64)
    z = (rng.standard_normal((vol, 12)) + 1j * rng.standard_normal((vol, 12))).astype(np.complex64)
    xd = x.astype(np.complex128)
    zd = z.astype(np.complex128)
    y = (zd - (np.vdot(xd, zd) / np.vdot(xd, xd)) * xd).astype(np.complex64)
    del xd, zd, z
    want, s_re, s_im = _exact_dot(x, y)
    assert abs(want) < 1e-3 * (s_re + s_im)  # the sum really cancels
    nrm, s_nrm, _ = _exact_dot(x, x)
    xg, yg = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for dt in (torch.complex64, torch.complex128):
        a, b = xg.to(dt), yg.to(dt)
        got = gb.mg_inner_product(mg.ctx, 0, a, b, fp64=True)
        assert abs(got.real - want.real) <= 1e-12 * s_re, (dt, got, want)
        assert abs(got.imag - want.imag) <= 1e-12 * s_im, (dt, got, want)
        got = gb.mg_inner_product(mg.ctx, 0, a, a, fp64=True)
        assert abs(got.real - nrm.real) <= 1e-12 * s_nrm and got.imag == 0.0, (dt, got, nrm)
    got = gb.mg_inner_product(mg.ctx, 0, xg, yg, fp64=False)
    assert abs(got.real - want.real) <= 1e-5 * s_re and abs(got.imag - want.imag) <= 1e-5 * s_im
    # a NaN anywhere reaches the result (the solvers' breakdown check)
    xg[vol // 3, 5] = complex("nan")
    got = gb.mg_inner_product(mg.ctx, 0, xg, yg, fp64=True)
    assert not np.isfinite(got.real)
