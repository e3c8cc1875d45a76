"""The allocation-free block orthonormalisation entry point.

mg_block_orthonormalise_noalloc serves callers that cannot let the library
allocate device memory (their device memory belongs to another allocator, a
fixed budget, or a latency-critical loop that cannot take cudaMalloc's
implicit synchronisation).  Its workspace is a file-scope device array
shared by all calls.  These tests call it through the C ABI and compare its
output with the context-based path (mg_set_nullvecs, then mg_get_nullvecs of
the orthonormalised vectors), on two calls in a row, so that a workspace
left over from the first call cannot hide in the second.  The file is
collected last: run alone in a fresh process it also covers the first-call
set-up of the workspace address.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from gpu_helpers import make_ctx, rel_l2, to_dev, to_np
from oracle import lattice as lat, multigrid as mgo

pytestmark = pytest.mark.gpu


def _context_path(gb, dims, block, v):
    nv = v.shape[0]
    mg, _ = make_ctx(gb, dims, [block], [nv])
    gb.mg_set_nullvecs(mg.ctx, 0, to_dev(v))
    out = torch.empty(v.shape, dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, out, kind=1)
    torch.cuda.synchronize()
    got = to_np(out)
    mg.close()
    return got


@pytest.mark.parametrize("dims,block,nv", [((4, 4, 4, 4), (2, 2, 2, 2), 6),
                                           ((4, 2, 4, 6), (2, 1, 2, 3), 4)])
def test_noalloc_matches_context_path_twice(gpu_lib, dims, block, nv):
    gb = gpu_lib
    vol = lat.volume(dims)
    for call, seed in enumerate((101, 202)):
        v = syn.gaussian_field((nv, vol, 12), seed)
        want = _context_path(gb, dims, block, v)
        out = torch.full((nv, vol, 12), float("nan"), dtype=torch.complex128, device="cuda")
        gb.mg_block_orthonormalise_noalloc(to_dev(v), out, dims, block)
        torch.cuda.synchronize()
        err = rel_l2(to_np(out), want)
        assert err < 1e-12, (call, err)


@pytest.mark.parametrize("dims,block,ndof,nv", [((4, 4, 2, 2), (2, 2, 2, 2), 48, 8),
                                                ((2, 2, 2, 4), (1, 2, 2, 2), 64, 12)])
def test_noalloc_coarse_level_vectors_match_oracle_twice(gpu_lib, dims, block, ndof, nv):
    """Coarse-level vectors (ndof = 2 Nv of the level above: 48 and 64
    dofs, chirality = first / second half of the dofs) against the oracle's
    block orthonormalisation, on two calls in a row."""
    gb = gpu_lib
    vol = lat.volume(dims)
    for call, seed in enumerate((401, 402)):
        v = syn.gaussian_field((nv, vol, ndof), seed)
        want = mgo.block_orthonormalise(v, dims, block)
        out = torch.full((nv, vol, ndof), float("nan"), dtype=torch.complex128, device="cuda")
        gb.mg_block_orthonormalise_noalloc(to_dev(v), out, dims, block)
        torch.cuda.synchronize()
        err = rel_l2(to_np(out), want)
        assert err < 1e-12, (call, err)


def test_noalloc_rejects_oversize_and_reports_rank(gpu_lib):
    gb = gpu_lib
    # 2^21 complex entries is the workspace limit: 24 x 8^4 x 24 exceeds it
    big = torch.zeros((24, 8 ** 4, 24), dtype=torch.complex128, device="cuda")
    with pytest.raises(gb.MGError) as e:
        gb.mg_block_orthonormalise_noalloc(big, torch.empty_like(big), (8, 8, 8, 8), (2, 2, 2, 2))
    assert e.value.status == gb.MG_ERR_ARG and "exceeds" in str(e.value)
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    v = syn.gaussian_field((3, lat.volume(dims), 12), 303)
    v[2] = 2.0 * v[0] + 1j * v[1]
    with pytest.raises(gb.MGError) as e:
        gb.mg_block_orthonormalise_noalloc(to_dev(v), torch.empty((3, 256, 12), dtype=torch.complex128,
                                                                 device="cuda"), dims, block)
    assert e.value.status == gb.MG_ERR_RANK
    # the status word is cleared per call: a good call right after succeeds
    w = syn.gaussian_field((3, lat.volume(dims), 12), 304)
    out = torch.empty((3, 256, 12), dtype=torch.complex128, device="cuda")
    gb.mg_block_orthonormalise_noalloc(to_dev(w), out, dims, block)
    torch.cuda.synchronize()
    assert np.isfinite(to_np(out)).all()
