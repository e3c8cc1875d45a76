"""Every launch policy of the FP32 fine operator against the FP64 oracle.

The autotuner picks one policy per shape; here each policy is pinned in turn
through mg_tune_set: stored 18-real links or two-row links rebuilt in
registers (third row = conj(row0 x row1) times the boundary sign), 8-real
links (a2, a3, b1 and two phases, the rest rebuilt from unitarity and
det U = 1, the boundary sign applied to the whole link), register budgets, and, in the batched form used by the setup sweeps and the
multi-RHS solve, 2 or 4 vectors per thread or the operator of 32 sites staged
in shared memory for all vectors.  A field that is not special unitary must never take the
two-row form.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import dirac, lattice as lat, multigrid as mgo
from gpu_helpers import make_ctx, oracle_fine, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

SINGLE = [0, 1, 2, 3, 4, 5, 10, 11]   # 1 vector per thread: (link form, register budget)
BATCHED = [6, 7, 8, 9]        # 2 or 4 vectors per thread; shared-memory operator tile


@pytest.mark.parametrize("antiperiodic", [1, 0])
@pytest.mark.parametrize("policy", SINGLE)
def test_single_vector_policy(gpu_lib, policy, antiperiodic):
    gb = gpu_lib
    dims = (4, 6, 4, 8)
    vol = lat.volume(dims)
    gb.mg_tune_set(f"wilson/v{vol}/n1/c1", policy)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=1, prec_coarse=1,
                     antiperiodic=antiperiodic, eps=0.5)
    psi = syn.gaussian_field((vol, 12), 71)
    out = torch.empty((vol, 12), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, to_dev(psi, torch.complex64))
    torch.cuda.synchronize()
    assert gb.mg_tune_get(f"wilson/v{vol}/n1/c1") == policy
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, antiperiodic=bool(antiperiodic))
    err = rel_l2(to_np(out), op.apply(psi))
    assert err < 1e-5, (policy, err)
    gb.mg_tune_set(f"wilson/v{vol}/n1/c1", -1)
    mg.close()


@pytest.mark.parametrize("policy", BATCHED + [1])
def test_batched_policy_in_setup(gpu_lib, policy):
    gb = gpu_lib
    dims, nv, sweeps = (4, 4, 4, 8), 4, 3
    vol = lat.volume(dims)
    gb.mg_tune_set(f"wilson/v{vol}/n{nv}/c1", policy)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], sweeps=sweeps, prec_fine=1,
                     prec_coarse=1)
    x0 = syn.gaussian_field((nv, vol, 12), 72)
    gb.mg_setup_nullvecs(mg.ctx, 0, to_dev(x0))
    raw = torch.empty((nv, vol, 12), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, raw, kind=0)
    torch.cuda.synchronize()
    assert gb.mg_tune_get(f"wilson/v{vol}/n{nv}/c1") == policy
    err = rel_l2(to_np(raw), mgo.null_vectors(oracle_fine(U, dims), x0, sweeps))
    assert err < 1e-5, (policy, err)
    gb.mg_tune_set(f"wilson/v{vol}/n{nv}/c1", -1)
    mg.close()


@pytest.mark.parametrize("eps", [0.3, 0.5, 0.9])
def test_eight_real_reconstruction_error_is_stated(gpu_lib, eps):
    """The 8-real form is eligible on these fields: its FP32 rebuild
    deviates from the FP64 links by a root-mean-square of FP32 rounding size
    and by at most 1e-3 anywhere; the operator built from it meets the FP32
    tier against the oracle."""
    gb = gpu_lib
    dims = (8, 4, 6, 8)
    vol = lat.volume(dims)
    key = f"wilson/v{vol}/n1/c1"
    gb.mg_tune_set(key, 10)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=1, prec_coarse=1, eps=eps)
    info = gb.mg_gauge_compression(mg.ctx)
    assert info["two_row"] and info["eight_real"], info
    assert info["max_dev8"] < 1e-3 and info["rms_dev8"] < 1e-6, info
    psi = syn.gaussian_field((vol, 12), 75)
    out = torch.empty((vol, 12), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, to_dev(psi, torch.complex64))
    torch.cuda.synchronize()
    assert gb.mg_tune_get(key) == 10
    err = rel_l2(to_np(out), oracle_fine(U, dims).apply(psi))
    assert err < 1e-5, err
    gb.mg_tune_set(key, -1)
    mg.close()


def test_non_unitary_field_keeps_stored_links(gpu_lib):
    """Links scaled off SU(3): neither the two-row nor the 8-real form is
    eligible (key suffix c0) and a pinned two-row policy is ignored."""
    gb = gpu_lib
    dims = (4, 4, 6, 4)
    vol = lat.volume(dims)
    U = syn.gauge_field(dims, 0.4, 5) * 1.05
    gb.mg_tune_set(f"wilson/v{vol}/n1/c0", 3)  # a two-row policy: not a candidate here
    mg, _ = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=1, prec_coarse=1, U=U)
    info = gb.mg_gauge_compression(mg.ctx)
    assert not info["two_row"] and not info["eight_real"], info
    psi = syn.gaussian_field((vol, 12), 73)
    out = torch.empty((vol, 12), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, to_dev(psi, torch.complex64))
    torch.cuda.synchronize()
    assert gb.mg_tune_get(f"wilson/v{vol}/n1/c0") in (0, 2)
    err = rel_l2(to_np(out), oracle_fine(U, dims).apply(psi))
    assert err < 1e-5, err
    gb.mg_tune_set(f"wilson/v{vol}/n1/c0", -1)
    mg.close()


@pytest.mark.parametrize("nrhs", [3, 8])
def test_apply_multi(gpu_lib, nrhs):
    """mg_wilson_clover_apply_multi: nrhs vectors back to back, one launch."""
    gb = gpu_lib
    dims = (4, 4, 6, 4)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=1, prec_coarse=1, eps=0.5)
    psi = syn.gaussian_field((nrhs, lat.volume(dims), 12), 74)
    out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply_multi(mg.ctx, out, to_dev(psi, torch.complex64), nrhs)
    torch.cuda.synchronize()
    op = oracle_fine(U, dims)
    err = rel_l2(to_np(out), np.stack([op.apply(p) for p in psi]))
    assert err < 1e-5, err
    with pytest.raises(gb.MGError):
        gb.mg_wilson_clover_apply_multi(mg.ctx, out, out, nrhs)
    mg.close()


TILED = [12, 13]   # 4x4x4x2 / 4x4x2x2 block, its halo staged by tensor copies


@pytest.mark.parametrize("antiperiodic", [1, 0])
@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (8, 4, 4, 6), (4, 8, 8, 4)])
@pytest.mark.parametrize("policy", TILED)
def test_tiled_policy(gpu_lib, policy, dims, antiperiodic):
    """The block-tiled operator: every site of a block reads its neighbours
    from the shared-memory tile (block interior plus one-site faces copied
    at wrapped coordinates) -- lattices whose extent equals the block's
    (the faces wrap onto the block itself) and several blocks per extent;
    both time boundaries."""
    gb = gpu_lib
    vol = lat.volume(dims)
    key = f"wilson/v{vol}/n1/c1"
    gb.mg_tune_set(key, policy)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=1, prec_coarse=1,
                     antiperiodic=antiperiodic, eps=0.5)
    psi = syn.gaussian_field((vol, 12), 76)
    out = torch.full((vol, 12), float("nan"), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply(mg.ctx, out, to_dev(psi, torch.complex64))
    gb.mg_device_status(mg.ctx)
    assert gb.mg_tune_get(key) == policy
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, antiperiodic=bool(antiperiodic))
    err = rel_l2(to_np(out), op.apply(psi))
    assert err < 1e-5, (policy, err)
    gb.mg_tune_set(key, -1)
    mg.close()


@pytest.mark.parametrize("nrhs", [3, 8])
@pytest.mark.parametrize("policy", TILED)
def test_tiled_policy_many_vectors(gpu_lib, policy, nrhs):
    """Several vectors in one tiled launch: the links stay in shared memory,
    the spinor tile is copied again for every vector (the copies of vector
    v + 1 wait until every thread has finished with vector v)."""
    gb = gpu_lib
    dims = (8, 4, 4, 6)
    vol = lat.volume(dims)
    key = f"wilson/v{vol}/n{nrhs}/c1"
    gb.mg_tune_set(key, policy)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [2], prec_fine=1, prec_coarse=1, eps=0.5)
    psi = syn.gaussian_field((nrhs, vol, 12), 77)
    out = torch.full(psi.shape, float("nan"), dtype=torch.complex64, device="cuda")
    gb.mg_wilson_clover_apply_multi(mg.ctx, out, to_dev(psi, torch.complex64), nrhs)
    gb.mg_device_status(mg.ctx)
    assert gb.mg_tune_get(key) == policy
    op = oracle_fine(U, dims)
    err = rel_l2(to_np(out), np.stack([op.apply(p) for p in psi]))
    assert err < 1e-5, (policy, err)
    gb.mg_tune_set(key, -1)
    mg.close()


@pytest.mark.parametrize("policy", TILED)
def test_tiled_policy_in_setup(gpu_lib, policy):
    gb = gpu_lib
    dims, nv, sweeps = (4, 4, 4, 8), 4, 3
    vol = lat.volume(dims)
    gb.mg_tune_set(f"wilson/v{vol}/n{nv}/c1", policy)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], sweeps=sweeps, prec_fine=1,
                     prec_coarse=1)
    x0 = syn.gaussian_field((nv, vol, 12), 78)
    gb.mg_setup_nullvecs(mg.ctx, 0, to_dev(x0))
    raw = torch.empty((nv, vol, 12), dtype=torch.complex128, device="cuda")
    gb.mg_get_nullvecs(mg.ctx, 0, raw, kind=0)
    gb.mg_device_status(mg.ctx)
    assert gb.mg_tune_get(f"wilson/v{vol}/n{nv}/c1") == policy
    err = rel_l2(to_np(raw), mgo.null_vectors(oracle_fine(U, dims), x0, sweeps))
    assert err < 1e-5, (policy, err)
    gb.mg_tune_set(f"wilson/v{vol}/n{nv}/c1", -1)
    mg.close()
