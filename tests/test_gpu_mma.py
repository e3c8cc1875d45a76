"""Multi-RHS coarse apply on the tcgen05 tensor cores (16-bit links and
operands, FP32 accumulation) against the FP64 oracle stencil apply."""
import time

import numpy as np
import pytest
import torch

import synthetic as syn
from gpu_helpers import make_ctx, rel_l2, to_dev, to_np
from oracle import dirac, lattice as lat

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("cdims,nv,nrhs", [
    ((2, 2, 4, 2), 24, 8), ((2, 2, 4, 2), 24, 64), ((2, 2, 2, 2), 32, 32),
    ((3, 2, 2, 2), 16, 4), ((4, 4, 2, 2), 24, 16)])
def test_coarse_apply_tensor_cores(gpu_lib, prec, cdims, nv, nrhs):
    gb = gpu_lib
    dims = tuple(c * 2 for c in cdims)
    mg, U = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], prec_fine=1, prec_coarse=prec)
    n, vol = 2 * nv, lat.volume(cdims)
    links = syn.gaussian_field((vol, 9, n, n), 51) / np.sqrt(n)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = syn.gaussian_field((vol, n, nrhs), 52)
    y = torch.full((vol, n, nrhs), float("nan"), dtype=torch.complex64, device="cuda")
    for _ in range(2):  # twice: the second call reuses TMEM / shared state
        gb.mg_coarse_apply(mg.ctx, 1, y, to_dev(x, torch.complex64), nrhs=nrhs)
    gb.mg_device_status(mg.ctx)
    cop = dirac.StencilOp(cdims, links)
    want = np.stack([cop.apply(x[:, :, k]) for k in range(nrhs)], axis=-1)
    err = rel_l2(to_np(y), want)
    assert err < 5e-3, err
    mg.close()


@pytest.mark.parametrize("cdims,nv,nrhs", [
    ((4, 4, 4, 8), 24, 8),     # 512 sites: several per CTA
    ((6, 4, 4, 6), 24, 64),
    ((4, 4, 4, 8), 32, 32),
    ((4, 4, 4, 8), 16, 4),
])
def test_every_launch_shape_on_many_sites(gpu_lib, cdims, nv, nrhs):
    """Every candidate launch shape of the autotuner, pinned in turn: the
    pipelined kernel (choice 100000 PC + 10000 IL + 1000 cps + 100 KH +
    10 SL + SA: operand converted in the kernel or pre-converted by a
    streaming pass, interleaved or split accumulator rows, cps CTAs per SM,
    KH half slots per stage, SL-deep load ring, SA-deep operand ring) and the
    register-staged kernel (choice = CTAs per SM), on lattices with more
    sites than SMs, so the rings and both TMEM accumulators cycle."""
    gb = gpu_lib
    dims = tuple(c * 2 for c in cdims)
    mg, _ = make_ctx(gb, dims, [(2, 2, 2, 2)], [nv], prec_fine=1, prec_coarse=2)
    n, vol = 2 * nv, lat.volume(cdims)
    links = syn.gaussian_field((vol, 9, n, n), 55) / np.sqrt(n)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = syn.gaussian_field((vol, n, nrhs), 56)
    cop = dirac.StencilOp(cdims, links)
    want = np.stack([cop.apply(x[:, :, k]) for k in range(nrhs)], axis=-1)
    key = f"mma2/bf16/n{n}/r{nrhs}/v{vol}/b1"
    xd = to_dev(x, torch.complex64)
    y = torch.empty((vol, n, nrhs), dtype=torch.complex64, device="cuda")
    gb.mg_tune_set(key, -1)
    gb.mg_coarse_apply(mg.ctx, 1, y, xd, nrhs=nrhs)  # tunes: times every candidate
    gb.mg_device_status(mg.ctx)
    choices = [c for c, _ in gb.mg_tune_report(key)]
    pc, inkernel = [c for c in choices if c >= 100000], [c for c in choices if c < 100000]
    assert any(1000 < c < 10000 for c in inkernel), choices
    assert any(c > 10000 for c in inkernel) and any(c <= 8 for c in choices), choices
    assert any(c % 100000 < 10000 for c in pc) and any(c % 100000 > 10000 for c in pc), choices
    for choice in choices:
        gb.mg_tune_set(key, choice)
        y.fill_(float("nan"))
        gb.mg_coarse_apply(mg.ctx, 1, y, xd, nrhs=nrhs)
        gb.mg_device_status(mg.ctx)
        assert gb.mg_tune_get(key) == choice, (choice, gb.mg_tune_get(key))
        err = rel_l2(to_np(y), want)
        assert err < 5e-3, (choice, err)
    gb.mg_tune_set(key, -1)
    mg.close()


def test_uneven_lattices_one_launch_and_graph(gpu_lib):
    """4^4, 6^4 and 8^3x16 coarse lattices (n = 48, BF16) in one persistent
    tensor-core launch, then the same launch captured in a CUDA graph and
    replayed with new inputs."""
    gb = gpu_lib
    cds = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 16)]
    nv, n, nrhs = 24, 48, 8
    mgs, ys, xs, want = [], [], [], []
    for k, cd in enumerate(cds):
        mg, _ = make_ctx(gb, tuple(2 * c for c in cd), [(2, 2, 2, 2)], [nv], prec_fine=1,
                         prec_coarse=2, eps=0.0)
        vol = lat.volume(cd)
        links = syn.gaussian_field((vol, 9, n, n), 60 + k) / np.sqrt(n)
        gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
        mgs.append((mg, dirac.StencilOp(cd, links)))
        xs.append(to_dev(syn.gaussian_field((vol, n, nrhs), 70 + k), torch.complex64))
        ys.append(torch.zeros((vol, n, nrhs), dtype=torch.complex64, device="cuda"))
    ctxs = [m.ctx for m, _ in mgs]
    gb.mg_coarse_apply_multi(ctxs, [1, 1, 1], ys, xs, nrhs)
    gb.mg_device_status(ctxs[0])
    for (m, cop), y, x in zip(mgs, ys, xs):
        xn = to_np(x)
        ref = np.stack([cop.apply(xn[:, :, r]) for r in range(nrhs)], axis=-1)
        assert rel_l2(to_np(y), ref) < 5e-3
    # capture and replay
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gb.mg_coarse_apply_multi(ctxs, [1, 1, 1], ys, xs, nrhs, stream=s)
    for k, x in enumerate(xs):
        x.copy_(to_dev(syn.gaussian_field(tuple(x.shape), 80 + k), torch.complex64))
        ys[k].zero_()
    g.replay()
    torch.cuda.synchronize()
    gb.mg_device_status(ctxs[0])
    for (m, cop), y, x in zip(mgs, ys, xs):
        xn = to_np(x)
        ref = np.stack([cop.apply(xn[:, :, r]) for r in range(nrhs)], axis=-1)
        assert rel_l2(to_np(y), ref) < 5e-3
    for m, _ in mgs:
        m.close()


def test_injected_wait_times_out_and_context_stays_usable(gpu_lib):
    """The tensor-core launch's mbarrier waits are bounded by a one-second
    budget: an injected wait on a barrier that nothing arrives at gives up,
    the launch writes nothing, mg_device_status reports MG_ERR_TIMEOUT once,
    and the next launch on the same context is correct."""
    gb = gpu_lib
    cdims, nv, nrhs = (2, 2, 4, 2), 24, 8
    mg, _ = make_ctx(gb, tuple(2 * c for c in cdims), [(2, 2, 2, 2)], [nv], prec_fine=1,
                     prec_coarse=2)
    n, vol = 2 * nv, lat.volume(cdims)
    links = syn.gaussian_field((vol, 9, n, n), 53) / np.sqrt(n)
    gb.mg_set_coarse_links(mg.ctx, 1, to_dev(links))
    x = to_dev(syn.gaussian_field((vol, n, nrhs), 54), torch.complex64)
    y = torch.zeros((vol, n, nrhs), dtype=torch.complex64, device="cuda")
    with pytest.raises(gb.MGError) as e:
        gb.mg_inject_fault(mg.ctx, "no_such_fault", 1)
    assert e.value.status == gb.MG_ERR_ARG
    gb.mg_inject_fault(mg.ctx, "coarse_mma_wait", 1)
    t0 = time.monotonic()
    gb.mg_coarse_apply(mg.ctx, 1, y, x, nrhs=nrhs)
    with pytest.raises(gb.MGError) as e:
        gb.mg_device_status(mg.ctx)
    waited = time.monotonic() - t0
    assert e.value.status == gb.MG_ERR_TIMEOUT
    assert 0.9 < waited < 30.0, waited
    assert not torch.any(y != 0)  # the stalled launch wrote nothing
    gb.mg_device_status(mg.ctx)  # the record was cleared
    gb.mg_coarse_apply(mg.ctx, 1, y, x, nrhs=nrhs)
    gb.mg_device_status(mg.ctx)
    cop = dirac.StencilOp(cdims, links)
    xn = to_np(x)
    want = np.stack([cop.apply(xn[:, :, k]) for k in range(nrhs)], axis=-1)
    assert rel_l2(to_np(y), want) < 5e-3
    mg.close()
