"""Learned null-vector proposer: GPU forward/loss/gradient against the FP64
oracle network, and training on the GPU."""
import numpy as np
import pytest
import torch

import synthetic as syn
from gpu_helpers import rel_l2, to_dev, to_np
from oracle import lattice as lat, learned as ol, multigrid as mgo

pytestmark = pytest.mark.gpu


def _param_ranges(nv):
    k, out = 0, []
    for name, shp in ol.param_shapes(nv):
        n = int(np.prod(shp))
        out.append((name, k, k + n))
        k += n
    return out


def _setup(gb, dims, block, nv, seed):
    U = syn.gauge_field(dims, 0.4, seed)
    T = mgo.block_orthonormalise(syn.gaussian_field((nv, lat.volume(dims), 12), seed + 1),
                                 dims, block)
    th = ol.init_params(nv, seed + 2).astype(np.float32).astype(np.float64)
    net = gb.mg_cnn_create(nv, 1)
    assert gb.mg_cnn_nparams(net) == th.size
    gb.mg_cnn_set_params(net, torch.from_numpy(th.astype(np.float32)).cuda())
    return U, T, th, net


@pytest.mark.parametrize("dims,block,nv", [((4, 4, 2, 2), (2, 2, 2, 2), 3),
                                           ((4, 4, 4, 4), (4, 4, 2, 2), 8),
                                           ((8, 8, 8, 8), (4, 4, 4, 4), 24)])
def test_forward_loss_gradient_match_oracle(gpu_lib, dims, block, nv):
    """The FP32 network (parameters rounded to FP32 on both sides) against
    the FP64 oracle at the FP32 tier, 1e-5 relative L2, for the vectors, the
    loss and the whole parameter gradient; the last case has the training
    shape of the learned setup (24 vectors, 4^4 aggregates)."""
    gb = gpu_lib
    U, T, th, net = _setup(gb, dims, block, nv, 81)
    out = torch.empty((nv, lat.volume(dims), 12), dtype=torch.complex128, device="cuda")
    gb.mg_cnn_forward(net, dims, to_dev(U), out)
    fw = ol.forward(th, U, dims, nv)
    assert rel_l2(to_np(out), ol.vectors(fw["o"], nv)) < 1e-5
    loss = gb.mg_cnn_loss_grad(net, dims, block, to_dev(U), to_dev(T))
    grad = torch.empty(th.size, dtype=torch.float32, device="cuda")
    gb.mg_cnn_get_params(net, grad, which=1)
    L, g = ol.loss_and_grad(th, U, dims, nv, T, block)
    assert abs(loss - L) < 1e-5 * max(1.0, abs(L))
    got = grad.cpu().numpy().astype(np.float64)
    parts = {name: rel_l2(got[a:b], g[a:b]) for name, a, b in _param_ranges(nv)}
    assert rel_l2(got, g) < 1e-5, parts
    gb.mg_cnn_destroy(net)


def test_training_reduces_loss(gpu_lib):
    gb = gpu_lib
    dims, block, nv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U, T, th, net = _setup(gb, dims, block, nv, 91)
    Ud, Td = to_dev(U), to_dev(T)
    l0 = gb.mg_cnn_loss_grad(net, dims, block, Ud, Td)
    for _ in range(60):
        gb.mg_cnn_loss_grad(net, dims, block, Ud, Td)
        gb.mg_cnn_adam_step(net, 3e-3)
    l1 = gb.mg_cnn_loss_grad(net, dims, block, Ud, Td)
    assert np.isfinite(l1) and l1 < l0 - 0.05, (l0, l1)
    gb.mg_cnn_destroy(net)


def test_trained_proposer_beats_its_untrained_self(gpu_lib):
    """Near-critical mass (m = -0.9, eps 0.3..0.6): a proposer trained on
    the plain setup's vectors of 16 fields has a lower held-out loss than
    the same network untrained (same initial parameters), and with its
    proposals (0 sweeps) the 3-level MG needs fewer outer iterations than
    with the untrained network's or with Gaussian starts."""
    gb = gpu_lib
    from paper_1612_07873_gb300 import learned
    dims, block, nv, mass = (16, 16, 16, 16), (4, 4, 4, 4), 24, -0.9
    samples = []
    for s in range(16):
        eps = 0.3 + 0.3 * np.random.default_rng(1000 + s).random()
        U = to_dev(syn.gauge_field(dims, eps, 1000 + s))
        samples.append((dims, U, learned.plain_vectors(U, dims, block, nv, mass, 1.0, 10, 5000 + s)))
    P = learned.Proposer(nv, seed=3)
    P0 = learned.Proposer(nv, seed=3)
    hist = P.train(samples, block, epochs=6, lr=2e-3)
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
    Ue = to_dev(syn.gauge_field(dims, 0.55, 2000))
    Te = learned.plain_vectors(Ue, dims, block, nv, mass, 1.0, 10, 6000)
    assert P.loss(dims, block, Ue, Te) < P0.loss(dims, block, Ue, Te)
    b = to_dev(syn.gaussian_field((lat.volume(dims), 12), 5, stream=99))
    p3 = gb.default_params(dims=dims, block=[block, (2, 2, 2, 2)], nvec=[nv, 32], mass=mass,
                           csw=1.0, nlevels=3, prec_fine=1, prec_coarse=1, seed=9000)
    rand0 = learned.mg_iterations(p3, Ue, None, 0, b)
    un0 = learned.mg_iterations(p3, Ue, P0.propose(dims, Ue), 0, b)
    cnn0 = learned.mg_iterations(p3, Ue, P.propose(dims, Ue), 0, b)
    assert rand0["status"] == 0 and un0["status"] == 0 and cnn0["status"] == 0
    assert cnn0["true_residual"] <= 1e-10
    assert cnn0["iters"] < un0["iters"], (cnn0["iters"], un0["iters"])
    assert cnn0["iters"] < rand0["iters"], (cnn0["iters"], rand0["iters"])
    P.close()
    P0.close()
