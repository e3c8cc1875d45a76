"""Learned setup: train the null-vector proposer on the plain setup's
vectors and use its proposals as the starting vectors of the adaptive setup.

Everything runs through the C ABI: the plain setup (mg_setup_nullvecs from
Gaussian starts) makes the training targets, mg_cnn_loss_grad and
mg_cnn_adam_step train the network on the GPU, mg_cnn_forward proposes
vectors that mg_setup_nullvecs then refines with fewer sweeps.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Multigrid, default_params, mg_build_coarse, mg_cnn_adam_step, mg_cnn_create,
               mg_cnn_destroy, mg_cnn_forward, mg_cnn_loss_grad, mg_gcr_solve, mg_get_nullvecs,
               mg_set_setup_sweeps, mg_setup_nullvecs)


def plain_vectors(gauge, dims, block, nvec, mass, csw, sweeps, seed, prec_fine=1):
    """Block-orthonormal null vectors of the plain setup (Gaussian x0 drawn
    on the device from `seed`, `sweeps` MR sweeps): [nvec][V][12] complex128."""
    p = default_params(dims=dims, block=[block], nvec=[nvec], mass=mass, csw=csw, nlevels=2,
                       prec_fine=prec_fine, prec_coarse=prec_fine, setup_sweeps=sweeps, seed=seed)
    mg = Multigrid(p, gauge)
    mg_setup_nullvecs(mg.ctx, 0, None)
    out = torch.empty((nvec, int(np.prod(dims)), 12), dtype=torch.complex128, device="cuda")
    mg_get_nullvecs(mg.ctx, 0, out, kind=1)
    torch.cuda.synchronize()
    mg.close()
    return out


class Proposer:
    """Owner of an mg_cnn network."""

    def __init__(self, nvec, seed=1):
        self.nvec = nvec
        self.net = mg_cnn_create(nvec, seed)

    def close(self):
        if self.net is not None:
            mg_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, samples, block, epochs, lr=2e-3, log=None):
        """samples: list of (dims, gauge, target); one Adam step per sample."""
        hist = []
        for ep in range(epochs):
            tot = 0.0
            for dims, gauge, target in samples:
                tot += mg_cnn_loss_grad(self.net, dims, block, gauge, target)
                mg_cnn_adam_step(self.net, lr)
            hist.append(tot / len(samples))
            if log:
                log(ep, hist[-1])
        return hist

    def step(self, dims, block, gauge, target, lr):
        """One training step (loss, gradient, Adam); returns the loss."""
        loss = mg_cnn_loss_grad(self.net, dims, block, gauge, target)
        mg_cnn_adam_step(self.net, lr)
        return loss

    def loss(self, dims, block, gauge, target):
        return mg_cnn_loss_grad(self.net, dims, block, gauge, target)

    def propose(self, dims, gauge):
        out = torch.empty((self.nvec, int(np.prod(dims)), 12), dtype=torch.complex128,
                          device="cuda")
        return mg_cnn_forward(self.net, dims, gauge, out)


def mg_iterations(params, gauge, init, sweeps, b, tol=1e-10, maxiter=500):
    """Outer GCR iterations of a solve after a setup of `sweeps` MR sweeps
    started from `init` (None: Gaussian from params.seed)."""
    mg = Multigrid(params, gauge)
    mg_set_setup_sweeps(mg.ctx, sweeps)
    mg_setup_nullvecs(mg.ctx, 0, init)
    mg_build_coarse(mg.ctx, 0)
    for l in range(1, params.nlevels - 1):
        mg_setup_nullvecs(mg.ctx, l, None)
        mg_build_coarse(mg.ctx, l)
    x = torch.zeros_like(b)
    st = mg_gcr_solve(mg.ctx, x, b, tol, maxiter, check=False)
    mg.close()
    return st
