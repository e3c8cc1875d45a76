"""Learned null-vector proposer (oracle, FP64).  Not in the paper: an
addition that proposes the random starting vectors x0 of Sec. 3.4 step 1.

Network (every layer a nearest-neighbour stencil on the lattice, the
"4D convolution" of this build):
  position  p(x)  = cos, sin (2 pi x_mu / L_mu), mu = 0..3      8 channels
  features  f(x)  = (Re, Im) of the four links U_mu(x), then p(x)    72 + 8
  layer 1   h1(x) = tanh(b1 + sum_{d=0..8} W1[d] f(x + shift(d)))   80 -> 32
  layer 2   h2(x) = tanh(b2 + sum_{d=0..8} W2[d] h1(x + shift(d)))  32 -> 32
  layer 3   o(x)  = b3 + W3 [h2(x); p(x)]                            40 -> 24 Nv
  vector i at site x, dof a: o[x][24 i + 2a] + i o[x][24 i + 2a + 1].
The links carry no position; p gives the network the phases of the lowest
lattice momenta, so it can produce the slowly varying low modes the setup
looks for and correct them from the local links.

Loss (proposed reading; raw null vectors are not unique): for every
aggregate A and chirality s, with B the (|A| nd/2) x Nv block of the
predicted vectors and T the orthonormal block of the target vectors
(the plain setup's block-orthonormalised null vectors),
  l(A, s) = 1 - tr(C^H G^{-1} C) / Nv,  G = B^H B + delta I, C = B^H T,
the fraction of the target subspace outside span(B); the loss is the mean
over blocks.  delta = kappa |B|_F^2 with kappa = 1e-5 / Nv keeps G
invertible at any scale of B; its derivative is part of the gradient:
  d f / d B^* = T A^H - B A A^H - kappa |A|_F^2 B,  A = G^{-1} C.
"""
from __future__ import annotations

import numpy as np

from . import lattice as lat
from .dirac import chirality_of_dof
from .multigrid import aggregate_blocks

NLINK, NPOS, NHID = 72, 8, 32
NFEAT = NLINK + NPOS


def param_shapes(nvec: int):
    """Parameter names and shapes of the three stencil layers (an addition,
    not in the paper; it proposes the x0 of Sec. 3.4 step 1)."""
    return [("W1", (9, NHID, NFEAT)), ("b1", (NHID,)), ("W2", (9, NHID, NHID)),
            ("b2", (NHID,)), ("W3", (24 * nvec, NHID + NPOS)), ("b3", (24 * nvec,))]


def unflatten(theta, nvec):
    """Flat parameter vector -> named arrays, in param_shapes order (the
    learned addition; no paper passage)."""
    out, k = {}, 0
    for name, shp in param_shapes(nvec):
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def flatten(p, nvec):
    """Named arrays -> flat parameter vector (inverse of unflatten)."""
    return np.concatenate([p[name].ravel() for name, _ in param_shapes(nvec)])


def positions(dims):
    """[V][8]: cos and sin of 2 pi x_mu / L_mu for mu = 0..3 (addition)."""
    c = lat.coords(dims).astype(np.float64)
    ph = 2.0 * np.pi * c / np.asarray(dims, dtype=np.float64)
    return np.stack([np.cos(ph), np.sin(ph)], axis=-1).reshape(-1, 8)


def features(U, dims):
    """[V][80]: (Re, Im) of U_mu(x)[a][b], ordered (mu, a, b, re/im) -- the
    links of Eq. (2) at x -- then the 8 position channels (addition)."""
    vol = U.shape[1]
    u = np.transpose(U, (1, 0, 2, 3)).reshape(vol, 36)
    links = np.stack([u.real, u.imag], axis=-1).reshape(vol, 72)
    return np.concatenate([links, positions(dims)], axis=1)


def conv9(inp, W, b, nbr):
    """out(x) = b + sum_d W[d] in(x + shift(d)): one layer, a stencil over
    the nine partners of Eq. (2) (the "4D convolution" of the addition)."""
    out = np.broadcast_to(b, (inp.shape[0], W.shape[1])).copy()
    for d in range(9):
        out += inp[nbr[:, d]] @ W[d].T
    return out


def forward(theta, U, dims, nvec):
    """The three layers of the proposer on one gauge field (addition),
    keeping every activation for the backward pass."""
    p = unflatten(theta, nvec)
    nbr = lat.neighbours(dims)
    f = features(U, dims)
    h1 = np.tanh(conv9(f, p["W1"], p["b1"], nbr))
    h2 = np.tanh(conv9(h1, p["W2"], p["b2"], nbr))
    hp = np.concatenate([h2, f[:, NLINK:]], axis=1)
    o = hp @ p["W3"].T + p["b3"]
    return dict(f=f, h1=h1, h2=h2, hp=hp, o=o, nbr=nbr, p=p)


def vectors(o, nvec):
    """[Nv][V][12] complex from the output channels: the proposed starting
    vectors x0 of Sec. 3.4 step 1."""
    vol = o.shape[0]
    z = o.reshape(vol, nvec, 12, 2)
    return np.transpose(z[..., 0] + 1j * z[..., 1], (1, 0, 2))


def subspace_loss(V, T, dims, block):
    """Mean over (aggregate, chirality) blocks of 1 - tr(C^H G^{-1} C)/Nv and its
    gradient dL/dV* (same layout as V).  The blocks are those of the
    per-aggregate QR of Sec. 3.4 step 3 (addition: the paper trains
    nothing)."""
    nv, vol, nd = V.shape
    grad = np.zeros_like(V)
    total, nblocks = 0.0, 0
    for s in (0, 1):
        B, order, dofs = aggregate_blocks(V, dims, block, s)   # [nagg][rows][Nv]
        Tb, _, _ = aggregate_blocks(T, dims, block, s)
        nagg = B.shape[0]
        kappa = 1e-5 / nv
        G = np.conj(np.swapaxes(B, 1, 2)) @ B
        G = G + kappa * np.real(np.trace(G, axis1=1, axis2=2))[:, None, None] * np.eye(nv)
        C = np.conj(np.swapaxes(B, 1, 2)) @ Tb
        A = np.linalg.solve(G, C)
        f = np.real(np.trace(np.conj(np.swapaxes(C, 1, 2)) @ A, axis1=1, axis2=2))
        total += float(np.sum(1.0 - f / nv))
        nblocks += nagg
        AH = np.conj(np.swapaxes(A, 1, 2))
        a2 = np.sum(np.abs(A) ** 2, axis=(1, 2))
        gB = -(Tb @ AH - B @ (A @ AH) - kappa * a2[:, None, None] * B) / nv
        tmp = np.zeros((nv, vol, len(dofs)), dtype=np.complex128)
        tmp[:, order, :] = gB.transpose(2, 0, 1).reshape(nv, vol, len(dofs))
        grad[:, :, dofs] += tmp
    return total / nblocks, grad / nblocks


def loss_and_grad(theta, U, dims, nvec, T, block):
    """Loss and its gradient with respect to the flat parameter vector, by
    the chain rule through the three layers (addition, not in the paper)."""
    fw = forward(theta, U, dims, nvec)
    p, nbr = fw["p"], fw["nbr"]
    V = vectors(fw["o"], nvec)
    L, gV = subspace_loss(V, T, dims, block)
    vol = V.shape[1]
    # real-parameter gradient: dL/dRe z = 2 Re(dL/dz*), dL/dIm z = 2 Im(dL/dz*)
    gz = np.transpose(gV, (1, 0, 2))                     # [V][Nv][12]
    go = np.stack([2 * gz.real, 2 * gz.imag], axis=-1).reshape(vol, 24 * nvec)
    g = {"W3": go.T @ fw["hp"], "b3": go.sum(0)}
    gh2 = go @ p["W3"][:, :NHID]
    gp2 = gh2 * (1.0 - fw["h2"] ** 2)
    g["b2"] = gp2.sum(0)
    g["W2"] = np.stack([gp2.T @ fw["h1"][nbr[:, d]] for d in range(9)])
    gh1 = np.zeros_like(fw["h1"])
    for d in range(9):  # h1(x + d) feeds out(x): scatter back to the source site
        np.add.at(gh1, nbr[:, d], gp2 @ p["W2"][d])
    gp1 = gh1 * (1.0 - fw["h1"] ** 2)
    g["b1"] = gp1.sum(0)
    g["W1"] = np.stack([gp1.T @ fw["f"][nbr[:, d]] for d in range(9)])
    return L, flatten(g, nvec)


def init_params(nvec: int, seed: int):
    """Seeded initial parameters: zero biases, weights N(0, 1/fan_in)
    (addition, not in the paper)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes(nvec):
        if name.startswith("b"):
            p[name] = np.zeros(shp)
        else:
            fan_in = shp[-1] * (9 if len(shp) == 3 else 1)
            p[name] = rng.standard_normal(shp) / np.sqrt(fan_in)
    return flatten(p, nvec)
