"""Adaptive geometric multigrid setup and Galerkin coarse operator (oracle).

Follows Sec. 3.4, setup steps 1-4, and Eq. (3).

Readings of passages where the paper is silent or garbled:

* Step 1 ("iterate the homogeneous system M x = 0 with a random x0 for k
  iterations"): one iteration ("sweep") is one minimal-residual step on
  M x = 0:  r = -M x,  p = M r,  alpha = <p, r> / <p, p>,  x <- x + alpha r.
  After the k sweeps each vector is scaled to unit 2-norm.  No
  orthogonalisation between vectors is done before the block QR.
* Step 3 (QR of each aggregate block) with the chiral split of the
  footnote: for every aggregate A and chirality s the (|A| * nd/2) x Nv
  matrix of the chirality-s components is orthonormalised by modified
  Gram-Schmidt in column order, every projection done twice ("twice is
  enough").  This is the unique QR with a positive real R diagonal.
  Coarse dof (s, i) = s*Nv + i.
* Eq. (3): the printed diagonal "-delta" stands for a dense block X per
  coarse site (coarse clover plus the hops inside the aggregate), the
  overall minus sign is absorbed into the links, and all nine blocks
  (X and the eight Y_{+-mu}) are stored explicitly.  A fine hop x -> x+mu
  goes into Y_{+mu} of agg(x) exactly when it leaves the aggregate
  through its +mu face (x_mu mod b_mu = b_mu - 1), and into X otherwise.
"""
from __future__ import annotations

import numpy as np

from . import lattice as lat
from .dirac import StencilOp, chirality_of_dof


class RankError(ValueError):
    """An aggregate block of null vectors is rank deficient: the QR of
    Sec. 3.4 step 3 has no positive-definite R."""


# ------------------------------------------------------------- step 1, 2
def null_vectors(op: StencilOp, x0: np.ndarray, sweeps: int) -> np.ndarray:
    """Sec. 3.4 steps 1-2: from each random x0[i] run `sweeps` minimal-
    residual steps on M x = 0, then normalise.  x0: [Nv][V][nd]."""
    out = []
    for x in np.asarray(x0, dtype=np.complex128):
        x = x.copy()
        for _ in range(sweeps):
            r = -op.apply(x)
            p = op.apply(r)
            alpha = np.vdot(p, r) / np.vdot(p, p)
            x = x + alpha * r
        out.append(x / np.linalg.norm(x))
    return np.stack(out)


# ------------------------------------------------------------- step 3
def mgs2(B: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt, each projection done twice, on the columns of
    every matrix in the batch B [..., rows, Nv]: the per-aggregate QR of
    Sec. 3.4 step 3."""
    Q = np.array(B, dtype=np.complex128, copy=True)
    scale = np.linalg.norm(Q, axis=(-2, -1))
    nv = Q.shape[-1]
    for i in range(nv):
        v = Q[..., i]
        for _ in range(2):
            for j in range(i):
                q = Q[..., j]
                v = v - np.sum(np.conj(q) * v, axis=-1, keepdims=True) * q
        nrm = np.linalg.norm(v, axis=-1)
        if np.any(nrm <= 1e-12 * scale):
            raise RankError(f"rank-deficient aggregate block at column {i}")
        Q[..., i] = v / nrm[..., None]
    return Q


def aggregate_blocks(vecs, dims, block, s):
    """[nagg][rows][Nv] matrices of the chirality-s components of the vectors,
    rows ordered (site inside the aggregate in lexicographic order, dof): the
    blocks that Sec. 3.4 step 3 orthonormalises, split by chirality as its
    footnote asks."""
    nv, vol, nd = vecs.shape
    agg = lat.aggregate_of(dims, block)
    nagg = lat.volume(lat.coarse_dims(dims, block))
    order = np.argsort(agg, kind="stable")
    dofs = np.nonzero(chirality_of_dof(nd) == s)[0]
    per = vol // nagg
    B = vecs[:, order][:, :, dofs]
    return B.reshape(nv, nagg, per * len(dofs)).transpose(1, 2, 0), order, dofs


def block_orthonormalise(vecs: np.ndarray, dims, block) -> np.ndarray:
    """Sec. 3.4 step 3 with the chiral split: returns Q [Nv][V][nd]; the
    prolongator column (s, i) is Q[i] restricted to chirality s."""
    vecs = np.asarray(vecs, dtype=np.complex128)
    nv, vol, nd = vecs.shape
    Q = np.zeros_like(vecs)
    for s in (0, 1):
        B, order, dofs = aggregate_blocks(vecs, dims, block, s)
        Qb = mgs2(B)
        nagg = Qb.shape[0]
        tmp = np.zeros((nv, vol, len(dofs)), dtype=np.complex128)
        tmp[:, order, :] = Qb.transpose(2, 0, 1).reshape(nv, vol, len(dofs))
        Q[:, :, dofs] = tmp
        del nagg
    return Q


# ------------------------------------------------------------- P and R
def local_prolongator(Q: np.ndarray) -> np.ndarray:
    """P(x): [V][nd][2Nv]; column (s, i) is Q[i](x) on chirality-s dofs, 0 else
    (the prolongator of Sec. 3.4 step 3, chirally split)."""
    nv, vol, nd = Q.shape
    chi = chirality_of_dof(nd)
    P = np.zeros((vol, nd, 2 * nv), dtype=np.complex128)
    for s in (0, 1):
        rows = np.nonzero(chi == s)[0]
        P[:, rows, s * nv:(s + 1) * nv] = Q[:, :, rows].transpose(1, 2, 0)
    return P


def prolong(Q, ec, dims, block):
    """e = P e_c:  e(x) = P(x) e_c(agg(x))  (prolongation, Sec. 3.4 and
    Sec. 6.6)."""
    agg = lat.aggregate_of(dims, block)
    return np.einsum("xaj,xj->xa", local_prolongator(Q), np.asarray(ec)[agg])


def restrict(Q, r, dims, block):
    """r_c = R r with R = P^dag:  r_c(xc) = sum_{x in A(xc)} P(x)^dag r(x)
    (restriction, Sec. 3.4 and Sec. 6.6)."""
    nv, vol, nd = Q.shape
    agg = lat.aggregate_of(dims, block)
    nagg = lat.volume(lat.coarse_dims(dims, block))
    contrib = np.einsum("xaj,xa->xj", np.conj(local_prolongator(Q)), np.asarray(r))
    out = np.zeros((nagg, 2 * nv), dtype=np.complex128)
    np.add.at(out, agg, contrib)
    return out


def dense_prolongator(Q, dims, block) -> np.ndarray:
    """The explicit (V*nd) x (Vc*2Nv) matrix P of Sec. 3.4 (tiny lattices
    only)."""
    nv, vol, nd = Q.shape
    agg = lat.aggregate_of(dims, block)
    nagg = lat.volume(lat.coarse_dims(dims, block))
    P = np.zeros((vol * nd, nagg * 2 * nv), dtype=np.complex128)
    Pl = local_prolongator(Q)
    for x in range(vol):
        a = agg[x]
        P[x * nd:(x + 1) * nd, a * 2 * nv:(a + 1) * 2 * nv] = Pl[x]
    return P


# ------------------------------------------------------------- step 4
def crosses_face(dims, block, d) -> np.ndarray:
    """[V] bool: does the hop in stencil slot d leave the aggregate?  Such
    hops make the links Y_{+-mu} of Eq. (3); the others fall into X."""
    if d == 0:
        return np.zeros(lat.volume(dims), dtype=bool)
    c = lat.coords(dims)
    mu = (d - 1) // 2
    b = block[mu]
    if (d - 1) % 2 == 0:
        return c[:, mu] % b == b - 1
    return c[:, mu] % b == 0


def galerkin(op: StencilOp, Q: np.ndarray, block) -> StencilOp:
    """Sec. 3.4 step 4: M_hat = P^dag M P, as the nine blocks of Eq. (3).

    For every fine site x and slot d the term P(x)^dag B[x, d] P(x + d)
    is added to slot d of agg(x) if the hop crosses the aggregate face in
    that direction and to slot 0 (X) of agg(x) otherwise."""
    dims = op.dims
    agg = lat.aggregate_of(dims, block)
    cdims = lat.coarse_dims(dims, block)
    nagg = lat.volume(cdims)
    P = local_prolongator(Q)
    n = P.shape[-1]
    Y = np.zeros((nagg, lat.NDIR, n, n), dtype=np.complex128)
    for d in range(lat.NDIR):
        T = np.einsum("xab,xbj->xaj", op.blocks[:, d], P[op.nbr[:, d]])
        C = np.einsum("xai,xaj->xij", np.conj(P), T)
        slot = np.where(crosses_face(dims, block, d), d, 0)
        np.add.at(Y, (agg, slot), C)
    return StencilOp(cdims, Y)


def gamma5_hat(n: int) -> np.ndarray:
    """Coarse gamma_5: +1 on chirality-0 dofs, -1 on chirality-1 dofs.  The
    chiral split of Sec. 3.4 keeps the coarse operator gamma_5-hermitian with
    it, which gives the backward links of Eq. (3) from the forward ones."""
    return np.where(chirality_of_dof(n) == 0, 1.0, -1.0)
