"""Krylov solvers and the K-cycle multigrid preconditioner (oracle).

Sec. 7.1: three-level K-cycle; flexible GCR with a Krylov space of 10
vectors on the fine and intermediate levels, preconditioned by the next
level; 4 pre- and 4 post-smoothing steps of minimal residual (MR); GCR as
the coarsest-grid solver.  Residual norms are L2 norms.

Readings of what the paper does not state:
* MR relaxation omega = 1 (exposed).
* Intermediate-level GCR stops at relative residual 0.25 or 10 iterations,
  the coarsest GCR at 0.1 or 100 iterations (both exposed).
* GCR orthogonalises the new direction A z_k against the previous
  normalised directions with modified Gram-Schmidt; after every cycle of
  nkrylov steps (or on meeting the tolerance) the true residual b - A x is
  recomputed and the cycle restarts, unless maxiter is reached.
* Red-black preconditioning (MGParams.schur): the smoother of every level
  runs MR on the Schur complement and reconstructs, and the coarsest GCR
  solves the Schur system (see ``schur``); the outer GCR keeps the full
  fine operator.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import multigrid as mgo
from . import schur as rb
from .dirac import StencilOp


def mr(apply, b, iters: int, omega: float = 1.0):
    """MR smoother from a zero guess (Sec. 7.1: 4 pre- and 4 post-smoothing
    MR steps; Sec. 3.3 for the Krylov background): r = b; per step p = A r,
    alpha = omega <p, r>/<p, p>, x += alpha r, r -= alpha p."""
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(iters):
        p = apply(r)
        alpha = omega * np.vdot(p, r) / np.vdot(p, p)
        x = x + alpha * r
        r = r - alpha * p
    return x


@dataclass
class GCRResult:
    """Solution, step count, residual history and final true residual of
    one GCR solve (Sec. 7.1 measures convergence in the L2 norm)."""
    x: np.ndarray
    iters: int
    history: list = field(default_factory=list)   # |r_k| / |b| per step
    true_residual: float = np.nan


def fgcr(apply, b, precond, tol: float, maxiter: int, nkrylov: int) -> GCRResult:
    """Flexible GCR(nkrylov) with right preconditioner `precond` (or None):
    the outer and intermediate solvers of Sec. 7.1 (Krylov space of 10).

    Step k: z = K r, w = A z; for j < k: beta = <w_j, w>, w -= beta w_j,
    z -= beta z_j; scale z, w by 1/|w|; alpha = <w, r>; x += alpha z;
    r -= alpha w.  Stop the cycle when |r| <= tol |b|, after nkrylov steps
    or at maxiter; then, unless maxiter is reached, recompute r = b - A x
    and return if it meets the tolerance, else start a new cycle."""
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    hist = []
    total = 0
    if bnorm == 0.0:
        return GCRResult(x, 0, hist, 0.0)
    while True:
        Z, W = [], []
        for _ in range(nkrylov):
            z = precond(r) if precond is not None else r.copy()
            w = apply(z)
            for zj, wj in zip(Z, W):
                beta = np.vdot(wj, w)
                w = w - beta * wj
                z = z - beta * zj
            nw = np.linalg.norm(w)
            w = w / nw
            z = z / nw
            alpha = np.vdot(w, r)
            x = x + alpha * z
            r = r - alpha * w
            Z.append(z)
            W.append(w)
            total += 1
            rn = np.linalg.norm(r)
            hist.append(rn / bnorm)
            if rn <= tol * bnorm or total >= maxiter:
                break
        if total >= maxiter:
            return GCRResult(x, total, hist, np.linalg.norm(b - apply(x)) / bnorm)
        r = b - apply(x)
        rn = np.linalg.norm(r)
        if rn <= tol * bnorm:
            return GCRResult(x, total, hist, rn / bnorm)


@dataclass
class MGParams:
    """Solver parameters of Sec. 7.1 and the readings where it is silent
    (omega, the inner and coarsest tolerances and iteration limits)."""
    nkrylov: int = 10
    mr_iters: int = 4
    mr_omega: float = 1.0
    inner_tol: float = 0.25
    inner_maxiter: int = 10
    coarse_tol: float = 0.1
    coarse_maxiter: int = 100
    schur: bool = False


class MultigridHierarchy:
    """The multigrid hierarchy of Sec. 3.4 with the K-cycle of Sec. 7.1.
    ops[l] is the level-l operator (ops[0] the fine Wilson-clover matrix),
    Qs[l] / blocks[l] the block-orthonormal null vectors and aggregate
    extents of the transfer from level l to l + 1."""

    def __init__(self, ops, Qs, blocks, params: MGParams | None = None):
        self.ops = list(ops)
        self.Qs = list(Qs)
        self.blocks = [tuple(b) for b in blocks]
        self.p = params or MGParams()
        self.inner_iters = [0] * len(self.ops)
        self.S = [rb.SchurOp(op) if self.p.schur and rb.supported(op.dims) else None
                  for op in self.ops]

    @classmethod
    def build(cls, fine: StencilOp, x0s, sweeps, blocks, params=None):
        """Full setup (Sec. 3.4 steps 1-4, then recursively on the coarse
        operator): for each level, null vectors from x0s[l], block QR,
        Galerkin coarse operator."""
        ops, Qs = [fine], []
        for l, (x0, blk) in enumerate(zip(x0s, blocks)):
            v = mgo.null_vectors(ops[l], x0, sweeps)
            Q = mgo.block_orthonormalise(v, ops[l].dims, blk)
            Qs.append(Q)
            ops.append(mgo.galerkin(ops[l], Q, blk))
        return cls(ops, Qs, blocks, params)

    def kcycle(self, level: int, r):
        """One K-cycle at `level` (Sec. 7.1): MR pre-smooth, restrict the
        residual (Sec. 6.6), solve on level + 1 with GCR (preconditioned by
        the next K-cycle unless level + 1 is the coarsest), prolong and add,
        MR post-smooth."""
        p = self.p
        A = self.ops[level].apply
        dims, blk, Q = self.ops[level].dims, self.blocks[level], self.Qs[level]
        S = self.S[level]
        if S is None:
            smooth = lambda v: mr(A, v, p.mr_iters, p.mr_omega)  # noqa: E731
        else:
            smooth = lambda v: S.reconstruct(v, mr(S.apply, S.source(v), p.mr_iters,  # noqa: E731
                                                   p.mr_omega))
        x = smooth(r)
        rc = mgo.restrict(Q, r - A(x), dims, blk)
        nxt = level + 1
        if nxt == len(self.ops) - 1:
            Sc = self.S[nxt]
            if Sc is None:
                res = fgcr(self.ops[nxt].apply, rc, None, p.coarse_tol, p.coarse_maxiter,
                           p.nkrylov)
                xc = res.x
            else:
                res = fgcr(Sc.apply, Sc.source(rc), None, p.coarse_tol, p.coarse_maxiter,
                           p.nkrylov)
                xc = Sc.reconstruct(rc, res.x)
        else:
            res = fgcr(self.ops[nxt].apply, rc, lambda v: self.kcycle(nxt, v),
                       p.inner_tol, p.inner_maxiter, p.nkrylov)
            xc = res.x
        self.inner_iters[nxt] += res.iters
        x = x + mgo.prolong(Q, xc, dims, blk)
        x = x + smooth(r - A(x))
        return x

    def solve(self, b, tol: float = 1e-10, maxiter: int = 200) -> GCRResult:
        """Outer flexible GCR on the fine operator preconditioned by the
        K-cycle, to |b - M x| <= tol |b| (Sec. 7.1)."""
        self.inner_iters = [0] * len(self.ops)
        return fgcr(self.ops[0].apply, b, lambda v: self.kcycle(0, v), tol, maxiter,
                    self.p.nkrylov)
