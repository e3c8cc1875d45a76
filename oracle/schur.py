"""Red-black (Schur complement) preconditioning -- oracle, FP64.  Test
infrastructure only: the product path never imports this module.

Sec. 3.3: the nearest-neighbour structure of M lets the solver work on the
Schur complement system of one parity; Sec. 7.1: red-black preconditioning
is used on every multigrid level.

Split the sites by parity p(x) = (x0 + x1 + x2 + x3) mod 2 (every extent
even, so that neighbours always have the other parity).  For a stencil
operator M (the nine blocks of Eq. 2 or Eq. 3) the d = 0 block is site-local
and the d = 1..8 blocks (the hops H) connect the two parities:

    M = [[A_e, H_eo], [H_oe, A_o]]
    Schur complement on the odd sites   S = A_o - H_oe A_e^-1 H_eo
    source                              b^ = b_o - H_oe A_e^-1 b_e
    reconstruction                      x_e = A_e^-1 (b_e - H_eo x_o)

and S x_o = b^ together with the reconstruction solves M x = b.

Readings (the paper names the method, not its details):
* the odd sites carry the Schur system (the even ones are eliminated);
* parity vectors are compact: the site x of parity p sits at h = x >> 1
  (valid when the x extent is even: each pair of sites 2h, 2h + 1 holds one
  site of each parity);
* smoothing on a level is z = reconstruct(r, MR_k(S, source(r))), an
  approximate solve of M z = r through the Schur system;
* the coarsest solve is GCR on S to the coarsest tolerance, then the
  reconstruction.
"""
from __future__ import annotations

import numpy as np

from . import lattice as lat
from .dirac import StencilOp


def parity(dims) -> np.ndarray:
    """Site parity (x + y + z + t) mod 2: the red-black colouring of Sec. 3.3."""
    return (lat.coords(dims).sum(axis=1) % 2).astype(np.int64)


def half_sites(dims, p: int) -> np.ndarray:
    """Sites of parity p in compact order (entry h is the site with x >> 1 == h),
    the checkerboard of Sec. 3.3."""
    sites = np.nonzero(parity(dims) == p)[0]
    assert np.array_equal(sites >> 1, np.arange(len(sites)))
    return sites


def supported(dims) -> bool:
    """Every extent even: only then is the periodic lattice two-coloured, so
    that the hops of Eq. (2) / Eq. (3) couple opposite parities (Sec. 3.3)."""
    return all(int(L) % 2 == 0 for L in dims)


class SchurOp:
    """The Schur complement of a StencilOp on the odd sites: the red-black
    preconditioning of Sec. 3.3, used on all levels in Sec. 7.1."""

    def __init__(self, op: StencilOp):
        assert supported(op.dims), "red-black needs every extent even"
        self.op = op
        self.e = half_sites(op.dims, 0)
        self.o = half_sites(op.dims, 1)
        hops = np.array(op.blocks, copy=True)
        hops[:, 0] = 0.0
        self.H = StencilOp(op.dims, hops)
        self.A = op.blocks[:, 0]                       # site-local blocks
        self.Ae_inv = np.linalg.inv(self.A[self.e])    # [V/2][nd][nd]

    def _embed(self, x_half, sites):
        full = np.zeros((self.op.vol, self.op.nd), dtype=np.complex128)
        full[sites] = x_half
        return full

    def apply(self, x_o):
        """S x_o = A_o x_o - H_oe A_e^-1 H_eo x_o (Sec. 3.3)."""
        t_e = self.H.apply(self._embed(x_o, self.o))[self.e]
        u_e = np.einsum("hij,hj->hi", self.Ae_inv, t_e)
        v_o = self.H.apply(self._embed(u_e, self.e))[self.o]
        return np.einsum("hij,hj->hi", self.A[self.o], x_o) - v_o

    def source(self, b):
        """b^ = b_o - H_oe A_e^-1 b_e, the right-hand side of the odd-site
        system (Sec. 3.3)."""
        u_e = np.einsum("hij,hj->hi", self.Ae_inv, b[self.e])
        return b[self.o] - self.H.apply(self._embed(u_e, self.e))[self.o]

    def reconstruct(self, b, x_o):
        """Full x from x_o: x_e = A_e^-1 (b_e - H_eo x_o) (Sec. 3.3)."""
        t_e = b[self.e] - self.H.apply(self._embed(x_o, self.o))[self.e]
        x = self._embed(x_o, self.o)
        x[self.e] = np.einsum("hij,hj->hi", self.Ae_inv, t_e)
        return x

    def dense(self):
        """S of Sec. 3.3 as a dense matrix (tiny lattices only), column by
        column."""
        n = len(self.o) * self.op.nd
        D = np.zeros((n, n), dtype=np.complex128)
        for k in range(n):
            u = np.zeros(n, dtype=np.complex128)
            u[k] = 1.0
            D[:, k] = self.apply(u.reshape(len(self.o), self.op.nd)).ravel()
        return D
