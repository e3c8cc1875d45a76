"""Wilson-clover operator of Eq. (2) and the generic stencil apply (oracle).

Readings of passages where the paper is silent:

* Gamma basis: DeGrand-Rossi chiral basis, gamma_5 = g1 g2 g3 g4 =
  diag(1, 1, -1, -1), so spins {0, 1} and {2, 3} are the two chiralities
  that the footnote of Sec. 3.4 aggregates separately.
* Projectors: P^{+-mu} = 1 +- gamma_mu ("projectors" in Sec. 3.2 up to the
  factor 2 that the -1/2 and the 4 + m diagonal of Eq. (2) require).
* Clover term A_x (Sec. 3.2 names it, gives no formula): the
  Sheikholeslami-Wohlert form
      A_x = c_sw * (i/4) * sum_{mu != nu} sigma_{mu nu} (x) Fhat_{mu nu}(x),
      sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],
      Fhat_{mu nu}  = (Q_{mu nu} - Q_{nu mu}) / 8,
  Q_{mu nu}(x) the sum of the four plaquette leaves at x, all with the
  same orientation.  A_x is Hermitian and commutes with gamma_5.
* Fermion boundary: periodic, antiperiodic in t when asked, realised as a
  factor -1 on every hop that wraps around the t extent.  The clover uses
  the links as given (plaquettes contain each boundary link twice).

Degrees of freedom per site: dof = spin*3 + color (12 complex).
"""
from __future__ import annotations

import numpy as np

from . import lattice as lat

# ---------------------------------------------------------------- gammas
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def _offdiag(ur, ll):
    return np.block([[_Z2, ur], [ll, _Z2]])


GAMMA = np.stack([
    _offdiag(1j * _S1, -1j * _S1),   # gamma_1 (x)
    _offdiag(-1j * _S2, 1j * _S2),   # gamma_2 (y)
    _offdiag(1j * _S3, -1j * _S3),   # gamma_3 (z)
    _offdiag(_I2, _I2),              # gamma_4 (t)
])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
I4 = np.eye(4, dtype=np.complex128)


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu], the spin matrices of the
    clover term A_x (Sec. 3.2; the paper names A_x without a formula)."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


def chirality_of_dof(nd: int) -> np.ndarray:
    """Chirality (0 upper, 1 lower) of each of the nd dofs of a site: the
    first half of the dofs is chirality 0 on every level (fine: spins 0, 1;
    coarse: dof = s*Nv + c with s the chirality).  The split that the
    footnote of Sec. 3.4 applies to the null vectors; the coarse dof order
    is the one of Sec. 6.2."""
    return (np.arange(nd) >= nd // 2).astype(np.int64)


# ---------------------------------------------------------------- clover
def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def clover_leaves(U, dims, sites, mu, nu):
    """Q_{mu nu}(x) at the given sites: the four plaquette leaves touching x,
    each a closed loop from x with the orientation (+mu, +nu, -mu, -nu)
    (field strength of the clover term, Sec. 3.2 reading)."""
    c = lat.coords(dims)[sites]
    e_mu = np.eye(4, dtype=np.int64)[mu]
    e_nu = np.eye(4, dtype=np.int64)[nu]
    at = lambda off: lat.index(dims, c + off)  # noqa: E731
    Um, Un = U[mu], U[nu]
    q = Um[at(0)] @ Un[at(e_mu)] @ _dag(Um[at(e_nu)]) @ _dag(Un[at(0)])
    q = q + Un[at(0)] @ _dag(Um[at(e_nu - e_mu)]) @ _dag(Un[at(-e_mu)]) @ Um[at(-e_mu)]
    q = q + _dag(Um[at(-e_mu)]) @ _dag(Un[at(-e_mu - e_nu)]) @ Um[at(-e_mu - e_nu)] @ Un[at(-e_nu)]
    q = q + _dag(Un[at(-e_nu)]) @ Um[at(-e_nu)] @ Un[at(e_mu - e_nu)] @ _dag(Um[at(0)])
    return q


def clover(U, dims, csw, sites=None) -> np.ndarray:
    """A_x (12x12, dof = spin*3 + color) at the given sites (all by default):
    the clover term of Eq. (2), Sec. 3.2, in the Sheikholeslami-Wohlert
    form c_sw (i/4) sum_{mu != nu} sigma_{mu nu} (x) Fhat_{mu nu}."""
    if sites is None:
        sites = np.arange(lat.volume(dims))
    sites = np.asarray(sites)
    A = np.zeros((len(sites), 12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            q_mn = clover_leaves(U, dims, sites, mu, nu)
            fhat = (q_mn - _dag(q_mn)) / 8.0          # Q_{nu mu} = Q_{mu nu}^dag
            s = sigma(mu, nu)
            A += np.einsum("ab,xij->xaibj", s, fhat).reshape(len(sites), 12, 12)
    return csw * 0.25j * A


# ---------------------------------------------------------------- Eq. (2)
def wilson_clover_blocks(U, dims, mass, csw, antiperiodic=True, sites=None):
    """The nine 12x12 blocks of M (Eq. 2) in every stencil slot, at the given
    sites: [n][9][12][12], so that (M psi)(x) = sum_d B[x, d] psi(x + shift(d)).

    slot 0          : (4 + m) 1 + A_x
    slot 1 + 2 mu   : -1/2 (1 - gamma_mu) (x) U_mu(x)            (x' = x + mu)
    slot 2 + 2 mu   : -1/2 (1 + gamma_mu) (x) U_mu(x - mu)^dag    (x' = x - mu)
    with a factor -1 on hops that wrap in t when antiperiodic.
    """
    vol = lat.volume(dims)
    if sites is None:
        sites = np.arange(vol)
    sites = np.asarray(sites)
    c = lat.coords(dims)[sites]
    n = len(sites)
    B = np.zeros((n, lat.NDIR, 12, 12), dtype=np.complex128)
    B[:, 0] = (4.0 + mass) * np.eye(12) + clover(U, dims, csw, sites)
    lt = dims[3]
    for mu in range(4):
        e = np.eye(4, dtype=np.int64)[mu]
        fwd_link = U[mu][sites]
        bwd_link = _dag(U[mu][lat.index(dims, c - e)])
        sf = np.ones(n)
        sb = np.ones(n)
        if antiperiodic and mu == 3:
            sf[c[:, 3] == lt - 1] = -1.0
            sb[c[:, 3] == 0] = -1.0
        pf = I4 - GAMMA[mu]
        pb = I4 + GAMMA[mu]
        B[:, 1 + 2 * mu] = -0.5 * sf[:, None, None] * np.einsum(
            "ab,xij->xaibj", pf, fwd_link).reshape(n, 12, 12)
        B[:, 2 + 2 * mu] = -0.5 * sb[:, None, None] * np.einsum(
            "ab,xij->xaibj", pb, bwd_link).reshape(n, 12, 12)
    return B


# ---------------------------------------------------------------- stencil
class StencilOp:
    """A nearest-neighbour operator stored as nine dense nd x nd blocks per
    site (Eq. 2 for the fine Wilson-clover matrix, Eq. 3 for every coarse
    level): (A psi)(x) = sum_{d=0..8} B[x, d] psi(x + shift(d))."""

    def __init__(self, dims, blocks):
        self.dims = tuple(int(v) for v in dims)
        self.blocks = np.asarray(blocks)
        self.vol = lat.volume(self.dims)
        assert self.blocks.shape[:2] == (self.vol, lat.NDIR)
        self.nd = self.blocks.shape[-1]
        self.nbr = lat.neighbours(self.dims)

    def apply(self, psi):
        """(A psi)(x) = sum_d B[x, d] psi(x + shift(d)): Eq. (2) for the fine
        operator, Eq. (3) for a coarse one.  psi: [V][nd] (or [k][V][nd])."""
        psi = np.asarray(psi)
        if psi.ndim == 3:
            return np.stack([self.apply(p) for p in psi])
        out = np.zeros_like(psi, dtype=np.complex128)
        for d in range(lat.NDIR):
            out += np.einsum("xij,xj->xi", self.blocks[:, d], psi[self.nbr[:, d]])
        return out

    def dense(self):
        """The full (V*nd) x (V*nd) matrix of Eq. (2) / Eq. (3), blocks of
        partners that coincide (extent 1 or 2) summed (tiny lattices only)."""
        n = self.vol * self.nd
        D = np.zeros((n, n), dtype=np.complex128)
        for x in range(self.vol):
            for d in range(lat.NDIR):
                y = self.nbr[x, d]
                D[x * self.nd:(x + 1) * self.nd, y * self.nd:(y + 1) * self.nd] += self.blocks[x, d]
        return D


def wilson_clover_op(U, dims, mass, csw, antiperiodic=True) -> StencilOp:
    """The Wilson-clover matrix M of Eq. (2) (Sec. 3.2) as a stencil."""
    return StencilOp(dims, wilson_clover_blocks(U, dims, mass, csw, antiperiodic))


def apply_at(blocks_at_sites, psi, dims, sites):
    """Eq. (3) (or Eq. (2)) at the given sites only: (A psi)(x) with B the
    blocks at those sites; used to sample outputs of a full-size lattice one
    by one."""
    c = lat.coords(dims)[np.asarray(sites)]
    out = np.zeros((len(sites), psi.shape[-1]), dtype=np.complex128)
    for d in range(lat.NDIR):
        nb = lat.index(dims, c + lat.shift(d))
        out += np.einsum("xij,xj->xi", blocks_at_sites[:, d], psi[nb])
    return out
