"""Lattice geometry for the oracle (Sec. 6.1: site index <-> coordinates).

Site index s = x + Lx*(y + Ly*(z + Lz*t)); direction mu = 0..3 is x, y, z, t.
Stencil slot d: 0 = the site itself, 1 + 2*mu = forward neighbour x + mu,
2 + 2*mu = backward neighbour x - mu.  Periodic wrap in every direction.
"""
from __future__ import annotations

import numpy as np

NDIR = 9  # diagonal + 8 hops


def volume(dims) -> int:
    """Number of sites of a 4D lattice (Sec. 3.1)."""
    return int(np.prod(dims))


def coords(dims) -> np.ndarray:
    """[V][4] integer coordinates of every site (site order of Sec. 6.1)."""
    lx, ly, lz, lt = dims
    s = np.arange(volume(dims))
    x = s % lx
    y = (s // lx) % ly
    z = (s // (lx * ly)) % lz
    t = s // (lx * ly * lz)
    return np.stack([x, y, z, t], axis=1)


def index(dims, c) -> np.ndarray:
    """Site index of coordinates c ([..., 4]), wrapped periodically (x
    fastest, the site order of Sec. 6.1)."""
    c = np.asarray(c)
    lx, ly, lz, lt = dims
    x = c[..., 0] % lx
    y = c[..., 1] % ly
    z = c[..., 2] % lz
    t = c[..., 3] % lt
    return x + lx * (y + ly * (z + lz * t))


def shift(d: int) -> np.ndarray:
    """Coordinate offset of stencil slot d: 0 for the site term, +-e_mu for
    the hops of Eq. (2) / Eq. (3)."""
    off = np.zeros(4, dtype=np.int64)
    if d > 0:
        mu = (d - 1) // 2
        off[mu] = 1 if (d - 1) % 2 == 0 else -1
    return off


def neighbours(dims) -> np.ndarray:
    """[V][9] site index of the stencil partner in every slot: the site and
    its eight nearest neighbours, the partners of Eq. (2) and Eq. (3)."""
    c = coords(dims)
    return np.stack([index(dims, c + shift(d)) for d in range(NDIR)], axis=1)


def coarse_dims(dims, block):
    """Extents of the coarse lattice: one site per aggregate of `block`
    fine sites (the geometric blocking of Sec. 3.4)."""
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError(f"lattice extent {L} not divisible by block {b}")
    return tuple(int(L // b) for L, b in zip(dims, block))


def aggregate_of(dims, block) -> np.ndarray:
    """[V] coarse site (aggregate) index of every fine site: floor(x / block),
    the hypercubic aggregates of Sec. 3.4."""
    c = coords(dims)
    cd = coarse_dims(dims, block)
    return index(cd, c // np.asarray(block))
