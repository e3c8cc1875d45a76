"""Seeded synthetic inputs for the multigrid tests and benchmark.

This module is shared by the CPU oracle tests and the CUDA-path tests and
holds none of the multigrid method's arithmetic: it only draws random
numbers and shapes them into inputs.

* ``gauge_field``  -- weak-field SU(3) links U = exp(i eps H), H a traceless
  Hermitian Gaussian matrix, one per (direction, site).  The paper's
  gauge configurations (Table 1) are not available; these fields stand in
  for them with the lattice shapes of the paper's workloads.
* ``gaussian_field`` -- complex Gaussian fields (Re, Im iid N(0, 1)), used
  as the random initial null-vector guesses x0 of the adaptive setup
  (Sec. 3.4, step 1) and as right-hand sides.
* ``free_field_starts`` -- deterministic plane-wave start vectors (the low
  modes of the free Wilson operator), a control for the learned setup.
* ``WORKLOADS`` -- lattice sizes and solver parameters of the five
  workloads (small 2-level FP64, production-shaped 3-level FP32, 16-bit
  storage, multi-RHS, learned setup).

Layouts (all complex128, C order):
  gauge  [mu][site][3][3]          mu = 0..3 for x, y, z, t
  field  [..., site, dof]          site = x + Lx*(y + Ly*(z + Lz*t))
"""
from __future__ import annotations

import os

import numpy as np

__all__ = ["gauge_field", "gauge_fields", "gaussian_field", "gauge_transform",
           "free_field_starts", "WORKLOADS", "volume"]


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def _rng(seed: int, stream: int) -> np.random.Generator:
    # PCG64 with a (seed, stream) key: portable and reproducible on x86 and Arm.
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _expm_i_herm(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*h) for a batch of 3x3 Hermitian h by scaling and squaring
    with a degree-12 Taylor polynomial, then one Gram-Schmidt pass over the
    rows and a phase fix so that det U = 1 exactly (up to rounding)."""
    a = 1j * eps * h
    nrm = np.abs(a).sum(axis=-1).max(axis=-1).max(initial=0.0)
    s = max(0, int(np.ceil(np.log2(max(nrm, 1e-300) / 0.05)))) if nrm > 0.05 else 0
    a = a / (2.0 ** s)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), a.shape)
    u = eye.copy()
    term = eye.copy()
    for k in range(1, 13):
        term = term @ a / k
        u = u + term
    for _ in range(s):
        u = u @ u
    # Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1) makes det = 1.
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


_CHUNK = 1 << 18


def _gauge_chunk(args):
    eps, seed, index, n = args
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x5A17, int(index)]))
    g = rng.standard_normal((n, 3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    if eps == 0.0:
        return np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    return _expm_i_herm(h, eps)


def gauge_field(dims, eps: float, seed: int, workers: int | None = None) -> np.ndarray:
    """Weak-field SU(3) gauge field, complex128 [4][V][3][3].

    H = (A + A^dag)/2 - tr(.)/3, A with Re, Im iid N(0, 1); U = exp(i eps H).
    eps = 0 gives the unit (free) field.  The 4V links are drawn in chunks of
    2^18 with one random stream per chunk, so the field does not depend on
    how many worker processes generate it.
    """
    vol = volume(dims)
    total = 4 * vol
    jobs = [(float(eps), seed, i, min(_CHUNK, total - i * _CHUNK))
            for i in range((total + _CHUNK - 1) // _CHUNK)]
    if workers is None:
        workers = min(len(jobs), os.cpu_count() or 1, 16)
    if workers > 1 and len(jobs) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_gauge_chunk, jobs))
    else:
        parts = [_gauge_chunk(j) for j in jobs]
    return np.concatenate(parts).reshape(4, vol, 3, 3)


def _one_field(args):
    dims, eps, seed = args
    return gauge_field(dims, eps, seed, workers=1)


def gauge_fields(dims, eps_list, seeds, workers: int | None = None) -> list:
    """gauge_field(dims, eps_list[i], seeds[i]) for every i, the fields
    drawn in parallel by `workers` spawned processes (each field is
    identical to its serial draw)."""
    jobs = [(tuple(dims), float(e), int(s)) for e, s in zip(eps_list, seeds)]
    if workers is None:
        workers = min(len(jobs), os.cpu_count() or 1, 16)
    if workers <= 1 or len(jobs) <= 1:
        return [_one_field(j) for j in jobs]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_one_field, jobs))


def random_su3(n: int, seed: int) -> np.ndarray:
    """n Haar-like random SU(3) matrices (Gaussian -> QR -> det fix)."""
    rng = _rng(seed, 0x6A7E)
    g = rng.standard_normal((n, 3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    q, r = np.linalg.qr(a)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q[:, :, 2] /= det[:, None]
    return q


def gauge_transform(dims, seed: int) -> np.ndarray:
    """A random site-local SU(3) gauge transformation G(x), [V][3][3]."""
    return random_su3(volume(dims), seed)


def gaussian_field(shape, seed: int, stream: int = 1) -> np.ndarray:
    """Complex Gaussian array of the given shape, Re and Im iid N(0, 1)."""
    rng = _rng(seed, 0x9A55 + int(stream))
    g = rng.standard_normal(tuple(shape) + (2,))
    return g[..., 0] + 1j * g[..., 1]


def free_field_starts(dims, nvec: int, antiperiodic: bool = True) -> np.ndarray:
    """nvec plane-wave vectors [nvec][V][12] complex128: vector i carries
    the unit spin-colour components a = i mod 6 (chirality 0) and a + 6
    (chirality 1), times exp(i p.x) with p the lowest momentum of the
    boundary conditions (p_t = pi / Lt when antiperiodic, else 0) plus
    2 pi / L_mu in direction mu = (i div 6) - 1 for i >= 6 (mu cycling over
    x, y, z, t).  These are low modes of the free (unit-gauge) operator and
    have rank nvec on every aggregate whose extents exceed 1; they carry no
    information about the gauge field."""
    vol = volume(dims)
    L = np.array(dims)
    idx = np.arange(vol)
    coords = np.stack([idx % L[0], (idx // L[0]) % L[1], (idx // (L[0] * L[1])) % L[2],
                       idx // (L[0] * L[1] * L[2])], axis=-1).astype(np.float64)
    p0 = np.array([0.0, 0.0, 0.0, np.pi / L[3] if antiperiodic else 0.0])
    out = np.zeros((nvec, vol, 12), dtype=np.complex128)
    for i in range(nvec):
        a, k = i % 6, i // 6
        p = p0.copy()
        if k >= 1:
            mu = (k - 1) % 4
            p[mu] += 2.0 * np.pi * (1 + (k - 1) // 4) / L[mu]
        phase = np.exp(1j * coords @ p)
        out[i, :, a] = phase
        out[i, :, a + 6] = phase
    return out


# Workload definitions.  Extents are (Lx, Ly, Lz, Lt); "block" lists the
# aggregate extents per coarsening; "nvec" the null vectors per coarsening.
WORKLOADS = {
    # Small 2-level FP64 case: fine 8^4, 2^4 aggregates -> coarse 4^4, 48 dofs.
    "c1_8^4_2lvl_fp64": dict(
        dims=(8, 8, 8, 8), eps=0.3, csw=1.0, mass=-0.2, antiperiodic=1,
        block=[(2, 2, 2, 2)], nvec=[24], sweeps=10, prec="f64", seed=1),
    # Production-shaped 3-level FP32 case: fine 32^3x64, 4^4 then 2^4 aggregates.
    "c2_32^3x64_3lvl_fp32": dict(
        dims=(32, 32, 32, 64), eps=0.5, csw=1.0, mass=-0.40, antiperiodic=1,
        block=[(4, 4, 4, 4), (2, 2, 2, 2)], nvec=[24, 32], sweeps=10, prec="f32",
        seed=11),
    # 16-bit storage form of the small case.
    "c3_8^4_2lvl_16bit": dict(
        dims=(8, 8, 8, 8), eps=0.3, csw=1.0, mass=-0.2, antiperiodic=1,
        block=[(2, 2, 2, 2)], nvec=[24], sweeps=10, prec="bf16", seed=1),
    # Multi-RHS coarse applies on the two coarse lattices of the 3-level case.
    "c4_multirhs": dict(
        lattices=[((8, 8, 8, 16), 48), ((4, 4, 4, 8), 64)],
        nrhs=[1, 8, 16, 32, 64], uneven=[(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 16)]),
}
