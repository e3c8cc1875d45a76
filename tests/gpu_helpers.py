"""Shared set-up for the GPU parity tests: build an mg_ctx and the matching
oracle objects from the same seeded synthetic inputs."""
import numpy as np
import torch

import synthetic as syn
from oracle import dirac, lattice as lat


def rel_l2(got, want) -> float:
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_np(t):
    return t.detach().to("cpu").to(torch.complex128).numpy()


def make_ctx(gb, dims, blocks, nvecs, mass=-0.2, csw=1.0, eps=0.3, seed=1, prec_fine=0,
             prec_coarse=0, sweeps=4, antiperiodic=1, U=None, red_black=0):
    if U is None:
        U = syn.gauge_field(dims, eps, seed)
    p = gb.default_params(dims=dims, block=blocks, nvec=nvecs, mass=mass, csw=csw,
                          nlevels=len(blocks) + 1, prec_fine=prec_fine, prec_coarse=prec_coarse,
                          setup_sweeps=sweeps, t_antiperiodic=antiperiodic, red_black=red_black)
    mg = gb.Multigrid(p, to_dev(U))
    return mg, U


def oracle_fine(U, dims, mass=-0.2, csw=1.0, antiperiodic=True):
    return dirac.wilson_clover_op(U, dims, mass, csw, antiperiodic)


def volume(dims):
    return lat.volume(dims)
