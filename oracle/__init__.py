"""Plain FP64 CPU oracle for the adaptive-multigrid coarse-operator hot path.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py``; the library (``paper_1612_07873_gb300``)
never imports it and shares no code with it.

It restates the method of Clark et al., "Accelerating Lattice QCD
Multigrid on GPUs Using Fine-Grained Parallelization" (SC16), in plain
numpy complex128, one definition per function, with no blocking, fusion or
reordering beyond what the definitions state:

* ``dirac``     -- gamma matrices, clover term A_x, Wilson-clover operator
                   M of Eq. (2) as nine dense 12x12 blocks per site, and the
                   generic nearest-neighbour stencil apply (Eq. 2 / Eq. 3).
* ``multigrid`` -- adaptive setup (Sec. 3.4 steps 1-3): null vectors by
                   iterating M x = 0, chiral split, per-aggregate QR by
                   twice-repeated modified Gram-Schmidt; prolongator P,
                   restrictor R = P^dag; Galerkin coarse operator
                   P^dag M P (step 4) in the stencil form of Eq. (3).
* ``solvers``   -- MR smoother, flexible GCR, K-cycle (Sec. 7.1).
* ``schur``     -- red-black (Schur complement) preconditioning of any
                   level's operator (Secs. 3.3, 7.1).
* ``learned``   -- the learned null-vector proposer (an addition, not in
                   the paper).

Every function names the passage it follows.  Where the paper is silent
the reading used is stated in the docstring (gamma basis, projector
normalisation, clover formula, the setup iteration, the coarse diagonal
and the solver tolerances).
"""
from . import lattice, dirac, multigrid, solvers, schur  # noqa: F401
