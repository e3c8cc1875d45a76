"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
closed form, an identity, a library routine or a brute-force product.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dirac, lattice as lat, multigrid as mgo, schur as rb, solvers

RNG = np.random.default_rng(1234)


def _rand(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


# ------------------------------------------------------------ lattice indexing
def test_site_index_neighbours_and_aggregates_by_brute_force():
    """Site order x fastest (s = x + Lx (y + Ly (z + Lz t))), stencil slot
    1 + 2 mu = x + mu and 2 + 2 mu = x - mu with periodic wrap, aggregate =
    floor(coordinate / block) in the same order; checked site by site on a
    lattice with four different extents."""
    dims, block = (4, 2, 6, 3), (2, 1, 3, 3)
    c = lat.coords(dims)
    s = 0
    for t in range(3):
        for z in range(6):
            for y in range(2):
                for x in range(4):
                    assert tuple(c[s]) == (x, y, z, t) and lat.index(dims, (x, y, z, t)) == s
                    s += 1
    nb = lat.neighbours(dims)
    agg = lat.aggregate_of(dims, block)
    cd = lat.coarse_dims(dims, block)
    assert cd == (2, 2, 2, 1)
    for s in range(lat.volume(dims)):
        assert nb[s, 0] == s
        for mu in range(4):
            up, dn = list(c[s]), list(c[s])
            up[mu] = (up[mu] + 1) % dims[mu]
            dn[mu] = (dn[mu] - 1) % dims[mu]
            assert nb[s, 1 + 2 * mu] == lat.index(dims, up)
            assert nb[s, 2 + 2 * mu] == lat.index(dims, dn)
        a = [c[s][m] // block[m] for m in range(4)]
        assert agg[s] == a[0] + cd[0] * (a[1] + cd[1] * (a[2] + cd[2] * a[3]))
    # every aggregate holds prod(block) sites
    assert np.all(np.bincount(agg) == np.prod(block))


# ------------------------------------------------------------ gamma algebra
def test_gamma_clifford_and_chiral_basis():
    G = dirac.GAMMA
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)
        for n in range(4):
            assert np.allclose(G[m] @ G[n] + G[n] @ G[m], 2.0 * (m == n) * np.eye(4))
    # DeGrand-Rossi chiral basis: gamma_5 diagonal, upper spins chirality +1.
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))
    # textbook sigma_12 = diag(sigma_3, sigma_3) in this basis
    assert np.allclose(dirac.sigma(0, 1), np.diag([1, -1, 1, -1]))


# ------------------------------------------------------------ free field
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 6)])
def test_free_field_plane_wave_spectrum(dims):
    """U = 1: M e^{ip.x} u = [m + sum(1 - cos p) + i sum gamma sin p] e^{ip.x} u
    with antiperiodic p_t = 2 pi (n + 1/2) / L_t (Eq. 2 with P = 1 -+ gamma)."""
    mass = -0.37
    U = syn.gauge_field(dims, 0.0, 0)
    op = dirac.wilson_clover_op(U, dims, mass, csw=1.3, antiperiodic=True)
    c = lat.coords(dims)
    for trial in range(6):
        n = RNG.integers(0, 64, size=4)
        p = 2 * np.pi * n / np.asarray(dims, dtype=float)
        p[3] = 2 * np.pi * (n[3] + 0.5) / dims[3]
        u = _rand((4, 3))
        phase = np.exp(1j * (c @ p))
        psi = (phase[:, None, None] * u[None]).reshape(-1, 12)
        sym = (mass + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(
            dirac.GAMMA[k] * np.sin(p[k]) for k in range(4))
        want = (phase[:, None, None] * (sym @ u)[None]).reshape(-1, 12)
        got = op.apply(psi)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


# ------------------------------------------------------------ clover
def _abelian_field(dims, mu, nu, k):
    """U_nu(x) = diag(e^{i phi_c x_mu}), phi = (1, 1, -2) * 2 pi k / L_mu; all other
    links 1.  Every plaquette in the (mu, nu) plane is diag(e^{i phi_c})."""
    vol = lat.volume(dims)
    U = np.zeros((4, vol, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    c = lat.coords(dims)
    phi = np.array([1.0, 1.0, -2.0]) * 2 * np.pi * k / dims[mu]
    for col in range(3):
        U[nu, :, col, col] = np.exp(1j * phi[col] * c[:, mu])
    return U, phi


@pytest.mark.parametrize("mu,nu,sig", [
    (0, 1, np.diag([1, -1, 1, -1])),      # sigma_12 = diag(s3, s3)
    (2, 3, np.diag([-1, 1, 1, -1])),      # sigma_34 = diag(-s3, s3)
])
def test_clover_abelian_constant_field(mu, nu, sig):
    """A constant abelian field strength: Fhat_{mu nu} = i sin(phi_c) per colour,
    A = c_sw (i/2) sigma_{mu nu} (x) Fhat = -c_sw/2 sin(phi_c) sigma_{mu nu}."""
    dims = (6, 6, 6, 6)
    csw = 1.7
    U, phi = _abelian_field(dims, mu, nu, 1)
    A = dirac.clover(U, dims, csw, sites=np.arange(0, lat.volume(dims), 37))
    want = -0.5 * csw * np.kron(sig, np.diag(np.sin(phi)))
    assert np.abs(A - want[None]).max() < 1e-14


def test_clover_hermitian_chiral_and_covariant():
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, 0.4, 3)
    A = dirac.clover(U, dims, 1.0)
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-14
    g5 = np.kron(dirac.GAMMA5, np.eye(3))
    assert np.abs(g5 @ A - A @ g5).max() < 1e-14
    G = syn.gauge_transform(dims, 5)
    nb = lat.neighbours(dims)
    Ug = np.stack([G @ U[m] @ np.conj(np.swapaxes(G[nb[:, 1 + 2 * m]], 1, 2)) for m in range(4)])
    Ag = dirac.clover(Ug, dims, 1.0)
    Gs = np.einsum("ab,xij->xaibj", np.eye(4), G).reshape(-1, 12, 12)
    assert np.abs(Ag - Gs @ A @ np.conj(np.swapaxes(Gs, 1, 2))).max() < 1e-13


def test_wilson_operator_gauge_covariance():
    """Eq. (2) under U_mu(x) -> G(x) U_mu(x) G(x+mu)^dag: M[U^G] (G psi) =
    G (M[U] psi), with the antiperiodic t boundary and the clover term.  A
    backward hop through U_mu(x) instead of U_mu(x-mu)^dag, or a forward
    hop through U^dag, breaks it."""
    dims = (4, 2, 3, 4)
    U = syn.gauge_field(dims, 0.5, 13)
    G = syn.gauge_transform(dims, 14)
    nb = lat.neighbours(dims)
    Ug = np.stack([G @ U[m] @ np.conj(np.swapaxes(G[nb[:, 1 + 2 * m]], 1, 2)) for m in range(4)])
    Gs = np.einsum("ab,xij->xaibj", np.eye(4), G).reshape(-1, 12, 12)
    psi = _rand((lat.volume(dims), 12))
    Mpsi = dirac.wilson_clover_op(U, dims, -0.3, 1.0, True).apply(psi)
    got = dirac.wilson_clover_op(Ug, dims, -0.3, 1.0, True).apply(np.einsum("xab,xb->xa", Gs, psi))
    want = np.einsum("xab,xb->xa", Gs, Mpsi)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


# ------------------------------------------------------------ gamma5-hermiticity
def _hierarchy(dims, block, nv, eps=0.3, mass=-0.2, seed=7, sweeps=4):
    U = syn.gauge_field(dims, eps, seed)
    op = dirac.wilson_clover_op(U, dims, mass, 1.0, True)
    x0 = syn.gaussian_field((nv, lat.volume(dims), 12), seed, stream=10)
    v = mgo.null_vectors(op, x0, sweeps)
    Q = mgo.block_orthonormalise(v, dims, block)
    return U, op, Q, mgo.galerkin(op, Q, block)


def test_gamma5_hermiticity_fine_and_coarse():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 6)
    u, v = _rand((lat.volume(dims), 12)), _rand((lat.volume(dims), 12))
    g5 = np.diag(dirac.GAMMA5).real.repeat(3)
    lhs = np.vdot(g5 * op.apply(g5 * u), v)
    assert abs(lhs - np.vdot(u, op.apply(v))) < 1e-12 * abs(lhs)
    n = cop.nd
    g5c = mgo.gamma5_hat(n)
    uc, vc = _rand((cop.vol, n)), _rand((cop.vol, n))
    lhs = np.vdot(g5c * cop.apply(g5c * uc), vc)
    assert abs(lhs - np.vdot(uc, cop.apply(vc))) < 1e-12 * abs(lhs)


def test_coarse_backward_link_relation():
    """Y_{-mu}(x) = g5 Y_{+mu}(x - mu)^dag g5 on a 6^4 -> 3^4 coarsening
    (extent 3 keeps the +mu and -mu partners apart)."""
    dims, block = (6, 6, 6, 6), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 3, sweeps=2)
    g5c = mgo.gamma5_hat(cop.nd)
    c = lat.coords(cop.dims)
    for mu in range(4):
        back = lat.index(cop.dims, c - np.eye(4, dtype=int)[mu])
        yp = cop.blocks[back, 1 + 2 * mu]
        want = g5c[None, :, None] * np.conj(np.swapaxes(yp, 1, 2)) * g5c[None, None, :]
        assert np.abs(cop.blocks[:, 2 + 2 * mu] - want).max() < 1e-13


# ------------------------------------------------------------ brute-force Galerkin
def test_galerkin_equals_dense_product_4to2():
    """Dense D (3072 x 3072), dense P, explicit P^dag D P on the 2^4 coarse
    lattice vs the assembled Eq. (3) stencil (extent-2 partners summed)."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 8)
    P = mgo.dense_prolongator(Q, dims, block)
    want = P.conj().T @ op.dense() @ P
    assert np.abs(want - cop.dense()).max() < 1e-13 * np.abs(want).max()


def test_galerkin_column_probe_6to3():
    """Column probing P^dag (D (P e_j)) with the stencil apply separates every
    one of the nine blocks on a 6^4 -> 3^4 coarsening."""
    dims, block = (6, 6, 6, 6), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 3, sweeps=2)
    P = mgo.dense_prolongator(Q, dims, block)
    n, vc = cop.nd, cop.vol
    nb = lat.neighbours(cop.dims)
    for xc in (0, 17, 40, 80):
        for d in range(9):
            y = nb[xc, d]
            for j in range(n):
                e = np.zeros(vc * n, dtype=np.complex128)
                e[y * n + j] = 1.0
                col = P.conj().T @ op.apply((P @ e).reshape(-1, 12)).ravel()
                got = cop.blocks[xc, d, :, j]
                assert np.abs(col[xc * n:(xc + 1) * n] - got).max() < 1e-13


# ------------------------------------------------------------ gauge invariance
def test_gauge_invariance_of_coarse_operator():
    """U -> G U G^dag(x+mu), x0 -> G x0: the setup, block QR and Galerkin
    product are covariant, so X and Y are unchanged."""
    dims, block, nv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = syn.gauge_field(dims, 0.4, 21)
    G = syn.gauge_transform(dims, 22)
    nb = lat.neighbours(dims)
    Ug = np.stack([G @ U[m] @ np.conj(np.swapaxes(G[nb[:, 1 + 2 * m]], 1, 2)) for m in range(4)])
    x0 = syn.gaussian_field((nv, lat.volume(dims), 12), 23)
    Gs = np.einsum("ab,xij->xaibj", np.eye(4), G).reshape(-1, 12, 12)
    x0g = np.einsum("xab,kxb->kxa", Gs, x0)
    out = []
    for UU, xx in ((U, x0), (Ug, x0g)):
        op = dirac.wilson_clover_op(UU, dims, -0.1, 1.0, True)
        Q = mgo.block_orthonormalise(mgo.null_vectors(op, xx, 3), dims, block)
        out.append(mgo.galerkin(op, Q, block))
    assert np.abs(out[0].blocks - out[1].blocks).max() < 1e-12
    def spectrum(op):
        ev = np.linalg.eigvals(op.dense())
        return ev[np.lexsort((np.round(ev.imag, 8), np.round(ev.real, 8)))]
    assert np.abs(spectrum(out[0]) - spectrum(out[1])).max() < 1e-10


# ------------------------------------------------------------ block QR
def test_block_qr_matches_householder():
    dims, block, nv = (4, 4, 4, 4), (2, 2, 2, 2), 5
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 31)
    Q = mgo.block_orthonormalise(v, dims, block)
    P = mgo.dense_prolongator(Q, dims, block)
    assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-14
    for s in (0, 1):
        B, order, dofs = mgo.aggregate_blocks(v, dims, block, s)
        Bq, _, _ = mgo.aggregate_blocks(Q, dims, block, s)
        for a in range(B.shape[0]):
            q, r = np.linalg.qr(B[a])
            ph = np.diagonal(r) / np.abs(np.diagonal(r))
            assert np.abs(q * ph[None, :] - Bq[a]).max() < 1e-13


def test_block_qr_rank_deficiency_detected():
    dims, block = (2, 2, 2, 2), (2, 2, 2, 2)
    v = syn.gaussian_field((3, 16, 12), 32)
    v[2] = v[0] * (0.5 - 0.25j)
    with pytest.raises(mgo.RankError):
        mgo.block_orthonormalise(v, dims, block)


def test_restrict_prolong_are_dense_p():
    dims, block, nv = (4, 2, 4, 2), (2, 2, 2, 1), 3
    v = syn.gaussian_field((nv, lat.volume(dims), 12), 33)
    Q = mgo.block_orthonormalise(v, dims, block)
    P = mgo.dense_prolongator(Q, dims, block)
    nc = lat.volume(lat.coarse_dims(dims, block))
    ec = _rand((nc, 2 * nv))
    r = _rand((lat.volume(dims), 12))
    assert np.abs(mgo.prolong(Q, ec, dims, block).ravel() - P @ ec.ravel()).max() < 1e-13
    assert np.abs(mgo.restrict(Q, r, dims, block).ravel() - P.conj().T @ r.ravel()).max() < 1e-13


# ------------------------------------------------------------ setup iteration
def test_null_vector_sweep_is_residual_minimising_step():
    """One sweep moves x along r = -M x by the alpha that minimises |M x|."""
    dims = (4, 4, 2, 2)
    U = syn.gauge_field(dims, 0.3, 41)
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, True)
    x0 = syn.gaussian_field((1, lat.volume(dims), 12), 42)
    x1 = mgo.null_vectors(op, x0, 1)[0]
    r = -op.apply(x0[0])
    a, *_ = np.linalg.lstsq(op.apply(r).reshape(-1, 1), -op.apply(x0[0]).ravel(), rcond=None)
    want = x0[0] + a[0] * r
    assert np.abs(x1 - want / np.linalg.norm(want)).max() < 1e-13
    assert abs(np.linalg.norm(x1) - 1.0) < 1e-14


# ------------------------------------------------------------ solvers
def test_mr_single_step_is_least_squares():
    A = _rand((30, 30)) + 20 * np.eye(30)
    b = _rand(30)
    x = solvers.mr(lambda v: A @ v, b, 1)
    a, *_ = np.linalg.lstsq((A @ b).reshape(-1, 1), b, rcond=None)
    assert np.abs(x - a[0] * b).max() < 1e-13


def test_fgcr_solves_to_direct_solution():
    A = _rand((60, 60)) + 30 * np.eye(60)     # field of values away from 0
    b = _rand(60)
    res = solvers.fgcr(lambda v: A @ v, b, None, 1e-12, 500, 10)
    assert np.abs(res.x - np.linalg.solve(A, b)).max() < 1e-10
    assert res.true_residual <= 1e-12
    # with an exact preconditioner GCR finishes in one step
    Ainv = np.linalg.inv(A)
    res = solvers.fgcr(lambda v: A @ v, b, lambda v: Ainv @ v, 1e-10, 5, 10)
    assert res.iters == 1


def test_two_level_mg_converges():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = syn.gauge_field(dims, 0.3, 51)
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, True)
    x0 = syn.gaussian_field((8, lat.volume(dims), 12), 52)
    mg = solvers.MultigridHierarchy.build(op, [x0], 10, [block])
    b = syn.gaussian_field((lat.volume(dims), 12), 53)
    res = mg.solve(b, 1e-10, 100)
    x = res.x
    assert np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b) <= 1e-10
    assert np.abs(x - np.linalg.solve(op.dense(), b.ravel()).reshape(x.shape)).max() < 1e-8


def test_three_level_mg_converges():
    dims = (8, 4, 4, 8)
    U = syn.gauge_field(dims, 0.3, 61)
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, True)
    vol = lat.volume(dims)
    x0a = syn.gaussian_field((6, vol, 12), 62)
    x0b = syn.gaussian_field((8, vol // 16, 12), 63)
    mg = solvers.MultigridHierarchy.build(op, [x0a, x0b], 6, [(2, 2, 2, 2), (2, 1, 1, 2)])
    assert mg.ops[2].nd == 16 and mg.ops[2].dims == (2, 2, 2, 2)
    b = syn.gaussian_field((vol, 12), 64)
    res = mg.solve(b, 1e-10, 100)
    assert res.true_residual <= 1e-10


# ------------------------------------------------------------ red-black (Schur)
def test_schur_solve_reconstructs_the_full_solution():
    """S x_o = b^ plus x_e = A_e^-1 (b_e - H_eo x_o) solves M x = b: compared
    with a dense direct solve of the full system (Secs. 3.3, 7.1)."""
    dims = (4, 2, 2, 4)
    U = syn.gauge_field(dims, 0.4, 81)
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, True)
    S = rb.SchurOp(op)
    b = syn.gaussian_field((lat.volume(dims), 12), 82)
    x_o = np.linalg.solve(S.dense(), S.source(b).ravel()).reshape(-1, 12)
    x = S.reconstruct(b, x_o)
    want = np.linalg.solve(op.dense(), b.ravel()).reshape(x.shape)
    assert np.abs(x - want).max() < 1e-12 * np.abs(want).max()


def test_schur_determinant_identity():
    """det M = det A_e * det S (block elimination), on a coarse operator."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 2)
    S = rb.SchurOp(cop)
    s_full, l_full = np.linalg.slogdet(cop.dense())
    s_s, l_s = np.linalg.slogdet(S.dense())
    s_a, l_a = np.linalg.slogdet(cop.blocks[S.e, 0])
    assert abs(l_full - (l_s + l_a.sum())) < 1e-9 * abs(l_full)
    assert abs(s_full - s_s * np.prod(s_a)) < 1e-9


def test_schur_gamma5_hermiticity_coarse():
    """The coarse Schur operator inherits g5hat-hermiticity from Eq. (3)."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 3)
    S = rb.SchurOp(cop)
    g5c = mgo.gamma5_hat(cop.nd)
    u, v = _rand((len(S.o), cop.nd)), _rand((len(S.o), cop.nd))
    lhs = np.vdot(g5c * S.apply(g5c * u), v)
    assert abs(lhs - np.vdot(u, S.apply(v))) < 1e-12 * abs(lhs)


def test_compact_parity_index():
    """Compact parity order: site x of parity p at h = x >> 1, each pair of
    sites (2h, 2h + 1) holding one site of each parity."""
    dims = (4, 2, 6, 2)
    par = rb.parity(dims)
    for p in (0, 1):
        sites = rb.half_sites(dims, p)
        assert np.array_equal(sites >> 1, np.arange(lat.volume(dims) // 2))
        assert np.all(par[sites] == p)
    # every hop joins the two parities
    assert np.all(par[lat.neighbours(dims)[:, 1:]] != par[:, None])


def test_three_level_mg_with_red_black_smoothing_converges():
    dims = (8, 4, 4, 8)
    U = syn.gauge_field(dims, 0.3, 61)
    op = dirac.wilson_clover_op(U, dims, -0.2, 1.0, True)
    vol = lat.volume(dims)
    x0a = syn.gaussian_field((6, vol, 12), 62)
    x0b = syn.gaussian_field((8, vol // 16, 12), 63)
    plain = solvers.MultigridHierarchy.build(op, [x0a, x0b], 6, [(2, 2, 2, 2), (2, 1, 1, 2)])
    rbp = solvers.MultigridHierarchy(plain.ops, plain.Qs, plain.blocks,
                                     solvers.MGParams(schur=True))
    assert all(S is not None for S in rbp.S)
    b = syn.gaussian_field((vol, 12), 64)
    res = rbp.solve(b, 1e-10, 100)
    assert res.true_residual <= 1e-10
    assert res.iters <= plain.solve(b, 1e-10, 100).iters


# ------------------------------------------------------------ learned proposer
def test_learned_loss_limits():
    """Subspace loss: 0 when the proposals span the target space, 1 when they
    span its orthogonal complement inside every block."""
    from oracle import learned as ol
    dims, block, nv = (4, 2, 2, 2), (2, 2, 2, 2), 3
    vol = lat.volume(dims)
    T = mgo.block_orthonormalise(syn.gaussian_field((nv, vol, 12), 71), dims, block)
    mix = _rand((nv, nv))
    V = np.einsum("ij,jxa->ixa", mix, T)
    L, _ = ol.subspace_loss(V, T, dims, block)
    # V = T M blockwise (M = mix^T): loss = (1/Nv) sum_i delta / (s_i^2 + delta),
    # delta = (1e-5 / Nv) |M|_F^2, s_i the singular values of M
    s2 = np.linalg.svd(mix, compute_uv=False) ** 2
    delta = 1e-5 / nv * s2.sum()
    assert abs(L - np.mean(delta / (s2 + delta))) < 1e-12
    W = syn.gaussian_field((nv, vol, 12), 72)
    Bw = mgo.block_orthonormalise(np.concatenate([T, W]), dims, block)[nv:]
    L, _ = ol.subspace_loss(Bw, T, dims, block)
    assert abs(L - 1.0) < 1e-10


def test_learned_gradient_matches_finite_differences():
    from oracle import learned as ol
    dims, block, nv = (4, 4, 2, 2), (2, 2, 2, 2), 3
    U = syn.gauge_field(dims, 0.4, 73)
    T = mgo.block_orthonormalise(syn.gaussian_field((nv, lat.volume(dims), 12), 74), dims, block)
    th = ol.init_params(nv, 75)
    L, g = ol.loss_and_grad(th, U, dims, nv, T, block)
    rng = np.random.default_rng(76)
    # parameters of every block, the position channels of the first layer
    # (W1[d][c][72..79]) and of the output layer (W3[j][32..39]) included
    off, picks = 0, []
    for name, shp in ol.param_shapes(nv):
        blk = np.arange(int(np.prod(shp))).reshape(shp) + off
        off += blk.size
        if name == "W1":
            picks += list(rng.choice(blk[..., :72].ravel(), 2, replace=False))
            picks += list(rng.choice(blk[..., 72:].ravel(), 3, replace=False))
        elif name == "W3":
            picks += list(rng.choice(blk[:, :32].ravel(), 2, replace=False))
            picks += list(rng.choice(blk[:, 32:].ravel(), 3, replace=False))
        else:
            picks += list(rng.choice(blk.ravel(), 1, replace=False))
    for i in picks:
        e = np.zeros_like(th)
        e[i] = 1e-6
        Lp, _ = ol.loss_and_grad(th + e, U, dims, nv, T, block)
        Lm, _ = ol.loss_and_grad(th - e, U, dims, nv, T, block)
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-5 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_galerkin_coarse_to_coarser_equals_dense_product():
    """Level 2 from the level-1 stencil operator: 8^4 -> 4^4 (n = 8) -> 2^4
    (n = 6).  The coarse level's chirality split is the first / second half
    of its dofs; explicit P2^dag A1 P2 equals the assembled level-2 stencil,
    and the level-2 operator is g5hat-hermitian."""
    dims, block = (8, 8, 8, 8), (2, 2, 2, 2)
    U, op, Q, cop = _hierarchy(dims, block, 4, sweeps=3)
    x1 = syn.gaussian_field((3, cop.vol, cop.nd), 41)
    Q2 = mgo.block_orthonormalise(mgo.null_vectors(cop, x1, 3), cop.dims, block)
    cop2 = mgo.galerkin(cop, Q2, block)
    assert cop2.nd == 6 and tuple(cop2.dims) == (2, 2, 2, 2)
    P2 = mgo.dense_prolongator(Q2, cop.dims, block)
    assert np.abs(P2.conj().T @ P2 - np.eye(P2.shape[1])).max() < 1e-14
    want = P2.conj().T @ cop.dense() @ P2
    assert np.abs(want - cop2.dense()).max() < 1e-13 * np.abs(want).max()
    g5 = mgo.gamma5_hat(cop2.nd)
    u, v = _rand((cop2.vol, cop2.nd)), _rand((cop2.vol, cop2.nd))
    lhs = np.vdot(g5 * cop2.apply(g5 * u), v)
    assert abs(lhs - np.vdot(u, cop2.apply(v))) < 1e-12 * abs(lhs)
