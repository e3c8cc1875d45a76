"""Checks of the seeded input generators shared by the oracle and the CUDA
path: the weak-field SU(3) links are special unitary, are the exponential
they claim to be, have the stated normalisation of H, and do not depend on
the number of worker processes that draw them."""
import numpy as np
import pytest

import synthetic as syn


def test_links_are_special_unitary():
    U = syn.gauge_field((4, 4, 4, 8), 0.5, 7).reshape(-1, 3, 3)
    eye = np.eye(3)
    uu = np.einsum("nji,njk->nik", U.conj(), U)
    assert np.abs(uu - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1.0).max() < 1e-14


def test_exponential_matches_library_expm():
    """exp(i eps h) by scaling and squaring equals scipy's expm (Pade) on
    traceless Hermitian h, also where the scaling step is taken (large eps)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    a = rng.standard_normal((64, 3, 3)) + 1j * rng.standard_normal((64, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    h -= (np.trace(h, axis1=-2, axis2=-1).real / 3.0)[:, None, None] * np.eye(3)
    for eps in (0.01, 0.3, 2.5):
        got = syn._expm_i_herm(h, eps)
        want = np.stack([scipy_linalg.expm(1j * eps * m) for m in h])
        assert np.abs(got - want).max() < 1e-13, eps


def test_field_strength_normalisation():
    """H = (A + A^dag)/2 - tr/3 with Re, Im of A iid N(0, 1) has
    E tr H^2 = 8: the diagonal of (A + A^dag)/2 is Re A_ii ~ N(0, 1) and the
    trace removal keeps 2/3 of its variance (3 x 2/3 = 2); each of the six
    off-diagonal entries has E|H_ij|^2 = 1/2 + 1/2 = 1.  For small eps,
    Re tr U / 3 = 1 - eps^2 tr H^2 / 6 + O(eps^4), so
    (1 - <Re tr U>/3) / eps^2 -> 8/6 = 4/3.  A missing 1/2 in H (factor 4
    in tr H^2) or no trace removal (tr H^2 = 9) moves it far outside 2 %."""
    eps = 0.02
    U = syn.gauge_field((8, 8, 8, 8), eps, 3).reshape(-1, 3, 3)
    tr = np.trace(U, axis1=-2, axis2=-1).real / 3.0
    ratio = (1.0 - tr.mean()) / eps ** 2
    assert abs(ratio - 4.0 / 3.0) < 0.02 * 4.0 / 3.0, ratio
    # Im tr U is odd in H: its mean vanishes within the sampling error
    assert abs(np.trace(U, axis1=-2, axis2=-1).imag.mean()) < 5 * eps ** 3


def test_unit_field_at_zero_eps():
    U = syn.gauge_field((2, 2, 2, 4), 0.0, 1)
    assert np.array_equal(U, np.broadcast_to(np.eye(3, dtype=np.complex128), U.shape))


def test_field_does_not_depend_on_worker_count():
    dims = (16, 16, 16, 20)  # 4 V = 327680 links: two chunks of 2^18
    a = syn.gauge_field(dims, 0.4, 9, workers=1)
    b = syn.gauge_field(dims, 0.4, 9, workers=2)
    assert np.array_equal(a, b)


def test_gaussian_field_moments_and_seeding():
    z = syn.gaussian_field((1 << 18,), 4)
    assert abs(z.mean()) < 0.02
    assert abs(np.mean(np.abs(z) ** 2) - 2.0) < 0.02
    assert abs(np.mean(z * z)) < 0.02  # Re and Im independent, equal variance
    assert np.array_equal(z, syn.gaussian_field((1 << 18,), 4))
    assert not np.array_equal(z, syn.gaussian_field((1 << 18,), 4, stream=2))


def test_random_su3_is_special_unitary():
    G = syn.gauge_transform((2, 2, 2, 2), 5)
    uu = np.einsum("nji,njk->nik", G.conj(), G)
    assert np.abs(uu - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(G) - 1.0).max() < 1e-14


def test_many_fields_equal_their_serial_draws():
    dims = (2, 2, 4, 4)
    eps, seeds = [0.3, 0.45, 0.6], [1000, 1001, 1002]
    par = syn.gauge_fields(dims, eps, seeds, workers=2)
    for e, s, u in zip(eps, seeds, par):
        assert np.array_equal(u, syn.gauge_field(dims, e, s, workers=1))


def test_free_field_starts_are_low_momentum_plane_waves():
    """Vector i: unit components i mod 6 and i mod 6 + 6 (one per
    chirality) times exp(i p.x), p_t = pi / Lt plus 2 pi / L_mu along mu =
    i div 6 - 1; every vector has unit modulus on its two components, and
    the translation by one site along mu multiplies it by exp(i p_mu)."""
    dims = (4, 6, 4, 8)
    v = syn.free_field_starts(dims, 24)
    vol = syn.volume(dims)
    assert v.shape == (24, vol, 12)
    for i in range(24):
        a, k = i % 6, i // 6
        nz = np.nonzero(np.abs(v[i]).sum(axis=0))[0]
        assert list(nz) == [a, a + 6]
        assert np.allclose(np.abs(v[i][:, [a, a + 6]]), 1.0)
        p = np.array([0.0, 0.0, 0.0, np.pi / dims[3]])
        if k >= 1:
            p[k - 1] += 2 * np.pi / dims[k - 1]
        # x -> x + 1 (away from the x wrap): phase exp(i p_x)
        s = 1 + dims[0] * (2 + dims[1] * (1 + dims[2] * 3))
        assert np.isclose(v[i][s + 1, a] / v[i][s, a], np.exp(1j * p[0]))
        st = dims[0] * dims[1] * dims[2]
        assert np.isclose(v[i][s + st, a] / v[i][s, a], np.exp(1j * p[3]))
