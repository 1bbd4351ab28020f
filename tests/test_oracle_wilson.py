"""Pins of the oracle's Wilson operator (Sec. 1, Eq. 1.2) against facts
that do not come from the oracle itself: the Clifford algebra, the free
field plane-wave closed form, gauge covariance, gamma5-hermiticity and the
adjoint relation (gamma5 D_w(mu))^dag = gamma5 D_w(-mu)."""
import itertools

import numpy as np
import pytest

from oracle import wilson as W
from oracle import freefield as F
from paper_0810_4228_gb300 import synth


def test_gamma_clifford_and_chiral_gamma5():
    g = W.gamma_matrices()
    for a, b in itertools.product(range(4), repeat=2):
        np.testing.assert_allclose(g[a] @ g[b] + g[b] @ g[a], 2 * (a == b) * np.eye(4), atol=1e-15)
    for a in range(4):
        np.testing.assert_allclose(g[a], g[a].conj().T, atol=0)
    g5 = W.gamma5_spin()
    np.testing.assert_allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)
    for a in range(4):  # gamma5 anticommutes with every gamma_nu
        np.testing.assert_allclose(g5 @ g[a] + g[a] @ g5, 0, atol=1e-15)


def test_kappa():
    assert W.kappa_from_mw(-1.5) == pytest.approx(0.2)
    assert W.kappa_from_mw(0.0) == pytest.approx(0.125)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (3, 2, 4, 4), (4, 4, 4, 4)])
@pytest.mark.parametrize("bc_t", [-1, 1])
@pytest.mark.parametrize("mu", [0.0, 0.3, -0.7])
def test_free_field_plane_waves(dims, bc_t, mu):
    """D_w(mu) exp(ipx) u = 2 kappa (a - i gamma.s) exp(ipx) u on U = 1."""
    kappa = 0.2
    U = synth.free_gauge_field(dims)
    D = W.wilson_dirac(U, dims, mu, kappa, bc_t)
    rng = np.random.default_rng(7)
    P = F.momenta(dims, bc_t)
    for j in rng.choice(len(P), size=min(6, len(P)), replace=False):
        p = P[j]
        u = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        col = int(rng.integers(3))
        psi = F.plane_wave(dims, p, u, col)
        lhs = D @ psi
        rhs = F.plane_wave(dims, p, F.dw_momentum(p, mu, kappa) @ u, col)
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_free_field_spectrum_closed_form():
    dims, mu, kappa = (2, 2, 2, 4), 0.3, 0.2
    D = W.wilson_dirac(synth.free_gauge_field(dims), dims, mu, kappa).toarray()
    ev = np.linalg.eigvals(D)
    ref = []
    for p in F.momenta(dims):
        lp, lm = F.dw_eigenvalues(p, mu, kappa)
        ref += [lp] * 6 + [lm] * 6  # 2 spins x 3 colours each
    key = lambda z: (round(z.real, 8), round(z.imag, 8))
    a = sorted(ev, key=key)
    b = sorted(ref, key=key)
    np.testing.assert_allclose(a, b, atol=1e-10)


@pytest.mark.parametrize("mu", [0.0, 0.4])
def test_gauge_covariance(mu):
    """U'_{x,nu} = g_x U_{x,nu} g_{x+nu}^dag, psi' = g psi:  D[U'] G psi = G D[U] psi."""
    dims, kappa = (2, 4, 2, 4), 0.2
    U = synth.gauge_field(dims, 0.7, seed=11)
    g = synth.gauge_transformation(dims, seed=12)
    fwd, _, _, _ = W.neighbours(dims)
    Up = np.einsum("vab,vnbc,vndc->vnad", g, U, g[fwd].conj())
    V = U.shape[0]
    psi = synth.gaussian_source(dims, seed=13)
    Gpsi = np.einsum("vab,vsb->vsa", g, psi.reshape(V, 4, 3)).reshape(-1)
    lhs = W.wilson_dirac(Up, dims, mu, kappa) @ Gpsi
    rhs = np.einsum("vab,vsb->vsa", g, (W.wilson_dirac(U, dims, mu, kappa) @ psi).reshape(V, 4, 3)).reshape(-1)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_gamma5_hermiticity_and_adjoint():
    dims, kappa = (2, 2, 4, 2), 0.2
    U = synth.gauge_field(dims, 1.0, seed=3)
    A0 = W.dense_a(U, dims, 0.0, kappa)
    np.testing.assert_allclose(A0, A0.conj().T, atol=1e-14)
    for mu in (0.3, -0.5):
        Ap = W.dense_a(U, dims, mu, kappa)
        Am = W.dense_a(U, dims, -mu, kappa)
        np.testing.assert_allclose(Ap.conj().T, Am, atol=1e-14)
        assert np.abs(Ap - Ap.conj().T).max() > 1e-3  # genuinely non-Hermitian


def test_links_are_su3():
    U = synth.gauge_field((2, 2, 2, 2), 1.0, seed=1).reshape(-1, 3, 3)
    np.testing.assert_allclose(np.einsum("nab,ncb->nac", U, U.conj()), np.broadcast_to(np.eye(3), U.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(U), 1, atol=1e-14)


def test_site_loop_matches_sparse():
    """The single-site evaluator (used for sampled checks at large volume)
    agrees with the sparse operator."""
    dims, mu, kappa = (2, 4, 2, 4), 0.3, 0.2
    U = synth.gauge_field(dims, 1.0, seed=5)
    x = synth.gaussian_source(dims, seed=6)
    A = W.a_operator(U, dims, mu, kappa)
    y = A @ x
    for site in (0, 5, 17, 63):
        np.testing.assert_allclose(W.wilson_site(U, dims, mu, kappa, x, site), y[12 * site:12 * site + 12], atol=1e-13)


def test_extent_two_hops_sum():
    """On an extent-2 direction the forward and backward neighbour are the
    same site; both hops must be kept (free field, one such direction)."""
    dims, mu, kappa = (2, 4, 4, 4), 0.2, 0.2
    U = synth.free_gauge_field(dims)
    b = synth.gaussian_source(dims, seed=9)
    np.testing.assert_allclose(W.wilson_dirac(U, dims, mu, kappa) @ b, F.dw_free_apply(dims, mu, kappa, b), atol=1e-12)
