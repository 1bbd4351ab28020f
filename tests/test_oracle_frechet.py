"""Pins of the oracle's derivatives: the block-triangular Frechet derivative
of sgn against Daleckii-Krein and finite differences, and dA/dmu, dA/dU
against finite differences of Eq. 1.2."""
import numpy as np

from oracle import frechet as Fr
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    A += 0.5 * np.diag(np.sign(rng.standard_normal(n)))
    E = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A, E


def test_block_equals_daleckii_krein():
    A, E = _rand(30, 1)
    np.testing.assert_allclose(Fr.frechet_sign_block(A, E), Fr.frechet_sign_dk(A, E), atol=1e-10)


def test_block_equals_finite_differences():
    A, E = _rand(30, 2)
    h = 1e-6
    fd = (S.sign_spectral(A + h * E) - S.sign_spectral(A - h * E)) / (2 * h)
    L = Fr.frechet_sign_block(A, E)
    assert np.abs(L - fd).max() <= 1e-6 * np.abs(fd).max()


def test_frechet_properties():
    """L(A, A) = 0 (sgn is constant along A -> (1+t) A) and
    L(A, E) anticommutes-consistently: S L + L S = 0 from S^2 = 1."""
    A, E = _rand(24, 3)
    np.testing.assert_allclose(Fr.frechet_sign_block(A, A), 0, atol=1e-10)
    Sg = S.sign_spectral(A)
    L = Fr.frechet_sign_block(A, E)
    np.testing.assert_allclose(Sg @ L + L @ Sg, 0, atol=1e-9)


def test_dA_dmu_finite_difference():
    dims, mu, kappa = (2, 2, 2, 4), 0.3, 0.2
    U = synth.gauge_field(dims, 0.9, 4)
    h = 1e-6
    fd = (W.a_operator(U, dims, mu + h, kappa) - W.a_operator(U, dims, mu - h, kappa)) / (2 * h)
    np.testing.assert_allclose(Fr.dA_dmu(U, dims, mu, kappa).toarray(), fd.toarray(), atol=1e-8)


def test_dA_dU_finite_difference():
    dims, mu, kappa = (2, 2, 2, 4), 0.3, 0.2
    U = synth.gauge_field(dims, 0.9, 5)
    rng = np.random.default_rng(6)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    x = synth.gaussian_source(dims, 7)
    h = 1e-6
    fd = (W.a_operator(U + h * dU, dims, mu, kappa) @ x - W.a_operator(U - h * dU, dims, mu, kappa) @ x) / (2 * h)
    np.testing.assert_allclose(Fr.dA_dU_apply(U, dU, dims, mu, kappa, x), fd, atol=1e-7)
