"""Pins of the oracle's sign function (Sec. 1 Eq. 1.3-1.4, Sec. 2 Roberts
iteration) and of the dense overlap operator (Eq. 1.1)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import freefield as F
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth


def test_complex_sign_scalar():
    rng = np.random.default_rng(0)
    z = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    s = S.csign(z)
    np.testing.assert_allclose(s, np.sign(z.real), atol=1e-15)
    np.testing.assert_allclose(s * s, 1, atol=1e-15)
    np.testing.assert_allclose(S.csign(np.array([3.0, -2.5])), [1, -1])


def _random_nonhermitian(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A / np.sqrt(n) + 0.3 * np.diag(np.sign(rng.standard_normal(n)))


def test_spectral_sign_identities():
    A = _random_nonhermitian(60, 1)
    Sg = S.sign_spectral(A)
    np.testing.assert_allclose(Sg @ Sg, np.eye(60), atol=1e-11)
    np.testing.assert_allclose(A @ Sg, Sg @ A, atol=1e-11)


def test_spectral_sign_equals_A_invsqrt_A2():
    """sgn(A) = A (A^2)^(-1/2) with the principal square root (scipy.sqrtm)."""
    A = _random_nonhermitian(40, 2)
    ref = A @ np.linalg.inv(sla.sqrtm(A @ A))
    np.testing.assert_allclose(S.sign_spectral(A), ref, atol=1e-10)


def test_hermitian_special_case():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((50, 50)) + 1j * rng.standard_normal((50, 50))
    H = M + M.conj().T
    w, X = np.linalg.eigh(H)
    ref = (X * np.sign(w)) @ X.conj().T
    np.testing.assert_allclose(S.sign_spectral(H), ref, atol=1e-11)
    np.testing.assert_allclose(S.sign_newton(H), ref, atol=1e-11)


def test_diagonal_and_scalar_cases():
    d = np.array([2 + 5j, -0.1 + 3j, 0.5 - 0.5j, -7.0])
    np.testing.assert_allclose(S.sign_spectral(np.diag(d)), np.diag(np.sign(d.real)), atol=1e-15)
    np.testing.assert_allclose(S.sign_newton(np.diag(d)), np.diag(np.sign(d.real)), atol=1e-13)
    assert S.sign_spectral(np.zeros((0, 0))).shape == (0, 0)


@pytest.mark.parametrize("scaled", [True, False])
def test_newton_equals_spectral(scaled):
    A = _random_nonhermitian(80, 4)
    Sn, it = S.sign_newton(A, scaled=scaled, return_iters=True)
    np.testing.assert_allclose(Sn, S.sign_spectral(A), atol=1e-11)
    assert it < 40


def test_newton_on_jordan_block():
    """Roberts' iteration handles a non-diagonalisable matrix (Jordan block):
    sgn of [[l, 1], [0, l]] with Re l > 0 is the identity."""
    J = np.array([[0.5 + 1j, 1.0], [0.0, 0.5 + 1j]])
    np.testing.assert_allclose(S.sign_newton(J), np.eye(2), atol=1e-13)


def test_sign_undefined_on_imaginary_axis():
    with pytest.raises(S.SignError):
        S.sign_spectral(np.diag([1.0, 2j]))


def _lattice_A(dims, mu, eps, seed, kappa=0.2):
    U = synth.gauge_field(dims, eps, seed) if eps > 0 else synth.free_gauge_field(dims)
    return U, W.dense_a(U, dims, mu, kappa)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_ginsparg_wilson(mu):
    """gamma5 D + D gamma5 = D gamma5 D for D = D_ov (Sec. 1)."""
    dims = (2, 2, 2, 4)
    _, A = _lattice_A(dims, mu, 0.8, seed=21)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), 32)
    D = S.overlap_dense(A, g5)
    G5 = np.diag(g5)
    np.testing.assert_allclose(G5 @ D + D @ G5, D @ G5 @ D, atol=1e-10)


def test_sign_squares_to_one_on_lattice():
    dims = (2, 2, 2, 4)
    _, A = _lattice_A(dims, 0.3, 0.8, seed=22)
    Sg = S.sign_spectral(A)
    np.testing.assert_allclose(Sg @ Sg, np.eye(A.shape[0]), atol=1e-10)
    np.testing.assert_allclose(S.sign_newton(A), Sg, atol=1e-10)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_dense_overlap_free_field(mu):
    """Dense D_ov on U = 1 equals the momentum-space closed form."""
    dims, kappa = (2, 2, 2, 4), 0.2
    _, A = _lattice_A(dims, mu, 0.0, 0, kappa)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), 32)
    Sg = S.sign_newton(A)  # free spectrum is highly degenerate; Newton is robust there
    b = synth.gaussian_source(dims, seed=5)
    ref = F.overlap_free_apply(dims, mu, kappa, b)
    np.testing.assert_allclose(b + g5 * (Sg @ b), ref, atol=1e-11)


def test_dense_overlap_gauge_transformed_free_field():
    """A gauge transform of U = 1: D_ov[U'] G b = G D_ov[1] b (closed form)."""
    dims, mu, kappa = (2, 2, 2, 4), 0.3, 0.2
    V = 32
    g = synth.gauge_transformation(dims, seed=8)
    fwd, _, _, _ = W.neighbours(dims)
    Up = np.einsum("vab,vdb->vad", g[:, None].repeat(4, 1).reshape(-1, 3, 3),
                   g[fwd].reshape(-1, 3, 3).conj()).reshape(V, 4, 3, 3)
    A = W.dense_a(Up, dims, mu, kappa)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), V)
    b = synth.gaussian_source(dims, seed=6)
    Gb = np.einsum("vab,vsb->vsa", g, b.reshape(V, 4, 3)).reshape(-1)
    lhs = Gb + g5 * (S.sign_newton(A) @ Gb)
    ref = F.overlap_free_apply(dims, mu, kappa, b)
    rhs = np.einsum("vab,vsb->vsa", g, ref.reshape(V, 4, 3)).reshape(-1)
    np.testing.assert_allclose(lhs, rhs, atol=1e-11)
