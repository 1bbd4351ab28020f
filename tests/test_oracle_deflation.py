"""Pins of the oracle's critical eigenpairs (Sec. 3, Eq. 3.1; Sec. 5)."""
import numpy as np
import pytest

from oracle import deflation as Dm
from oracle import wilson as W
from paper_0810_4228_gb300 import synth


def _A(dims, eps=0.8, seed=31, mu=0.3):
    U = synth.gauge_field(dims, eps, seed)
    return W.a_operator(U, dims, mu, 0.2)


def _check_pairs(A, d, tol):
    Ad = A @ d.R if not isinstance(A, np.ndarray) else A @ d.R
    np.testing.assert_allclose(Ad, d.R * d.lam, atol=tol)
    LA = (A.conj().T @ d.L).conj().T
    np.testing.assert_allclose(LA, d.lam[:, None] * d.L.conj().T, atol=tol)
    np.testing.assert_allclose(d.L.conj().T @ d.R, np.eye(d.m), atol=tol)


@pytest.mark.parametrize("select", ["re", "abs"])
def test_dense_pairs(select):
    A = _A((2, 2, 2, 4)).toarray()
    d = Dm.eigenpairs_dense(A, 16, select)
    _check_pairs(A, d, 1e-11)
    w = np.linalg.eigvals(A)
    key = np.abs(w.real) if select == "re" else np.abs(w)
    kd = np.abs(d.lam.real) if select == "re" else np.abs(d.lam)
    np.testing.assert_allclose(np.sort(kd), np.sort(key)[:16], atol=1e-12)


def test_arpack_matches_dense():
    dims = (4, 4, 2, 4)
    A = _A(dims, eps=1.0)
    d = Dm.eigenpairs_arpack(A, 10, select="re")
    _check_pairs(A, d, 1e-9)
    w = np.linalg.eigvals(A.toarray())
    # the selected eigenvalues are eigenvalues of A
    for l in d.lam:
        assert np.min(np.abs(w - l)) < 1e-9


def test_biorthonormalise():
    rng = np.random.default_rng(0)
    R = rng.standard_normal((50, 5)) + 1j * rng.standard_normal((50, 5))
    L = rng.standard_normal((50, 5)) + 1j * rng.standard_normal((50, 5))
    L2 = Dm.biorthonormalise(R, L)
    np.testing.assert_allclose(L2.conj().T @ R, np.eye(5), atol=1e-12)
    # the span of L is unchanged
    P = L @ np.linalg.pinv(L)
    np.testing.assert_allclose(P @ L2, L2, atol=1e-10)


def test_cluster_safe_m():
    key = np.array([0.1, 0.2, 0.2, 0.2 + 1e-14, 0.3])
    assert Dm.cluster_safe_m(key, 2) == 1
    assert Dm.cluster_safe_m(key, 4) == 4
    assert Dm.cluster_safe_m(key, 3) == 1
