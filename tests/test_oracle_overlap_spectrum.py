"""Pins of the overlap operator's spectrum in the oracle (Eq. 1.1): at mu = 0 the operator is
1 + gamma5 sgn(H) with H = gamma5 D_w Hermitian, i.e. 1 + a unitary, so every eigenvalue lies on
the circle |lambda - 1| = 1; on the free field at nonzero mu every momentum block is the closed
form 1 + (a - i gamma.s) / sqrt(a^2 + s.s), whose eigenvalues are 1 + (a -+ i r) / sqrt(a^2 + r^2),
r = sqrt(s.s), each twice in spin and three times in colour."""
import numpy as np
from scipy.optimize import linear_sum_assignment

from oracle import freefield as F
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

KAPPA = 0.2


def _g5(V):
    return np.tile(np.repeat([1.0, 1, -1, -1], 3), V)


def test_zero_mu_spectrum_on_the_circle():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 1.0, 501)
    A = W.dense_a(U, dims, 0.0, KAPPA)
    w = S.overlap_eigenvalues(A, _g5(32))
    np.testing.assert_allclose(np.abs(w - 1.0), 1.0, atol=1e-12)
    assert np.all(np.diff(np.abs(w)) >= -1e-15)  # nearest 0 first


def test_free_field_spectrum_closed_form():
    dims, mu = (2, 2, 2, 4), 0.3
    V = 32
    A = W.dense_a(synth.free_gauge_field(dims), dims, mu, KAPPA)
    w = S.overlap_eigenvalues(A, _g5(V))
    m_w = 1.0 / (2 * KAPPA) - 4.0
    ref = []
    for p in F.momenta(dims):
        pt = p.astype(np.complex128)
        pt[3] -= 1j * mu
        a = m_w + np.sum(1 - np.cos(pt))
        r = np.sqrt(np.sum(np.sin(pt) ** 2))
        for lam in (1 + (a - 1j * r) / np.sqrt(a * a + r * r), 1 + (a + 1j * r) / np.sqrt(a * a + r * r)):
            ref += [lam] * 6
    ref = np.array(ref)
    assert w.shape == ref.shape
    cost = np.abs(w[:, None] - ref[None, :])
    i, j = linear_sum_assignment(cost)
    assert cost[i, j].max() < 1e-9
    # off the circle at nonzero mu (the spectrum is not that of 1 + a unitary)
    assert np.abs(np.abs(w - 1.0) - 1.0).max() > 1e-3
