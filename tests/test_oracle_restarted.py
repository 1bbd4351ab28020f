"""Pins of the oracle's restarted Arnoldi approximation (oracle.krylov.sign_arnoldi_restarted).

* One cycle is the plain Arnoldi approximation of Sec. 2 (Eq. 2.6).
* After c cycles of m steps the restarted approximation is p(A) b with p the polynomial of degree
  < c m that interpolates sgn at the eigenvalues of the accumulated Hessenberg matrix (the
  Eiermann-Ernst characterisation of restarted Krylov approximations of f(A) b); checked against
  that polynomial built directly in Lagrange form on the dense A of a 2^3 x 4 lattice.
* With LR deflation (Sec. 3) it converges to the dense sgn(A) b, geometrically in the cycles.
* A source in a two-dimensional invariant Krylov space (one free-field momentum) stops the
  process in the first cycle at the closed form.
"""
import numpy as np

from oracle import deflation as Dm
from oracle import freefield as F
from oracle import krylov as K
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

KAPPA = 0.2


def _case(eps=1.0, seed=61, mu=0.3):
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, eps, seed)
    A = W.a_operator(U, dims, mu, KAPPA)
    b = synth.gaussian_source(dims, 62)
    return A, A.toarray(), b


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_one_cycle_is_plain_arnoldi():
    A, _, b = _case()
    assert _rel(K.sign_arnoldi_restarted(A.dot, b, 25, 1), K.sign_arnoldi(A.dot, b, 25)) < 1e-13


def test_interpolates_sgn_at_the_accumulated_ritz_values():
    A, Ad, b = _case()
    y, info = K.sign_arnoldi_restarted(A.dot, b, 3, 4, return_info=True)
    th = np.linalg.eigvals(info["H"])
    assert len(th) == 12 and np.min(np.abs(th.real)) > 1e-3
    py = np.zeros_like(b)
    for i, t in enumerate(th):  # Lagrange basis polynomial l_i(A) b, then sgn(theta_i) l_i(A) b
        v = b.copy()
        for jj, tj in enumerate(th):
            if jj != i:
                v = (Ad @ v - tj * v) / (t - tj)
        py += S.csign(np.array([t]))[0] * v
    assert _rel(y, py) < 1e-9


def test_deflated_restart_converges_to_dense():
    A, Ad, b = _case()
    ref = S.sign_spectral(Ad) @ b
    d = Dm.eigenpairs_dense(Ad, 16)
    errs = [_rel(K.sign_arnoldi_restarted(A.dot, b, 30, c, d), ref) for c in (2, 4, 8, 12)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-10, errs


def test_invariant_krylov_space_stops_at_the_closed_form():
    dims, mu = (2, 2, 2, 4), 0.3
    V = 32
    t = np.arange(V) % 4
    rng = np.random.default_rng(5)
    spin = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    b = (np.exp(1j * np.pi * 3 * t / 4)[:, None] * spin[None, :]).reshape(-1)
    A = W.a_operator(synth.free_gauge_field(dims), dims, mu, KAPPA)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), V)
    ref = g5 * (F.overlap_free_apply(dims, mu, KAPPA, b) - b)
    y, info = K.sign_arnoldi_restarted(A.dot, b, 10, 5, return_info=True)
    assert info["k_used"] <= 2
    assert _rel(y, ref) < 1e-12
