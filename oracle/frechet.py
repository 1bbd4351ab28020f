"""Derivatives of the sign function and of A = gamma5 D_w(mu).

* ``frechet_sign_block``: the Frechet derivative L(A, E) of sgn at A in
  direction E, read from the upper-right block of
  sgn([[A, E], [0, A]]) = [[sgn A, L(A, E)], [0, sgn A]].  The block
  matrix is defective in general, so its sign is taken with Roberts'
  iteration (Sec. 2), which needs no eigenvectors.
* ``frechet_sign_dk``: the same derivative for diagonalisable A by the
  Daleckii-Krein formula L = X ((X^-1 E X) o Phi) X^-1 with
  Phi_ij = (sgn l_i - sgn l_j)/(l_i - l_j) and Phi_ii = 0 (sgn is locally
  constant), a second route used to pin the first.
* ``dA_dmu``: dA/dmu = -kappa gamma5 (e^mu T_4^+ - e^-mu T_4^-), from
  Eq. 1.2 (only the temporal hops depend on mu).
* ``dA_dU_apply``: the directional derivative of A x with respect to the
  link field, for a perturbation dU (same shape as U).  A is linear in the
  links: each hop uses either U_{x,nu} or U_{x-nu,nu}^dag.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .sign import sign_newton, csign
from .wilson import gamma5_operator, hop_term, wilson_dirac

__all__ = ["frechet_sign_block", "frechet_sign_dk", "dA_dmu", "dA_dU_apply"]


def frechet_sign_block(A: np.ndarray, E: np.ndarray) -> np.ndarray:
    n = A.shape[0]
    B = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    B[:n, :n] = A
    B[n:, n:] = A
    B[:n, n:] = E
    return sign_newton(B)[:n, n:]


def frechet_sign_dk(A: np.ndarray, E: np.ndarray) -> np.ndarray:
    lam, X = np.linalg.eig(A)
    Xi = np.linalg.inv(X)
    s = csign(lam)
    dl = lam[:, None] - lam[None, :]
    ds = s[:, None] - s[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        Phi = np.where(np.abs(dl) > 0, ds / np.where(dl == 0, 1, dl), 0.0)
    return X @ ((Xi @ E @ X) * Phi) @ Xi


def dA_dmu(U, dims, mu: float, kappa: float, bc_t: int = -1) -> sp.csr_matrix:
    """dA/dmu for A = gamma5 D_w(mu): only the temporal hops of Eq. 1.2
    carry e^{+-mu}, so dD_w/dmu = -kappa (e^mu T_4^+ - e^-mu T_4^-)."""
    V = int(np.prod(dims))
    dD = -kappa * (np.exp(mu) * hop_term(U, dims, 3, +1, bc_t)
                   - np.exp(-mu) * hop_term(U, dims, 3, -1, bc_t))
    return (gamma5_operator(V) @ dD).tocsr()


def dA_dU_apply(U, dU, dims, mu: float, kappa: float, x, bc_t: int = -1):
    """(dA/dU)[dU] x: A is linear in the pair (U, U^dag) hop by hop; the
    forward hop uses U_{x,nu} and the backward hop U_{x-nu,nu}^dag, so the
    derivative is the hopping part of A built from dU in the forward and
    dU^dag in the backward hop, i.e. A[U + dU] - A[U] without the diagonal
    (linear in dU for the forward, conjugate-linear for the backward term)."""
    V = int(np.prod(dims))
    I = sp.identity(12 * V, dtype=np.complex128, format="csr")
    g5 = gamma5_operator(V)
    hop_dU = g5 @ (wilson_dirac(dU, dims, mu, kappa, bc_t) - I)
    return hop_dU @ x
