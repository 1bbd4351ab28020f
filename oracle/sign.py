"""Matrix sign function of a non-Hermitian matrix (Sec. 1 and Sec. 2).

* ``csign``: the sign of a complex number, sgn z = z / sqrt(z^2), the
  square root taking its branch cut on the negative real axis (Eq. 1.4);
  equal to sgn(Re z) off the imaginary axis.
* ``sign_spectral``: the spectral definition f(A) = U diag(f(lambda_i)) U^-1
  (Eq. 1.3) with f = sgn.
* ``sign_newton``: Roberts' iteration S <- (S + S^-1)/2, S^0 = A
  (Sec. 2, the unnumbered display after Eq. 2.6), optionally with
  |det S|^(-1/n) scaling of the first iterates (the iteration converges to
  the same limit; scaling only shortens the initial phase).
* ``overlap_dense``: D_ov = 1 + gamma5 sgn(gamma5 D_w) (Eq. 1.1).
* ``overlap_eigenvalues``: the spectrum of that D_ov, nearest 0 first (the eigenvalue problem
  the closing remark of Sec. 5 names as the methods' next application; the paper gives no
  method for it, so the definition is the dense eigendecomposition).
"""
from __future__ import annotations

import numpy as np

__all__ = ["csign", "sign_spectral", "sign_newton", "overlap_dense", "overlap_eigenvalues", "SignError"]


class SignError(ArithmeticError):
    """sgn is undefined: an eigenvalue lies on the imaginary axis (the
    branch cut of Eq. 1.4), or the Newton iteration did not converge."""


def csign(z):
    """sgn z = z / sqrt(z^2), principal square root (Eq. 1.4)."""
    z = np.asarray(z, dtype=np.complex128)
    return z / np.sqrt(z * z)


def sign_spectral(A: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """sgn(A) = X diag(sgn lambda_i) X^-1 from a full eigendecomposition (Eq. 1.3)."""
    A = np.asarray(A, dtype=np.complex128)
    if A.shape[0] == 0:
        return A.copy()
    w, X = np.linalg.eig(A)
    scale = max(np.abs(w).max(), 1e-300)
    if np.abs(w.real).min() < tol * scale:
        raise SignError("eigenvalue on the imaginary axis: sgn undefined")
    s = csign(w)
    # X diag(s) X^-1, computed as a solve instead of an explicit inverse
    return np.linalg.solve(X.T, (X * s[None, :]).T).T


def sign_newton(A: np.ndarray, scaled: bool = True, rtol: float = 1e-14,
                maxit: int = 100, n_scaled: int = 8, return_iters: bool = False):
    """Roberts' matrix iteration S^{n+1} = (S^n + (S^n)^-1)/2, S^0 = A (Sec. 2).

    With ``scaled`` the first ``n_scaled`` iterates are multiplied by
    c_n = |det S^n|^(-1/n) before the update (determinant scaling).
    The iteration converges quadratically, so once an update changes S by
    at most sqrt(rtol) ||S||_F one more update brings the change to about
    rtol; that final update is taken and S returned.
    """
    S = np.array(A, dtype=np.complex128)
    n = S.shape[0]
    if n == 0:
        return (S, 0) if return_iters else S
    for it in range(1, maxit + 1):
        if scaled and it <= n_scaled:
            _, logdet = np.linalg.slogdet(S)
            S = np.exp(-logdet.real / n) * S
        Sn = 0.5 * (S + np.linalg.inv(S))
        diff = np.linalg.norm(Sn - S)
        S = Sn
        if diff <= np.sqrt(rtol) * np.linalg.norm(S):
            S = 0.5 * (S + np.linalg.inv(S))
            return (S, it + 1) if return_iters else S
    raise SignError("Newton iteration for sgn did not converge")


def overlap_dense(A: np.ndarray, gamma5_diag: np.ndarray, sign=None) -> np.ndarray:
    """D_ov = 1 + gamma5 sgn(A) with A = gamma5 D_w (Eq. 1.1).

    ``gamma5_diag`` is the diagonal of gamma5 on the whole lattice.
    """
    S = sign_spectral(A) if sign is None else sign
    return np.eye(A.shape[0], dtype=np.complex128) + gamma5_diag[:, None] * S


def overlap_eigenvalues(A: np.ndarray, gamma5_diag: np.ndarray, sign=None) -> np.ndarray:
    """All eigenvalues of D_ov = 1 + gamma5 sgn(A) (Eq. 1.1), sorted by modulus (nearest 0 first)."""
    w = np.linalg.eigvals(overlap_dense(A, gamma5_diag, sign))
    return w[np.argsort(np.abs(w), kind="stable")]
