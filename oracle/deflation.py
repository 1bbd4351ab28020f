"""Critical left/right eigenpairs for LR deflation (Sec. 3 and Sec. 5).

A R_m = R_m Lambda_m,  L_m^dag A = Lambda_m L_m^dag,  L_m^dag R_m = I_m
(Sec. 3, Eq. 3.1).  Two sources:

* ``eigenpairs_dense``: a full eigendecomposition A = X diag(lambda) X^-1;
  R = columns of X, L^dag = rows of X^-1, so L^dag R = I holds exactly.
* ``eigenpairs_arpack``: ARPACK (as in Sec. 5) in shift-invert mode about
  0, on A for the right and on A^dag for the left eigenvectors; the two
  sets are paired by lambda_left = conj(lambda_right) and made
  bi-orthonormal by L <- L (L^dag R)^-H.

The paper's deflation phase takes the eigenvalues of smallest magnitude
(Sec. 5); the critical ones for sgn are those nearest the imaginary axis.
``select`` chooses between the two orderings ("re": smallest |Re lambda|,
"abs": smallest |lambda|); the exact sgn(A) b does not depend on the
choice, only the Krylov size needed does.
"""
from __future__ import annotations

import numpy as np

from .krylov import Deflation

__all__ = ["eigenpairs_dense", "eigenpairs_arpack", "biorthonormalise", "cluster_safe_m"]


def _order(lam, select):
    if select == "re":
        return np.argsort(np.abs(lam.real), kind="stable")
    if select == "abs":
        return np.argsort(np.abs(lam), kind="stable")
    raise ValueError(select)


def cluster_safe_m(lam_sorted_key: np.ndarray, m: int, rtol: float = 1e-8) -> int:
    """Largest m' <= m that does not split a cluster of (numerically) equal
    selection keys; deflating half of a degenerate cluster is ill-posed."""
    m = min(m, len(lam_sorted_key))
    while 0 < m < len(lam_sorted_key) and abs(lam_sorted_key[m] - lam_sorted_key[m - 1]) <= rtol * max(abs(lam_sorted_key[m]), 1e-300):
        m -= 1
    return m


def biorthonormalise(R: np.ndarray, L: np.ndarray) -> np.ndarray:
    """L <- L (L^dag R)^-H, so that the new L^dag R = I."""
    M = L.conj().T @ R
    return L @ np.linalg.inv(M).conj().T


def eigenpairs_dense(A: np.ndarray, m: int, select: str = "re") -> Deflation:
    A = np.asarray(A, dtype=np.complex128)
    lam, X = np.linalg.eig(A)
    Xinv = np.linalg.inv(X)
    idx = _order(lam, select)[:m]
    return Deflation(lam=lam[idx].copy(), R=X[:, idx].copy(), L=Xinv[idx, :].conj().T.copy())


def eigenpairs_arpack(A, m: int, select: str = "re", extra: int | None = None,
                      tol: float = 1e-12, seed: int = 0, permc_spec: str = "MMD_AT_PLUS_A") -> Deflation:
    """Right and left eigenpairs of the sparse A near 0 by ARPACK shift-invert.

    The inverse is applied through a sparse LU factorisation of A; ``permc_spec`` is its column
    ordering (the same factors up to rounding for any ordering; a minimum-degree ordering of
    A^T + A suits the structurally symmetric stencil and keeps the fill several times smaller
    than the unsymmetric COLAMD default on 4D lattices)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    A = sp.csc_matrix(A, dtype=np.complex128)
    n_ev = m + (extra if extra is not None else max(4, m // 2))
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    lu = sla.splu(A, permc_spec=permc_spec)
    op = sla.LinearOperator(A.shape, matvec=lu.solve, dtype=np.complex128)
    opH = sla.LinearOperator(A.shape, matvec=lambda x: lu.solve(x, trans="H"),
                             dtype=np.complex128)
    mu_r, Rv = sla.eigs(op, k=n_ev, v0=v0, tol=tol, which="LM")
    mu_l, Lv = sla.eigs(opH, k=n_ev, v0=v0, tol=tol, which="LM")
    lam_r = 1.0 / mu_r
    lam_l = np.conj(1.0 / mu_l)
    order = _order(lam_r, select)
    key = (np.abs(lam_r.real) if select == "re" else np.abs(lam_r))[order]
    m = cluster_safe_m(key, m)
    idx = order[:m]
    R = Rv[:, idx]
    lam = lam_r[idx]
    L = np.empty_like(R)
    for j, l in enumerate(lam):
        i = int(np.argmin(np.abs(lam_l - l)))
        L[:, j] = Lv[:, i]
    return Deflation(lam=lam.copy(), R=R.copy(), L=biorthonormalise(R, L))
