"""Krylov approximations of sgn(A) b (Secs. 2-5), FP64, numpy.

* ``arnoldi``         -- A V_k = V_k H_k + beta_k v_{k+1} e_k^T, v_1 = b/|b|
                         (Sec. 2, Eq. 2.2-2.3); orthogonalisation by classical
                         Gram-Schmidt applied twice (the paper does not fix the
                         variant).
* ``sign_arnoldi``    -- y = |b| V_k f(H_k) e_1 (Eq. 2.6), with LR deflation
                         y = R f(Lambda) L^dag b + |b_perp| V_k f(H_k) e_1
                         (Sec. 3, Eq. 3.4).
* ``lanczos2``        -- two-sided Lanczos short recurrences (Sec. 4, Eq. 4.2):
                         beta_i v_{i+1}  = (A - alpha_i) v_i - gamma_{i-1} v_{i-1}
                         gamma_i^* w_{i+1} = (A^dag - alpha_i^*) w_i - beta_{i-1}^* w_{i-1}
                         alpha_i = w_i^dag A v_i, and w_{i+1}^dag v_{i+1} = 1.
                         The split of beta_i gamma_i = w_hat^dag v_hat is not fixed by
                         the paper; here beta_i = |v_hat|, gamma_i = w_hat^dag v_hat / beta_i.
* ``sign_lanczos2``   -- y = |b| V_k f(G_k) e_1 (Eq. 4.4); deflated
                         y = R f(Lambda) L^dag b + |b_perp^R| V_k f(G_k) e_1 with
                         b_perp^R = (1 - R L^dag) b, b_perp^L = (1 - L R^dag) b (Eq. 4.5).
                         Deflated start vectors: v_1 = b_perp^R/|b_perp^R| and
                         w_1 = b_perp^L / conj(b_perp^L^dag v_1), so that w_1^dag v_1 = 1.
* ``sign_arnoldi_restarted`` -- the Arnoldi approximation restarted every m steps with a
                         basis of m + 1 vectors (the restart the paper's discussion of the
                         N k^2 basis cost in Sec. 5 calls for; the paper gives no scheme).  The
                         restart follows Eiermann and Ernst (SIAM J. Numer. Anal. 44, 2006):
                         cycle c continues from the last basis vector of cycle c - 1, its
                         Hessenberg block joins the accumulated matrix H_c (block lower
                         bidiagonal, upper Hessenberg), and y gains |b| V_c [f(H_c) e_1] over
                         the rows of cycle c (the earlier rows of f(H_c) e_1 equal those of
                         f(H_{c-1}) e_1 because H_c is block lower triangular).  The inner sign
                         of H_c is Roberts' iteration: H_c is far from normal and its spectral
                         evaluation loses all accuracy after a few cycles.
* ``sign_lanczos2_twopass`` -- the two-pass procedure mentioned in Sec. 5:
                         pass 1 keeps only alpha, beta, gamma; pass 2 regenerates
                         v_i from them and accumulates y.

``matvec``/``rmatvec`` are callables applying A and A^dag.  The inner
function f(H_k), f(G_k) defaults to the spectral sign (Eq. 1.3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .sign import csign, sign_newton, sign_spectral

__all__ = [
    "Deflation",
    "KrylovBreakdown",
    "arnoldi",
    "lanczos2",
    "tridiag",
    "inner_sign_e1",
    "sign_arnoldi",
    "sign_arnoldi_restarted",
    "sign_lanczos2",
    "sign_lanczos2_twopass",
    "overlap_from_sign",
]


class KrylovBreakdown(ArithmeticError):
    """Serious breakdown of the two-sided Lanczos process: w_hat^dag v_hat = 0
    with v_hat, w_hat nonzero."""

    def __init__(self, step, msg="two-sided Lanczos serious breakdown"):
        super().__init__(f"{msg} at step {step}")
        self.step = step


@dataclass
class Deflation:
    """Critical eigenpairs: A R = R Lambda, L^dag A = Lambda L^dag, L^dag R = I (Sec. 3)."""

    lam: np.ndarray  # (m,)
    R: np.ndarray    # (N, m)
    L: np.ndarray    # (N, m)

    @property
    def m(self) -> int:
        return int(self.lam.shape[0])


def _inner(M: np.ndarray, inner: str) -> np.ndarray:
    if inner == "spectral":
        return sign_spectral(M)
    if inner == "newton":
        return sign_newton(M)
    raise ValueError(inner)


def inner_sign_e1(M: np.ndarray, inner: str = "spectral") -> np.ndarray:
    """First column of sgn(M) for the projected k x k matrix."""
    if M.shape[0] == 0:
        return np.zeros(0, dtype=np.complex128)
    return _inner(M, inner)[:, 0]


def arnoldi(matvec, b: np.ndarray, k: int, lucky_tol: float = 1e-14):
    """Arnoldi process (Sec. 2).  Returns (V[N, j+1], H[j+1, j], |b|) with
    j <= k the number of steps taken (j < k only on a lucky breakdown,
    where K_j(A, b) is invariant and the last column of V is zero)."""
    b = np.asarray(b, dtype=np.complex128)
    N = b.shape[0]
    nb = np.linalg.norm(b)
    V = np.zeros((N, k + 1), dtype=np.complex128)
    H = np.zeros((k + 1, k), dtype=np.complex128)
    if nb == 0 or k == 0:
        return V[:, :1], H[:1, :0], nb
    V[:, 0] = b / nb
    anorm = 0.0
    for j in range(k):
        w = matvec(V[:, j])
        anorm = max(anorm, np.linalg.norm(w))
        h = V[:, : j + 1].conj().T @ w
        w = w - V[:, : j + 1] @ h
        h2 = V[:, : j + 1].conj().T @ w
        w = w - V[:, : j + 1] @ h2
        H[: j + 1, j] = h + h2
        hn = np.linalg.norm(w)
        H[j + 1, j] = hn
        if hn <= lucky_tol * max(anorm, 1.0):
            return V[:, : j + 2], H[: j + 2, : j + 1], nb
        V[:, j + 1] = w / hn
    return V, H, nb


def lanczos2(matvec, rmatvec, v1: np.ndarray, w1: np.ndarray, k: int,
             lucky_tol: float = 1e-14, breakdown_tol: float = 1e-14):
    """Two-sided Lanczos (Sec. 4, Eq. 4.2), with w1^dag v1 = 1 on entry.

    Returns (V[N, j], W[N, j], alpha[j], beta[j-1], gamma[j-1]), j <= k the
    steps taken (j < k on a lucky breakdown, v_hat = 0).  Raises
    ``KrylovBreakdown`` on a serious breakdown.
    """
    N = v1.shape[0]
    V = np.zeros((N, k), dtype=np.complex128)
    W = np.zeros((N, k), dtype=np.complex128)
    alpha = np.zeros(k, dtype=np.complex128)
    beta = np.zeros(max(k - 1, 0), dtype=np.complex128)
    gamma = np.zeros(max(k - 1, 0), dtype=np.complex128)
    if k == 0:
        return V, W, alpha, beta, gamma
    V[:, 0] = v1
    W[:, 0] = w1
    anorm = 0.0
    for i in range(k):
        t = matvec(V[:, i])
        s = rmatvec(W[:, i])
        anorm = max(anorm, np.linalg.norm(t))
        alpha[i] = np.vdot(W[:, i], t)
        if i == k - 1:
            break
        vh = t - alpha[i] * V[:, i]
        wh = s - np.conj(alpha[i]) * W[:, i]
        if i > 0:
            vh -= gamma[i - 1] * V[:, i - 1]
            wh -= np.conj(beta[i - 1]) * W[:, i - 1]
        nv = np.linalg.norm(vh)
        if nv <= lucky_tol * max(anorm, 1.0):
            j = i + 1
            return V[:, :j], W[:, :j], alpha[:j], beta[: j - 1], gamma[: j - 1]
        delta = np.vdot(wh, vh)
        if abs(delta) <= breakdown_tol * nv * np.linalg.norm(wh):
            raise KrylovBreakdown(i + 1)
        beta[i] = nv
        gamma[i] = delta / nv
        V[:, i + 1] = vh / beta[i]
        W[:, i + 1] = wh / np.conj(gamma[i])
    return V, W, alpha, beta, gamma


def tridiag(alpha, beta, gamma) -> np.ndarray:
    """G_k with alpha on the diagonal, beta below and gamma above (Sec. 4, Eq. 4.1)."""
    G = np.diag(np.asarray(alpha, dtype=np.complex128))
    if len(beta):
        G += np.diag(beta, -1) + np.diag(gamma, 1)
    return G


def _split(b, defl: Deflation | None):
    """Deflated pieces of the source (Sec. 3 and Sec. 4):
    exact = R sgn(Lambda) L^dag b, b_R = (1 - R L^dag) b, b_L = (1 - L R^dag) b."""
    if defl is None or defl.m == 0:
        return np.zeros_like(b), b, b
    p = defl.L.conj().T @ b
    q = defl.R.conj().T @ b
    exact = defl.R @ (csign(defl.lam) * p)
    return exact, b - defl.R @ p, b - defl.L @ q


def sign_arnoldi(matvec, b, k: int, defl: Deflation | None = None,
                 inner: str = "spectral", return_info: bool = False):
    """sgn(A) b by the (deflated) Arnoldi approximation, Eq. 2.6 / Eq. 3.4."""
    b = np.asarray(b, dtype=np.complex128)
    exact, bperp, _ = _split(b, defl)
    V, H, nb = arnoldi(matvec, bperp, k)
    j = H.shape[1]
    c = inner_sign_e1(H[:j, :j], inner)
    y = exact + nb * (V[:, :j] @ c)
    if return_info:
        return y, {"k_used": j, "H": H[:j, :j], "V": V[:, :j], "c": nb * c}
    return y


def sign_arnoldi_restarted(matvec, b, m: int, cycles: int, defl: Deflation | None = None,
                           inner: str = "newton", return_info: bool = False):
    """sgn(A) b by Arnoldi restarted every m steps (at most cycles cycles, cycles * m steps in all);
    with LR deflation the restarted process runs on b_perp (Sec. 3, Eq. 3.4)."""
    b = np.asarray(b, dtype=np.complex128)
    exact, bperp, _ = _split(b, defl)
    nb = np.linalg.norm(bperp)
    y = exact.copy()
    if nb == 0 or m == 0 or cycles == 0:
        return (y, {"k_used": 0, "H": np.zeros((0, 0), complex)}) if return_info else y
    Ht = np.zeros((cycles * m + 1, cycles * m), dtype=np.complex128)
    v = bperp / nb
    K = 0
    for _ in range(cycles):
        V, H, _ = arnoldi(matvec, v, m)
        j = H.shape[1]                       # steps of this cycle (< m on a lucky breakdown)
        Ht[K:K + j + 1, K:K + j] = H         # includes the coupling entry H[j, j-1] below the block
        f = inner_sign_e1(Ht[:K + j, :K + j], inner)
        y = y + nb * (V[:, :j] @ f[K:K + j])
        K += j
        if j < m or H[j, j - 1] == 0:        # invariant Krylov space: the approximation is final
            break
        v = V[:, j]
    if return_info:
        return y, {"k_used": K, "H": Ht[:K, :K]}
    return y


def _lanczos_start(b, defl):
    exact, bR, bL = _split(b, defl)
    nR = np.linalg.norm(bR)
    if nR == 0:
        return exact, None, None, 0.0
    v1 = bR / nR
    d = np.vdot(bL, v1)
    if d == 0:
        raise KrylovBreakdown(0, "deflated start vectors are biorthogonal")
    w1 = bL / np.conj(d)
    return exact, v1, w1, nR


def sign_lanczos2(matvec, rmatvec, b, k: int, defl: Deflation | None = None,
                  inner: str = "spectral", return_info: bool = False):
    """sgn(A) b by the (deflated) two-sided Lanczos approximation, Eq. 4.4 / Eq. 4.5."""
    b = np.asarray(b, dtype=np.complex128)
    exact, v1, w1, nR = _lanczos_start(b, defl)
    if v1 is None or k == 0:
        return (exact, {"k_used": 0}) if return_info else exact
    V, W, a, be, ga = lanczos2(matvec, rmatvec, v1, w1, k)
    G = tridiag(a, be, ga)
    c = inner_sign_e1(G, inner)
    y = exact + nR * (V @ c)
    if return_info:
        return y, {"k_used": len(a), "alpha": a, "beta": be, "gamma": ga,
                   "V": V, "W": W, "c": nR * c}
    return y


def sign_lanczos2_twopass(matvec, rmatvec, b, k: int, defl: Deflation | None = None,
                          inner: str = "spectral", coeffs=None):
    """Two-pass two-sided Lanczos (Sec. 5): pass 1 computes only the
    coefficients alpha, beta, gamma (or takes them from ``coeffs``); pass 2
    regenerates v_{i+1} = ((A - alpha_i) v_i - gamma_{i-1} v_{i-1}) / beta_i
    and accumulates y = R sgn(Lambda) L^dag b + |b_perp^R| sum_i c_i v_i."""
    b = np.asarray(b, dtype=np.complex128)
    exact, v1, w1, nR = _lanczos_start(b, defl)
    if v1 is None or k == 0:
        return exact
    if coeffs is None:
        _, _, a, be, ga = lanczos2(matvec, rmatvec, v1, w1, k)
    else:
        a, be, ga = coeffs
    c = nR * inner_sign_e1(tridiag(a, be, ga), inner)
    y = exact + c[0] * v1
    vprev, v = np.zeros_like(v1), v1
    for i in range(len(a) - 1):
        vn = matvec(v) - a[i] * v
        if i > 0:
            vn -= ga[i - 1] * vprev
        vn /= be[i]
        y += c[i + 1] * vn
        vprev, v = v, vn
    return y


def overlap_from_sign(b, sgn_b, gamma5_diag):
    """D_ov b = b + gamma5 sgn(A) b (Eq. 1.1)."""
    return b + gamma5_diag * sgn_b
