"""Closed form of D_w(mu) and D_ov(mu) on the free field U = 1.

For U = 1 the operator of Eq. 1.2 is diagonal in momentum space.  On the
plane wave psi(x) = exp(i p.x) u (u a spinor, any colour), with
p_k = 2 pi n_k / L_k (k = 1, 2, 3) and p_4 = (2 n_4 + theta) pi / L_4
(theta = 1 for antiperiodic, 0 for periodic time), the hops give
e^{+-mu} e^{+-i p_4} = e^{+-i (p_4 - i mu)}, so with
    p~_k = p_k,  p~_4 = p_4 - i mu,
    a = m_w + sum_nu (1 - cos p~_nu),   s_nu = sin p~_nu,
one has
    D_w(p)   = 2 kappa (a - i gamma.s),
    A(p)^2   = (gamma5 D_w(p))^2 = 4 kappa^2 (a^2 + s.s) * 1,
    sgn A(p) = A(p) / (2 kappa sqrt(a^2 + s.s))   (principal root, Eq. 1.4),
    D_ov(p)  = 1 + (a - i gamma.s) / sqrt(a^2 + s.s).
The eigenvalues of D_w(p) are 2 kappa (a +- i sqrt(s.s)).

``overlap_free_apply`` applies D_ov to any vector by FFT, which pins the
iterative and dense sign at any volume.  The hop convention is the one
stated in ``oracle.wilson``.
"""
from __future__ import annotations

import numpy as np

from .wilson import gamma_matrices

__all__ = ["momenta", "dw_momentum", "overlap_momentum", "dw_eigenvalues",
           "plane_wave", "overlap_free_apply", "dw_free_apply"]


def momenta(dims, bc_t: int = -1):
    """All lattice momenta, shape (V, 4), in canonical site order of the FFT grid."""
    L = tuple(int(x) for x in dims)
    n = np.indices(L).reshape(4, -1).T.astype(np.float64)
    p = 2 * np.pi * n / np.array(L, dtype=np.float64)
    if bc_t == -1:
        p[:, 3] += np.pi / L[3]
    return p


def _a_s(p, mu, m_w):
    p = np.asarray(p, dtype=np.complex128)
    pt = p.copy()
    pt[..., 3] = pt[..., 3] - 1j * mu
    a = m_w + np.sum(1 - np.cos(pt), axis=-1)
    s = np.sin(pt)
    return a, s


def dw_momentum(p, mu: float, kappa: float) -> np.ndarray:
    """D_w(p) as a 4x4 spin matrix (identity in colour)."""
    m_w = 1.0 / (2 * kappa) - 4.0
    a, s = _a_s(p, mu, m_w)
    g = gamma_matrices()
    return 2 * kappa * (a * np.eye(4) - 1j * np.einsum("n,nij->ij", s, g))


def overlap_momentum(p, mu: float, kappa: float) -> np.ndarray:
    """D_ov(p) = 1 + (a - i gamma.s) / sqrt(a^2 + s.s) as a 4x4 spin matrix."""
    m_w = 1.0 / (2 * kappa) - 4.0
    a, s = _a_s(p, mu, m_w)
    g = gamma_matrices()
    r = np.sqrt(a * a + np.dot(s, s))
    return np.eye(4) + (a * np.eye(4) - 1j * np.einsum("n,nij->ij", s, g)) / r


def dw_eigenvalues(p, mu: float, kappa: float):
    m_w = 1.0 / (2 * kappa) - 4.0
    a, s = _a_s(p, mu, m_w)
    r = np.sqrt(np.dot(s, s))
    return 2 * kappa * (a + 1j * r), 2 * kappa * (a - 1j * r)


def plane_wave(dims, p, u, colour: int = 0) -> np.ndarray:
    """exp(i p.x) u (x) e_colour as a flat (12V,) vector."""
    L = tuple(int(x) for x in dims)
    x = np.indices(L).reshape(4, -1).T
    ph = np.exp(1j * (x @ np.asarray(p, dtype=np.float64)))
    psi = np.zeros((x.shape[0], 4, 3), dtype=np.complex128)
    psi[:, :, colour] = ph[:, None] * np.asarray(u)[None, :]
    return psi.reshape(-1)


def _apply_momentum_matrix(dims, mats_fn, b, bc_t):
    L = tuple(int(x) for x in dims)
    psi = np.asarray(b, dtype=np.complex128).reshape(L + (4, 3))
    x4 = np.arange(L[3])
    twist = np.exp(1j * np.pi * x4 / L[3]) if bc_t == -1 else np.ones(L[3])
    phi = psi / twist[None, None, None, :, None, None]
    phik = np.fft.fftn(phi, axes=(0, 1, 2, 3))
    p = momenta(L, bc_t).reshape(L + (4,))
    out = np.empty_like(phik)
    for idx in np.ndindex(*L):
        out[idx] = mats_fn(p[idx]) @ phik[idx]
    res = np.fft.ifftn(out, axes=(0, 1, 2, 3)) * twist[None, None, None, :, None, None]
    return res.reshape(-1)


def overlap_free_apply(dims, mu: float, kappa: float, b, bc_t: int = -1):
    """D_ov(mu) b on the free field, by FFT and the 4x4 closed form."""
    return _apply_momentum_matrix(dims, lambda p: overlap_momentum(p, mu, kappa), b, bc_t)


def dw_free_apply(dims, mu: float, kappa: float, b, bc_t: int = -1):
    """D_w(mu) b on the free field, by FFT and the 4x4 closed form."""
    return _apply_momentum_matrix(dims, lambda p: dw_momentum(p, mu, kappa), b, bc_t)
