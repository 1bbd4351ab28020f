"""Wilson-Dirac operator at chemical potential mu and A = gamma5 D_w(mu).

Follows Sec. 1 of the paper: Eq. 1.1 (D_ov = 1 + gamma5 sgn(gamma5 D_w)),
Eq. 1.2 (D_w(mu) = 1 - kappa sum_i (T_i^+ + T_i^-)
                     - kappa (e^mu T_4^+ + e^-mu T_4^-)),
and the hopping terms T_nu^+-, kappa = 1/(8 + 2 m_w), U in SU(3).

Readings taken where the paper is silent or ambiguous:

* T_nu^+ is the hop to the forward neighbour with projector (1 + gamma_nu):
  (T_nu^+ psi)(x) = (1 + gamma_nu) U_{x,nu} psi(x + nu);
  (T_nu^- psi)(x) = (1 - gamma_nu) U_{x-nu,nu}^dagger psi(x - nu);
  e^{+mu} multiplies T_4^+.
* Euclidean gamma matrices in the chiral basis,
  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]],
  so gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1).
* periodic boundary conditions in space, antiperiodic (bc_t = -1, default)
  or periodic (bc_t = +1) in time.

Index conventions are those of ``paper_0810_4228_gb300.synth``: canonical
site index with time fastest, vector index 12*site + 3*spin + colour.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = [
    "gamma_matrices",
    "gamma5_spin",
    "kappa_from_mw",
    "neighbours",
    "hop_term",
    "wilson_dirac",
    "gamma5_operator",
    "a_operator",
    "dense_a",
    "wilson_site",
]


def gamma_matrices():
    """Euclidean (gamma_1..gamma_4) in the chiral basis, shape (4, 4, 4)."""
    s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    Z = np.zeros((2, 2), dtype=np.complex128)
    I2 = np.eye(2, dtype=np.complex128)
    g = [np.block([[Z, -1j * s], [1j * s, Z]]) for s in (s1, s2, s3)]
    g.append(np.block([[Z, I2], [I2, Z]]))
    return np.array(g)


def gamma5_spin():
    """gamma5 = gamma1 gamma2 gamma3 gamma4 (Sec. 1, below Eq. 1.1)."""
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]


def kappa_from_mw(m_w: float) -> float:
    """kappa = 1/(8 + 2 m_w), Sec. 1."""
    return 1.0 / (8.0 + 2.0 * m_w)


def _coords(dims):
    L = tuple(int(x) for x in dims)
    return np.indices(L).reshape(4, -1).T


def _index(c, dims):
    L = dims
    return ((c[:, 0] * L[1] + c[:, 1]) * L[2] + c[:, 2]) * L[3] + c[:, 3]


def neighbours(dims, bc_t: int = -1):
    """Forward/backward neighbour indices and boundary phases.

    Returns ``fwd[V,4], bwd[V,4], ph_f[V,4], ph_b[V,4]``: the site x+nu,
    the site x-nu and the factor (bc_t or 1) a hop across the time edge picks up.
    """
    dims = tuple(int(x) for x in dims)
    c = _coords(dims)
    V = c.shape[0]
    fwd = np.empty((V, 4), dtype=np.int64)
    bwd = np.empty((V, 4), dtype=np.int64)
    ph_f = np.ones((V, 4))
    ph_b = np.ones((V, 4))
    for nu in range(4):
        cf = c.copy()
        cf[:, nu] = (cf[:, nu] + 1) % dims[nu]
        cb = c.copy()
        cb[:, nu] = (cb[:, nu] - 1) % dims[nu]
        fwd[:, nu] = _index(cf, dims)
        bwd[:, nu] = _index(cb, dims)
        if nu == 3:
            ph_f[c[:, 3] == dims[3] - 1, nu] = bc_t
            ph_b[c[:, 3] == 0, nu] = bc_t
    return fwd, bwd, ph_f, ph_b


def hop_term(U, dims, nu: int, sign: int, bc_t: int = -1) -> sp.csr_matrix:
    """T_nu^+ (sign=+1) or T_nu^- (sign=-1) of Eq. 1.2 as a sparse matrix,
    including the boundary phase of hops across the time edge:
    (T_nu^+ psi)(x) = (1 + gamma_nu) U_{x,nu} psi(x + nu),
    (T_nu^- psi)(x) = (1 - gamma_nu) U_{x-nu,nu}^dag psi(x - nu)."""
    dims = tuple(int(x) for x in dims)
    V = int(np.prod(dims))
    U = np.asarray(U, dtype=np.complex128).reshape(V, 4, 3, 3)
    g = gamma_matrices()
    I4 = np.eye(4, dtype=np.complex128)
    fwd, bwd, ph_f, ph_b = neighbours(dims, bc_t)
    loc = np.arange(12)
    r = (12 * np.arange(V))[:, None, None] + loc[None, :, None]
    if sign > 0:
        link, nb, ph, proj = U[:, nu], fwd[:, nu], ph_f[:, nu], I4 + g[nu]
    else:
        link = U[bwd[:, nu], nu].conj().transpose(0, 2, 1)
        nb, ph, proj = bwd[:, nu], ph_b[:, nu], I4 - g[nu]
    blk = np.einsum("st,vab->vsatb", proj, link).reshape(V, 12, 12) * ph[:, None, None]
    c = (12 * nb)[:, None, None] + loc[None, None, :]
    M = sp.coo_matrix(
        (blk.ravel(), (np.broadcast_to(r, (V, 12, 12)).ravel(),
                       np.broadcast_to(c, (V, 12, 12)).ravel())),
        shape=(12 * V, 12 * V),
    ).tocsr()  # duplicates (extent-2 directions) are summed
    return M


def wilson_dirac(U, dims, mu: float, kappa: float, bc_t: int = -1) -> sp.csr_matrix:
    """Sparse D_w(mu) of Eq. 1.2, (12V x 12V) complex128 CSR."""
    V = int(np.prod(dims))
    M = sp.identity(12 * V, dtype=np.complex128, format="csr")
    for nu in range(4):
        cp = np.exp(mu) if nu == 3 else 1.0
        cm = np.exp(-mu) if nu == 3 else 1.0
        M = M - kappa * (cp * hop_term(U, dims, nu, +1, bc_t) + cm * hop_term(U, dims, nu, -1, bc_t))
    M = M.tocsr()
    M.eliminate_zeros()
    return M


def gamma5_operator(V: int) -> sp.csr_matrix:
    """gamma5 acting on the whole lattice: diag over sites of gamma5 (x) 1_colour."""
    d = np.kron(np.ones(V), np.kron(np.real(np.diag(gamma5_spin())), np.ones(3)))
    return sp.diags(d.astype(np.complex128)).tocsr()


def a_operator(U, dims, mu: float, kappa: float, bc_t: int = -1) -> sp.csr_matrix:
    """A = gamma5 D_w(mu), the argument of the sign function in Eq. 1.1."""
    V = int(np.prod(dims))
    return (gamma5_operator(V) @ wilson_dirac(U, dims, mu, kappa, bc_t)).tocsr()


def dense_a(U, dims, mu: float, kappa: float, bc_t: int = -1) -> np.ndarray:
    return a_operator(U, dims, mu, kappa, bc_t).toarray()


def wilson_site(U, dims, mu: float, kappa: float, x, site: int, bc_t: int = -1,
                gamma5: bool = True) -> np.ndarray:
    """(gamma5) D_w(mu) x evaluated at one site, by a direct loop over its
    eight hops (Eq. 1.2).  Used to check single outputs of very large
    lattices, where the sparse matrix is not built.  Returns 12 complex.
    """
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(V, 4, 3, 3)
    x = np.asarray(x).reshape(V, 4, 3)
    g = gamma_matrices()
    I4 = np.eye(4)
    c = np.array(np.unravel_index(site, dims))
    out = x[site].astype(np.complex128).copy()
    for nu in range(4):
        cf = c.copy()
        cf[nu] = (cf[nu] + 1) % dims[nu]
        cb = c.copy()
        cb[nu] = (cb[nu] - 1) % dims[nu]
        f = int(np.ravel_multi_index(cf, dims))
        b = int(np.ravel_multi_index(cb, dims))
        phf = bc_t if (nu == 3 and c[3] == dims[3] - 1) else 1
        phb = bc_t if (nu == 3 and c[3] == 0) else 1
        cp = np.exp(mu) if nu == 3 else 1.0
        cm = np.exp(-mu) if nu == 3 else 1.0
        hop_f = (I4 + g[nu]) @ x[f] @ U[site, nu].T        # (1+g) U psi(x+nu)
        hop_b = (I4 - g[nu]) @ x[b] @ U[b, nu].conj()      # (1-g) U^dag psi(x-nu)
        out -= kappa * (cp * phf * hop_f + cm * phb * hop_b)
    if gamma5:
        out = np.real(np.diag(gamma5_spin()))[:, None] * out
    return out.reshape(12)
