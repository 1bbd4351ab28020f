"""Seeded synthetic inputs: gauge fields, sources and gauge transformations.

This module only draws inputs.  It holds none of the arithmetic of the
method (no Wilson operator, no sign function, no Krylov step), so that
the FP64 oracle and the CUDA path can both be fed from it without
sharing any of the computation they are compared on.

Conventions shared by every consumer (they define the *meaning* of the
arrays, not any computation):

* ``dims = (L1, L2, L3, L4)``; direction index ``nu = 0, 1, 2, 3`` is
  x1, x2, x3 and x4 = Euclidean time.
* canonical site index ``s = ((x1*L2 + x2)*L3 + x3)*L4 + x4`` (time
  fastest).
* gauge field ``U[s, nu, a, b]`` complex128, the SU(3) link from site
  ``x`` to ``x + nu-hat``.
* spinor field ``psi[s, spin, colour]`` complex128, flattened index
  ``12*s + 3*spin + colour``.

The paper measured on quenched gauge ensembles (Sec. 5) that are not
available here; links are drawn as ``U = exp(i*eps*H)`` with ``H`` a
traceless Hermitian matrix ``sum_a h_a lambda_a / 2`` (Gell-Mann
``lambda_a``), ``h_a ~ N(0, 1)`` i.i.d.  ``eps`` sets the roughness
(``eps = 0`` is the free field ``U = 1``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "site_coords",
    "gell_mann",
    "random_su3",
    "gauge_field",
    "free_gauge_field",
    "gaussian_source",
    "point_source",
    "point_sources",
    "gauge_transformation",
]


def volume(dims) -> int:
    d = tuple(int(x) for x in dims)
    if len(d) != 4 or min(d) < 1:
        raise ValueError(f"dims must be four positive extents, got {dims!r}")
    return d[0] * d[1] * d[2] * d[3]


def site_coords(dims) -> np.ndarray:
    """(V, 4) int array of the coordinates of every canonical site index."""
    L = tuple(int(x) for x in dims)
    g = np.indices(L).reshape(4, -1).T  # C order == time fastest
    return np.ascontiguousarray(g)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def random_su3(n: int, eps: float, rng: np.random.Generator) -> np.ndarray:
    """``n`` matrices ``exp(i*eps*H)``, ``H = sum_a h_a lambda_a/2``, h ~ N(0,1)."""
    h = rng.standard_normal((n, 8))
    H = np.einsum("na,aij->nij", h, gell_mann()) * 0.5
    w, X = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("nij,nj,nkj->nik", X, ph, X.conj())


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Seeded SU(3) gauge field ``U[V, 4, 3, 3]`` (complex128)."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    return random_su3(V * 4, float(eps), rng).reshape(V, 4, 3, 3)


def free_gauge_field(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1
    return U


def gaussian_source(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian source, real and imaginary parts i.i.d. N(0,1).

    Shape (12V,) or (nrhs, 12V) complex128.
    """
    V = volume(dims)
    rng = np.random.default_rng(seed)
    shape = (12 * V,) if nrhs is None else (int(nrhs), 12 * V)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def point_source(dims, site: int = 0, spin: int = 0, colour: int = 0) -> np.ndarray:
    V = volume(dims)
    b = np.zeros(12 * V, dtype=np.complex128)
    b[12 * site + 3 * spin + colour] = 1
    return b


def point_sources(dims, site: int = 0) -> np.ndarray:
    """All 12 spin-colour point sources at ``site``, shape (12, 12V)."""
    V = volume(dims)
    B = np.zeros((12, 12 * V), dtype=np.complex128)
    for sc in range(12):
        B[sc, 12 * site + sc] = 1
    return B


def gauge_transformation(dims, seed: int, eps: float = 3.0) -> np.ndarray:
    """Seeded site field ``g[V, 3, 3]`` of SU(3) matrices."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    return random_su3(V, float(eps), rng)


def gauge_field_torch(dims, eps: float, seed: int, device="cuda"):
    """Seeded SU(3) field of the same recipe drawn with torch on ``device``
    (for lattices too large to draw on the host).  Canonical layout
    [V, 4, 3, 3] complex128.  Not bit-identical to ``gauge_field``."""
    import torch

    V = volume(dims)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lam = torch.from_numpy(gell_mann()).to(device)
    out = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device=device)
    chunk = 1 << 20
    flat = out.view(V * 4, 3, 3)
    for s in range(0, V * 4, chunk):
        e = min(V * 4, s + chunk)
        h = torch.randn((e - s, 8), generator=g, device=device, dtype=torch.float64)
        H = torch.einsum("na,aij->nij", h.to(torch.complex128), lam) * 0.5
        flat[s:e] = torch.linalg.matrix_exp(1j * eps * H)
    return out
