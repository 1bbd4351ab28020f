"""CPU test of the stencil's building blocks in csrc/ovl_common.cuh, the host-and-device helpers
that every Wilson kernel composes (Sec. 1, Eq. 1.2): the header is compiled for the host and each
helper is compared with an independent definition.

* spin projection and reconstruction: recon(project(psi)) = (1 + S gamma_nu) psi with the
  oracle's chiral gamma matrices;
* the SU(3) products U h and U^dag h against numpy, and the third-row reconstruction of the
  12-real link format against the full matrix of a random SU(3) element;
* complex division (Smith's algorithm) against exact rational arithmetic, at magnitudes where
  the textbook formula over- or underflows;
* the even/odd device layout: site_coord / internal_index are inverse bijections onto the
  lattice, the parity half matches (x1 + x2 + x3 + x4) mod 2, and neighbour() lands on the
  oracle's forward and backward neighbours, on lattices with odd spatial extents too."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import wilson as W
from paper_0810_4228_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0810_4228_gb300", "csrc")

WRAP = r"""
#include "ovl_common.cuh"
using namespace ovl;

template <int NU, int S>
static void pr(const Spinor<double>& p, Spinor<double>& acc) {
    Half<double> h;
    project<NU, S>(p, h);
    recon_acc<NU, S>(acc, h, 1.0);
}

extern "C" {
// out = recon(project(p)) for direction nu and sign S; p, out: 12 complex, index 3 * spin + colour
void w_proj_recon(const double* p, int nu, int S, double* out) {
    Spinor<double> sp, acc;
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            sp.s[s][a] = mk(p[2 * (3 * s + a)], p[2 * (3 * s + a) + 1]);
            acc.s[s][a] = mk(0.0, 0.0);
        }
    const int k = 2 * nu + (S > 0 ? 0 : 1);
    switch (k) {
        case 0: pr<0, 1>(sp, acc); break;
        case 1: pr<0, -1>(sp, acc); break;
        case 2: pr<1, 1>(sp, acc); break;
        case 3: pr<1, -1>(sp, acc); break;
        case 4: pr<2, 1>(sp, acc); break;
        case 5: pr<2, -1>(sp, acc); break;
        case 6: pr<3, 1>(sp, acc); break;
        default: pr<3, -1>(sp, acc); break;
    }
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            out[2 * (3 * s + a)] = acc.s[s][a].r;
            out[2 * (3 * s + a) + 1] = acc.s[s][a].i;
        }
}
// U: 9 complex row-major; h: 6 complex [spin][colour]; out = U h (dag = 0) or U^dag h (dag = 1)
void w_mul_link(const double* U, const double* h, int dag, double* out) {
    Link<double> L;
    Half<double> x, o;
    for (int e = 0; e < 9; ++e) L.u[e / 3][e % 3] = mk(U[2 * e], U[2 * e + 1]);
    for (int e = 0; e < 6; ++e) x.h[e / 3][e % 3] = mk(h[2 * e], h[2 * e + 1]);
    if (dag) mul_link_dag(L, x, o);
    else mul_link(L, x, o);
    for (int e = 0; e < 6; ++e) {
        out[2 * e] = o.h[e / 3][e % 3].r;
        out[2 * e + 1] = o.h[e / 3][e % 3].i;
    }
}
// rows 0 and 1 of U (6 complex) -> the reconstructed row 2 (3 complex)
void w_row2(const double* U, double* out) {
    Link<double> L;
    for (int e = 0; e < 6; ++e) L.u[e / 3][e % 3] = mk(U[2 * e], U[2 * e + 1]);
    reconstruct_row2(L);
    for (int a = 0; a < 3; ++a) {
        out[2 * a] = L.u[2][a].r;
        out[2 * a + 1] = L.u[2][a].i;
    }
}
// a / b by the library's complex division (the recurrence's 1 / beta, 1 / conj(gamma))
void w_cdiv(double ar, double ai, double br, double bi, double* out) {
    const cx<double> z = cdiv(mk(ar, ai), mk(br, bi));
    out[0] = z.r;
    out[1] = z.i;
}
// for every internal index i: coords[i] = (x1, x2, x3, x4, parity), back[i] = internal_index(x),
// nbr[i][2 nu + d] = neighbour(x, nu, d ? -1 : +1)
void w_geom(const int* dims, int* coords, int* back, int* nbr) {
    Geom g;
    for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
    g.L4h = dims[3] / 2;
    g.V = dims[0] * dims[1] * dims[2] * dims[3];
    g.Vh = g.V / 2;
    g.bc_t = -1;
    for (int i = 0; i < g.V; ++i) {
        const Coord c = site_coord(g, i);
        for (int k = 0; k < 4; ++k) coords[5 * i + k] = c.x[k];
        coords[5 * i + 4] = c.par;
        back[i] = internal_index(g, c.x);
        for (int nu = 0; nu < 4; ++nu) {
            nbr[8 * i + 2 * nu] = neighbour(g, c, nu, +1);
            nbr[8 * i + 2 * nu + 1] = neighbour(g, c, nu, -1);
        }
    }
}
}
"""


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "wrap.cu")
    with open(src, "w") as f:
        f.write(WRAP)
    so = os.path.join(d, "libstencilhost.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", CSRC,
                    "-o", so, src], check=True, capture_output=True)
    L = ctypes.CDLL(so)
    pd, pi = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.w_proj_recon.argtypes = [pd, ctypes.c_int, ctypes.c_int, pd]
    L.w_mul_link.argtypes = [pd, pd, ctypes.c_int, pd]
    L.w_row2.argtypes = [pd, pd]
    L.w_geom.argtypes = [pi, pi, pi, pi]
    L.w_cdiv.argtypes = [ctypes.c_double] * 4 + [pd]
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("nu", range(4))
@pytest.mark.parametrize("S", [1, -1])
def test_projection_and_reconstruction(lib, nu, S):
    """The hop's spin algebra: only additions and multiplications by +-1, +-i, so the result is
    exact against (1 + S gamma_nu) psi with the oracle's gamma matrices (colour by colour)."""
    rng = np.random.default_rng(10 * nu + (S > 0))
    P = np.eye(4) + S * W.gamma_matrices()[nu]
    for _ in range(20):
        psi = _crand(rng, 4, 3)
        out = np.empty(12, dtype=np.complex128)
        lib.w_proj_recon(_dp(np.ascontiguousarray(psi.reshape(12))), nu, S, _dp(out))
        ref = P @ psi
        assert np.abs(out.reshape(4, 3) - ref).max() <= 1e-15 * np.abs(ref).max()


def test_projector_rank_two(lib):
    """(1 + S gamma_nu) / 2 is a projector of rank 2: the reconstruction from the two projected spins
    is the full image, and applying the pair twice doubles the result."""
    rng = np.random.default_rng(5)
    for nu in range(4):
        for S in (1, -1):
            psi = _crand(rng, 4, 3)
            once = np.empty(12, dtype=np.complex128)
            twice = np.empty(12, dtype=np.complex128)
            lib.w_proj_recon(_dp(np.ascontiguousarray(psi.reshape(12))), nu, S, _dp(once))
            lib.w_proj_recon(_dp(once), nu, S, _dp(twice))
            assert np.allclose(twice, 2 * once, rtol=0, atol=1e-13)
            assert np.linalg.matrix_rank(np.eye(4) + S * W.gamma_matrices()[nu]) == 2


@pytest.mark.parametrize("dag", [0, 1])
def test_link_products(lib, dag):
    rng = np.random.default_rng(20 + dag)
    U = synth.random_su3(8, 1.0, rng)
    for u in U:
        h = _crand(rng, 2, 3)
        out = np.empty(6, dtype=np.complex128)
        lib.w_mul_link(_dp(np.ascontiguousarray(u.reshape(9))), _dp(np.ascontiguousarray(h.reshape(6))), dag, _dp(out))
        M = u.conj().T if dag else u
        ref = (M @ h.T).T
        assert np.abs(out.reshape(2, 3) - ref).max() <= 1e-14 * np.abs(ref).max()


def test_third_row_of_su3(lib):
    """The 12-real link format keeps rows 0 and 1; row 2 = conj(row0 x row1) for det U = 1."""
    rng = np.random.default_rng(30)
    U = synth.random_su3(50, 1.0, rng)
    for u in U:
        assert abs(np.linalg.det(u) - 1) < 1e-12
        out = np.empty(3, dtype=np.complex128)
        lib.w_row2(_dp(np.ascontiguousarray(u[:2].reshape(6))), _dp(out))
        assert np.abs(out - u[2]).max() < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (3, 2, 5, 4), (4, 3, 2, 6), (4, 4, 4, 8)])
def test_even_odd_layout_and_neighbours(lib, dims):
    V = int(np.prod(dims))
    coords = np.empty((V, 5), dtype=np.int32)
    back = np.empty(V, dtype=np.int32)
    nbr = np.empty((V, 8), dtype=np.int32)
    lib.w_geom(_ip(np.array(dims, dtype=np.int32)), _ip(coords), _ip(back), _ip(nbr))
    x = coords[:, :4].astype(np.int64)
    assert np.array_equal(back, np.arange(V))  # internal_index inverts site_coord
    assert (x >= 0).all() and (x < np.array(dims)).all()
    canon = ((x[:, 0] * dims[1] + x[:, 1]) * dims[2] + x[:, 2]) * dims[3] + x[:, 3]
    assert np.array_equal(np.sort(canon), np.arange(V))  # a bijection onto the lattice
    par = x.sum(axis=1) & 1
    assert np.array_equal(coords[:, 4], par)
    assert np.array_equal(par, (np.arange(V) >= V // 2).astype(par.dtype))
    # internal index = parity * V/2 + canonical index / 2 (the documented device layout)
    assert np.array_equal(np.arange(V), par * (V // 2) + canon // 2)
    # neighbours against the oracle's (canonical indices mapped to internal ones)
    fwd, bwd, _, _ = W.neighbours(dims)
    internal_of_canon = np.empty(V, dtype=np.int64)
    internal_of_canon[canon] = np.arange(V)
    for nu in range(4):
        assert np.array_equal(nbr[:, 2 * nu], internal_of_canon[fwd[canon, nu]])
        assert np.array_equal(nbr[:, 2 * nu + 1], internal_of_canon[bwd[canon, nu]])


def test_complex_division(lib):
    """a / b within a few ulps of the exact quotient (fractions), including |b|^2 outside the double
    range, where dividing by |b|^2 directly would overflow or underflow."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(40)
    cases = [(complex(*rng.standard_normal(2)) * 10.0 ** rng.integers(-8, 8),
              complex(*rng.standard_normal(2)) * 10.0 ** rng.integers(-8, 8)) for _ in range(500)]
    cases += [(1e300 + 1e300j, 1e300 + 2e300j), (1e-300 + 3e-300j, 2e-300 - 1e-300j), (1 + 1j, 1e-170 + 1e-170j),
              (3.0 + 0j, 0 + 2j), (0j, 1 - 1j)]
    for a, b in cases:
        out = np.empty(2)
        lib.w_cdiv(a.real, a.imag, b.real, b.imag, _dp(out))
        assert np.isfinite(out).all(), (a, b)
        ar, ai, br, bi = (Fr(v) for v in (a.real, a.imag, b.real, b.imag))
        d = br * br + bi * bi
        qr, qi = (ar * br + ai * bi) / d, (ai * br - ar * bi) / d
        mag = max(abs(qr), abs(qi))
        tol = 8 * Fr(2) ** -53 * mag
        assert abs(Fr(out[0]) - qr) <= tol and abs(Fr(out[1]) - qi) <= tol, (a, b, out)
