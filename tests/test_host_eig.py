"""CPU test of the library's host-side dense eigensolver (used in the
deflation set-up): compiled from its source with g++ and compared with
LAPACK through numpy on random, Hessenberg, triangular-like and clustered
complex matrices."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_0810_4228_gb300", "csrc", "host_eig.cpp")

WRAP = r"""
#include <complex>
#include <vector>
namespace ovl { int host_eig(int, std::vector<std::complex<double>>&, std::vector<std::complex<double>>&,
                             std::vector<std::complex<double>>&); }
extern "C" int eig_wrap(int n, double* a, double* w, double* x) {
    std::vector<std::complex<double>> A(n * n), W, X;
    for (int i = 0; i < n * n; ++i) A[i] = {a[2 * i], a[2 * i + 1]};
    int r = ovl::host_eig(n, A, W, X);
    for (int i = 0; i < n; ++i) { w[2 * i] = W[i].real(); w[2 * i + 1] = W[i].imag(); }
    for (int i = 0; i < n * n; ++i) { x[2 * i] = X[i].real(); x[2 * i + 1] = X[i].imag(); }
    return r;
}
"""


@pytest.fixture(scope="module")
def eig():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "wrap.cpp"), "w") as f:
        f.write(WRAP)
    so = os.path.join(d, "eig.so")
    subprocess.run([gxx, "-O2", "-shared", "-fPIC", "-o", so, SRC, os.path.join(d, "wrap.cpp")], check=True)
    lib = ctypes.CDLL(so)

    def run(A):
        n = A.shape[0]
        a = np.ascontiguousarray(A, dtype=np.complex128)
        w = np.empty(n, dtype=np.complex128)
        x = np.empty((n, n), dtype=np.complex128)
        r = lib.eig_wrap(n, a.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                         x.ctypes.data_as(ctypes.c_void_p))
        assert r == 0
        return w, x
    return run


@pytest.mark.parametrize("n", [1, 2, 3, 10, 40, 120])
def test_random(eig, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w, X = eig(A)
    np.testing.assert_allclose(A @ X, X * w, atol=1e-10 * np.abs(A).max() * n)
    ref = np.linalg.eigvals(A)
    for l in ref:
        assert np.min(np.abs(w - l)) < 1e-9 * max(1, abs(l))


def test_nearly_hermitian_lattice_like(eig):
    """Spectrum close to the real axis with clusters, as the Rayleigh quotients
    of gamma5 D_w(mu) at small mu."""
    rng = np.random.default_rng(5)
    n = 60
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = (M + M.conj().T) / 2
    H += 1e-3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    w, X = eig(H)
    np.testing.assert_allclose(H @ X, X * w, atol=1e-9)
    np.testing.assert_allclose(np.sort_complex(w), np.sort_complex(np.linalg.eigvals(H)), atol=1e-9)


def test_diagonal_and_triangular(eig):
    D = np.diag([3 + 1j, -2, 0.5j, 7.0])
    w, X = eig(D)
    np.testing.assert_allclose(np.sort_complex(w), np.sort_complex(np.diag(D)), atol=1e-14)
    T = np.triu(np.arange(1, 17).reshape(4, 4).astype(complex))
    w, X = eig(T)
    np.testing.assert_allclose(T @ X, X * w, atol=1e-10)
