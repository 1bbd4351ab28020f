"""CPU test of the double-float arithmetic (csrc/df32.cuh) that the regeneration pass, the inner
quadrature and the double-float Arnoldi basis run on: its host instantiation (the same header,
compiled by nvcc for the CPU with FMA contraction off) is checked against exact rational arithmetic
(fractions.Fraction) on random and adversarial inputs.

Bounds (u = 2^-24, the FP32 unit roundoff): a double split into hi + lo is within u^2 of it; a
product of two double-float numbers within 8 u^2 of the exact product of their values; a sum
within 8 u^2 of the sum of the magnitudes; a sum of n products accumulated by dfacc within
(n + 8) u^2 of the sum of the products' magnitudes.  These are the accuracy claims the kernels'
tolerances rest on (48 significant bits, 1e-11 agreement with FP64)."""
import ctypes
import os
import random
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0810_4228_gb300", "csrc")
U2 = Fraction(1, 2 ** 48)

WRAP = r"""
#include "df32.cuh"
using ovl::df;
extern "C" {
void w_split(double a, float* o) { df x(a); o[0] = x.hi; o[1] = x.lo; }
void w_mul(float ah, float al, float bh, float bl, float* o) {
    df z = df(ah, al) * df(bh, bl); o[0] = z.hi; o[1] = z.lo;
}
void w_add(float ah, float al, float bh, float bl, float* o) {
    df z = df(ah, al) + df(bh, bl); o[0] = z.hi; o[1] = z.lo;
}
void w_add_lazy(float ah, float al, float bh, float bl, float* o) {
    df z = ovl::df_add_lazy(df(ah, al), df(bh, bl)); o[0] = z.hi; o[1] = z.lo;
}
// sum_i s_i a_i b_i with dfacc (s_i = -1 where neg[i])
void w_dot(int n, const float* a, const float* b, const int* neg, float* o) {
    ovl::dfacc A;
    for (int i = 0; i < n; ++i) {
        df x(a[2 * i], a[2 * i + 1]), y(b[2 * i], b[2 * i + 1]);
        if (i == 0) ovl::dfacc_first(A, x, y, neg[i] != 0);
        else ovl::dfacc_add(A, x, y, neg[i] != 0);
    }
    df z = ovl::dfacc_value(A); o[0] = z.hi; o[1] = z.lo;
}
// the double-float link products of the regeneration: U (9 complex, row-major) and h (6 complex,
// [spin][colour]) given as doubles, split into double-float; out = U h or U^dag h as hi, lo pairs
void w_link_df(const double* U, const double* h, int dag, float* out) {
    ovl::Link<df> L;
    ovl::Half<df> x, o;
    for (int e = 0; e < 9; ++e) L.u[e / 3][e % 3] = ovl::mk(df(U[2 * e]), df(U[2 * e + 1]));
    for (int e = 0; e < 6; ++e) x.h[e / 3][e % 3] = ovl::mk(df(h[2 * e]), df(h[2 * e + 1]));
    if (dag) ovl::mul_link_dag<df>(L, x, o);
    else ovl::mul_link<df>(L, x, o);
    for (int e = 0; e < 6; ++e) {
        const ovl::cx<df> z = o.h[e / 3][e % 3];
        out[4 * e] = z.r.hi; out[4 * e + 1] = z.r.lo; out[4 * e + 2] = z.i.hi; out[4 * e + 3] = z.i.lo;
    }
}
// 32 lanes, each with an AccF sum of n products, combined as a warp's xor-butterfly of accf_add
// (the order of the kernels' shuffle reductions); lane 0's pair out
void w_accf_warp(int n, const float* x, const float* y, const float* sg, float* o) {
    ovl::AccF a[32], b[32];
    for (int l = 0; l < 32; ++l)
        for (int i = 0; i < n; ++i) ovl::acc_prod(a[l], x[l * n + i], y[l * n + i], sg[l * n + i]);
    for (int off = 16; off > 0; off >>= 1) {
        for (int l = 0; l < 32; ++l) b[l] = ovl::accf_add(a[l], a[l ^ off]);
        for (int l = 0; l < 32; ++l) a[l] = b[l];
    }
    o[0] = a[0].hi; o[1] = a[0].lo;
}
// sum_i sg_i x_i y_i of FP32 data with the kernels' in-block accumulator AccF (hi, lo unrounded)
void w_accf(int n, const float* x, const float* y, const float* sg, float* o) {
    ovl::AccF A;
    for (int i = 0; i < n; ++i) ovl::acc_prod(A, x[i], y[i], sg[i]);
    o[0] = A.hi; o[1] = A.lo;
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
    so = os.path.join(d, "libdfhost.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", CSRC,
                    "-o", so, src], check=True, capture_output=True)
    L = ctypes.CDLL(so)
    f, pf, pi = ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)
    L.w_split.argtypes = [ctypes.c_double, pf]
    for nm in ("w_mul", "w_add", "w_add_lazy"):
        getattr(L, nm).argtypes = [f, f, f, f, pf]
    L.w_dot.argtypes = [ctypes.c_int, pf, pf, pi, pf]
    L.w_accf.argtypes = [ctypes.c_int, pf, pf, pf, pf]
    L.w_accf_warp.argtypes = [ctypes.c_int, pf, pf, pf, pf]
    pd = ctypes.POINTER(ctypes.c_double)
    L.w_link_df.argtypes = [pd, pd, ctypes.c_int, pf]
    return L


def _out():
    return (ctypes.c_float * 2)()


def _val(o):
    return Fraction(float(o[0])) + Fraction(float(o[1]))


def _rand_df(rng, scale_exp=20):
    """A normalised double-float number (hi + lo, |lo| <= ulp(hi)/2) from a random double."""
    x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-scale_exp, scale_exp)
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return float(hi), float(lo)


def test_split_of_a_double(lib):
    rng = random.Random(1)
    for _ in range(2000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        o = _out()
        lib.w_split(x, o)
        assert abs(_val(o) - Fraction(x)) <= U2 * abs(Fraction(x))
        assert abs(o[1]) <= abs(o[0]) * 2.0 ** -23  # normalised: lo below ulp(hi)
    o = _out()
    lib.w_split(0.0, o)
    assert o[0] == 0.0 and o[1] == 0.0


def test_product(lib):
    rng = random.Random(2)
    for _ in range(3000):
        a, b = _rand_df(rng), _rand_df(rng)
        o = _out()
        lib.w_mul(a[0], a[1], b[0], b[1], o)
        exact = (Fraction(a[0]) + Fraction(a[1])) * (Fraction(b[0]) + Fraction(b[1]))
        assert abs(_val(o) - exact) <= 8 * U2 * abs(exact)


@pytest.mark.parametrize("lazy", [False, True])
def test_sum_including_cancellation(lib, lazy):
    rng = random.Random(3)
    fn = lib.w_add_lazy if lazy else lib.w_add
    for it in range(3000):
        a = _rand_df(rng)
        if it % 3 == 0:  # near cancellation: b close to -a
            b0 = -a[0]
            b = (b0, float(np.float32(-a[1] * rng.uniform(0.5, 1.5))))
        else:
            b = _rand_df(rng)
        o = _out()
        fn(a[0], a[1], b[0], b[1], o)
        A, B = Fraction(a[0]) + Fraction(a[1]), Fraction(b[0]) + Fraction(b[1])
        assert abs(_val(o) - (A + B)) <= 8 * U2 * (abs(A) + abs(B))


@pytest.mark.parametrize("n", [1, 4, 24, 200])
def test_sum_of_products(lib, n):
    """dfacc: the link products (n = 6 complex terms), the sweeps' per-lane sums (n up to a few
    hundred) and the quadrature's solves all reduce to sums of products like this one."""
    rng = random.Random(10 + n)
    for _ in range(200):
        xs = [_rand_df(rng, 6) for _ in range(n)]
        ys = [_rand_df(rng, 6) for _ in range(n)]
        neg = [rng.random() < 0.5 for _ in range(n)]
        a = (ctypes.c_float * (2 * n))(*[v for p in xs for v in p])
        b = (ctypes.c_float * (2 * n))(*[v for p in ys for v in p])
        s = (ctypes.c_int * n)(*[int(v) for v in neg])
        o = _out()
        lib.w_dot(n, a, b, s, o)
        terms = [(Fraction(x[0]) + Fraction(x[1])) * (Fraction(y[0]) + Fraction(y[1])) * (-1 if g else 1)
                 for x, y, g in zip(xs, ys, neg)]
        exact = sum(terms, Fraction(0))
        mag = sum((abs(t) for t in terms), Fraction(0))
        assert abs(_val(o) - exact) <= (n + 8) * U2 * mag


def _accf(lib, x, y, sg):
    n = len(x)
    o = _out()
    lib.w_accf(n, (ctypes.c_float * n)(*x), (ctypes.c_float * n)(*y), (ctypes.c_float * n)(*sg), o)
    return o


@pytest.mark.parametrize("n", [1, 12, 24, 200, 2000])
def test_compensated_fp32_sum_of_products(lib, n):
    """AccF, the per-thread accumulator of the FP32 kernels' reductions (alpha = w^dag t, the norms
    and w^^dag v^ of Eq. 4.2): every FP32 product enters exactly (FMA TwoProduct), the leading parts
    are added with TwoSum and the errors in FP32, so hi + lo is within gamma_2n^2 of the sum of
    the products' magnitudes (gamma_m = m u / (1 - m u)) of the exact sum, the bound of the
    compensated dot product (Ogita, Rump and Oishi, 2005) without its final rounding."""
    rng = random.Random(100 + n)
    u = Fraction(1, 2 ** 24)
    g2n = (2 * n * u) / (1 - 2 * n * u)
    for _ in range(100 if n < 2000 else 10):
        x = [float(np.float32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-8, 8))) for _ in range(n)]
        y = [float(np.float32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-8, 8))) for _ in range(n)]
        sg = [rng.choice((1.0, -1.0)) for _ in range(n)]
        o = _accf(lib, x, y, sg)
        terms = [Fraction(a) * Fraction(b) * int(g) for a, b, g in zip(x, y, sg)]
        exact = sum(terms, Fraction(0))
        mag = sum((abs(t) for t in terms), Fraction(0))
        assert abs(_val(o) - exact) <= g2n * g2n * mag


def test_compensated_fp32_sum_under_cancellation(lib):
    """Products that cancel to a sum 1e6 times smaller than their magnitudes: plain FP32
    accumulation loses every digit, AccF keeps the exact sum to the gamma_2n^2 bound."""
    rng = random.Random(7)
    n = 64
    u = Fraction(1, 2 ** 24)
    g2n = (2 * n * u) / (1 - 2 * n * u)
    for _ in range(50):
        half = [(float(np.float32(rng.uniform(0.5, 1) * 2.0 ** rng.randint(-4, 4))),
                 float(np.float32(rng.uniform(0.5, 1)))) for _ in range(n // 2)]
        x = [a for a, _ in half] + [a for a, _ in half]
        y = [b for _, b in half] + [float(np.float32(b * (1 + rng.uniform(-1e-6, 1e-6)))) for _, b in half]
        sg = [1.0] * (n // 2) + [-1.0] * (n // 2)
        order = list(range(n))
        rng.shuffle(order)
        x, y, sg = [x[i] for i in order], [y[i] for i in order], [sg[i] for i in order]
        o = _accf(lib, x, y, sg)
        terms = [Fraction(a) * Fraction(b) * int(g) for a, b, g in zip(x, y, sg)]
        exact = sum(terms, Fraction(0))
        mag = sum((abs(t) for t in terms), Fraction(0))
        err = abs(_val(o) - exact)
        assert err <= g2n * g2n * mag
        plain = np.float32(0)
        for a, b, g in zip(x, y, sg):
            plain = np.float32(plain + np.float32(np.float32(a) * np.float32(b)) * np.float32(g))
        assert err * 1000 < abs(Fraction(float(plain)) - exact) or abs(Fraction(float(plain)) - exact) == 0


@pytest.mark.parametrize("n", [1, 12, 48])
def test_compensated_fp32_warp_reduction(lib, n):
    """32 per-lane AccF sums combined by the warp butterfly of accf_add (TwoSum of the leading parts,
    the trailing parts and the error in FP32), as in the batched kernels' block and sequence sums:
    within gamma_m^2 of the magnitudes, m = 2 n + 2 log2(32) + 2 roundings along any path."""
    rng = random.Random(300 + n)
    u = Fraction(1, 2 ** 24)
    m = 2 * n + 12
    gm = (m * u) / (1 - m * u)
    N = 32 * n
    for _ in range(40):
        x = [float(np.float32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-8, 8))) for _ in range(N)]
        y = [float(np.float32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-8, 8))) for _ in range(N)]
        sg = [rng.choice((1.0, -1.0)) for _ in range(N)]
        o = _out()
        lib.w_accf_warp(n, (ctypes.c_float * N)(*x), (ctypes.c_float * N)(*y), (ctypes.c_float * N)(*sg), o)
        terms = [Fraction(a) * Fraction(b) * int(g) for a, b, g in zip(x, y, sg)]
        exact = sum(terms, Fraction(0))
        mag = sum((abs(t) for t in terms), Fraction(0))
        assert abs(_val(o) - exact) <= gm * gm * mag


@pytest.mark.parametrize("dag", [0, 1])
def test_double_float_link_products(lib, dag):
    """U h and U^dag h in double-float (the link multiply of the double-float regeneration, Eq. 1.2),
    with U a random SU(3) matrix and h a random half spinor split from doubles: every output
    component, a sum of six products, is within (6 + 8) u^2 of its terms' magnitudes of the exact
    sum of the split inputs' products, and within 1e-13 of the FP64 product (the splits keep 48 of
    the inputs' 53 bits)."""
    import sys
    sys.path.insert(0, ROOT)
    from paper_0810_4228_gb300 import synth
    rng = np.random.default_rng(50 + dag)
    Us = synth.random_su3(30, 1.0, rng)
    pd = ctypes.POINTER(ctypes.c_double)

    def split(x):
        hi = float(np.float32(x))
        return Fraction(hi) + Fraction(float(np.float32(x - hi)))

    for u in Us:
        h = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
        ub = np.ascontiguousarray(u.reshape(9)).view(np.float64)
        hb = np.ascontiguousarray(h.reshape(6)).view(np.float64)
        out = (ctypes.c_float * 24)()
        lib.w_link_df(ub.ctypes.data_as(pd), hb.ctypes.data_as(pd), dag, out)
        got = np.array([float(Fraction(out[4 * e]) + Fraction(out[4 * e + 1])) +
                        1j * float(Fraction(out[4 * e + 2]) + Fraction(out[4 * e + 3])) for e in range(6)]).reshape(2, 3)
        M = u.conj().T if dag else u
        ref = (M @ h.T).T
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        # exact sums of the split inputs, component by component
        Us_ = [[(split(M[a, k].real), split(M[a, k].imag)) for k in range(3)] for a in range(3)]
        hs_ = [[(split(h[sp, k].real), split(h[sp, k].imag)) for k in range(3)] for sp in range(2)]
        for sp in range(2):
            for a in range(3):
                tr = [Us_[a][k][0] * hs_[sp][k][0] for k in range(3)] + [-Us_[a][k][1] * hs_[sp][k][1] for k in range(3)]
                ti = [Us_[a][k][0] * hs_[sp][k][1] for k in range(3)] + [Us_[a][k][1] * hs_[sp][k][0] for k in range(3)]
                e = 3 * sp + a
                for terms, q in ((tr, 0), (ti, 2)):
                    val = Fraction(out[4 * e + q]) + Fraction(out[4 * e + q + 1])
                    mag = sum((abs(t) for t in terms), Fraction(0))
                    assert abs(val - sum(terms, Fraction(0))) <= 14 * U2 * mag
