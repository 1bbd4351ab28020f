// Double-float arithmetic: a real number as the unevaluated sum hi + lo of two
// FP32 values with |lo| <= ulp(hi) / 2, about 48 significant bits, evaluated on
// the FP32 pipe.  Products enter exactly through a fused multiply-add
// (e = fma(a, b, -a b) is the rounding error of a b) and sums through Knuth's
// TwoSum; every result is renormalised (Dekker's Fast2Sum).  The _rn
// intrinsics keep the compiler from contracting the error-free
// transformations.  Relative rounding of a product or a sum of like-signed
// terms is about 2^-44, and the absolute error of a sum about 2^-44 times the
// sum of the magnitudes of its terms.
//
// Storage: one complex number as float4 {re.hi, re.lo, im.hi, im.lo} (16 bytes,
// as a complex128), in the FP64 layouts of vectors ([component][site]) and
// links ([nu][element][site]).
#pragma once

#include "ovl_common.cuh"

namespace ovl {

struct df {
    float hi, lo;
    OVL_HD df() {}
    OVL_HD df(float h, float l) : hi(h), lo(l) {}
    OVL_HD df(int x) : hi((float)x), lo(0.f) {}
    // split of a double (host set-up and per-launch coefficients)
    OVL_HD df(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    OVL_HD double to_double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn(a, b)
#define DF_SUB(a, b) __fsub_rn(a, b)
#define DF_MUL(a, b) __fmul_rn(a, b)
#define DF_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) fmaf(a, b, c)
#endif

OVL_HD df df_fast2sum(float s, float e) {
    const float h = DF_ADD(s, e);
    return df(h, DF_SUB(e, DF_SUB(h, s)));
}

OVL_HD df operator+(df a, df b) {
    const float s = DF_ADD(a.hi, b.hi);
    const float bb = DF_SUB(s, a.hi);
    float e = DF_ADD(DF_SUB(a.hi, DF_SUB(s, bb)), DF_SUB(b.hi, bb));
    e = DF_ADD(e, DF_ADD(a.lo, b.lo));
    return df_fast2sum(s, e);
}
// Sum without the final renormalisation: hi + lo holds the sum to the rounding of the lo part,
// but lo may exceed ulp(hi) / 2 by a few ulps.  Every consumer (products, which take the cross
// terms with lo in FP32; further sums; the renormalising multiply or store) handles such pairs at
// the same accuracy; used for intermediate sums whose result feeds another operation.
OVL_HD df df_add_lazy(df a, df b) {
    const float s = DF_ADD(a.hi, b.hi);
    const float bb = DF_SUB(s, a.hi);
    float e = DF_ADD(DF_SUB(a.hi, DF_SUB(s, bb)), DF_SUB(b.hi, bb));
    e = DF_ADD(e, DF_ADD(a.lo, b.lo));
    return df(s, e);
}
OVL_HD df operator-(df a) { return df(-a.hi, -a.lo); }
OVL_HD df operator-(df a, df b) { return a + (-b); }
OVL_HD df operator*(df a, df b) {
    const float p = DF_MUL(a.hi, b.hi);
    float e = DF_FMA(a.hi, b.hi, -p);
    e = DF_FMA(a.hi, b.lo, e);
    e = DF_FMA(a.lo, b.hi, e);
    return df_fast2sum(p, e);
}
OVL_HD df& operator+=(df& a, df b) { a = a + b; return a; }
OVL_HD df& operator-=(df& a, df b) { a = a - b; return a; }

// Sum of products of double-float numbers with one renormalisation at the end: every product
// enters as its exact FP32 leading product and an FP32 error term (the cross terms of hi and lo
// included), the leading products are added with TwoSum, the error terms in plain FP32.
struct dfacc {
    float s, e;
};
OVL_HD void dfacc_first(dfacc& A, df a, df b, bool neg) {
    float p = DF_MUL(a.hi, b.hi);
    float pe = DF_FMA(a.hi, b.hi, -p);
    pe = DF_FMA(a.hi, b.lo, pe);
    pe = DF_FMA(a.lo, b.hi, pe);
    A.s = neg ? -p : p;
    A.e = neg ? -pe : pe;
}
OVL_HD void dfacc_add(dfacc& A, df a, df b, bool neg) {
    float p = DF_MUL(a.hi, b.hi);
    float pe = DF_FMA(a.hi, b.hi, -p);
    pe = DF_FMA(a.hi, b.lo, pe);
    pe = DF_FMA(a.lo, b.hi, pe);
    if (neg) {
        p = -p;
        pe = -pe;
    }
    const float s = DF_ADD(A.s, p);
    const float bb = DF_SUB(s, A.s);
    const float t = DF_ADD(DF_SUB(A.s, DF_SUB(s, bb)), DF_SUB(p, bb));
    A.s = s;
    A.e = DF_ADD(A.e, DF_ADD(t, pe));
}
OVL_HD df dfacc_value(const dfacc& A) { return df_fast2sum(A.s, A.e); }

// out = U h for both half-spinor spins (Sec. 1, Eq. 1.2 hop), each output component one sum of
// six double-float products
template <>
OVL_HD void mul_link<df>(const Link<df>& U, const Half<df>& h, Half<df>& o) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dfacc re, im;
            dfacc_first(re, U.u[a][0].r, h.h[s][0].r, false);
            dfacc_add(re, U.u[a][0].i, h.h[s][0].i, true);
            dfacc_first(im, U.u[a][0].r, h.h[s][0].i, false);
            dfacc_add(im, U.u[a][0].i, h.h[s][0].r, false);
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                dfacc_add(re, U.u[a][k].r, h.h[s][k].r, false);
                dfacc_add(re, U.u[a][k].i, h.h[s][k].i, true);
                dfacc_add(im, U.u[a][k].r, h.h[s][k].i, false);
                dfacc_add(im, U.u[a][k].i, h.h[s][k].r, false);
            }
            o.h[s][a] = mk(dfacc_value(re), dfacc_value(im));
        }
}
// out = U^dag h
template <>
OVL_HD void mul_link_dag<df>(const Link<df>& U, const Half<df>& h, Half<df>& o) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dfacc re, im;
            dfacc_first(re, U.u[0][a].r, h.h[s][0].r, false);
            dfacc_add(re, U.u[0][a].i, h.h[s][0].i, false);
            dfacc_first(im, U.u[0][a].r, h.h[s][0].i, false);
            dfacc_add(im, U.u[0][a].i, h.h[s][0].r, true);
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                dfacc_add(re, U.u[k][a].r, h.h[s][k].r, false);
                dfacc_add(re, U.u[k][a].i, h.h[s][k].i, false);
                dfacc_add(im, U.u[k][a].r, h.h[s][k].i, false);
                dfacc_add(im, U.u[k][a].i, h.h[s][k].r, true);
            }
            o.h[s][a] = mk(dfacc_value(re), dfacc_value(im));
        }
}

OVL_HD cx<df> add_lazy(const cx<df>& a, const cx<df>& b) { return mk(df_add_lazy(a.r, b.r), df_add_lazy(a.i, b.i)); }

struct __align__(16) dfc {
    float rh, rl, ih, il;
};

OVL_HD cx<df> dfc2c(dfc v) { return mk(df(v.rh, v.rl), df(v.ih, v.il)); }
OVL_HD dfc c2dfc(cx<df> z) {
    dfc v;
    v.rh = z.r.hi;
    v.rl = z.r.lo;
    v.ih = z.i.hi;
    v.il = z.i.lo;
    return v;
}
OVL_HD cx<df> d2df(double2 a) { return mk(df(a.x), df(a.y)); }
OVL_HD double2 df2d(cx<df> z) { return make_double2(z.r.to_double(), z.i.to_double()); }

__device__ __forceinline__ void load_spinor(const dfc* __restrict__ x, int V, int i, Spinor<df>& p) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(x) + (size_t)c * V + i);
        p.s[c / 3][c % 3] = mk(df(v.x, v.y), df(v.z, v.w));
    }
}
__device__ __forceinline__ void load_spinor_cg(const dfc* x, int V, int i, Spinor<df>& p) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(x) + (size_t)c * V + i);
        p.s[c / 3][c % 3] = mk(df(v.x, v.y), df(v.z, v.w));
    }
}
__device__ __forceinline__ void store_spinor(dfc* __restrict__ x, int V, int i, const Spinor<df>& p) {
#pragma unroll
    for (int c = 0; c < 12; ++c) x[(size_t)c * V + i] = c2dfc(p.s[c / 3][c % 3]);
}
__device__ __forceinline__ void load_link_df(const dfc* __restrict__ U, int V, int nu, int i, Link<df>& L) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(U) + ((size_t)nu * 9 + e) * V + i);
        L.u[e / 3][e % 3] = mk(df(v.x, v.y), df(v.z, v.w));
    }
}

// in-block accumulators: compensated FP32 pairs for FP32 data, plain FP64 for FP64 data.
// AccF adds each exact product p + pe (TwoProduct by FMA) with TwoSum into hi and collects the
// rounding errors and the pe terms in lo (the compensated dot product of Ogita, Rump and Oishi,
// 2005, kept as an unevaluated pair); host-callable so that its accuracy can be checked on the CPU.
struct AccF {
    float hi = 0.f, lo = 0.f;
};
OVL_HD void acc_add(AccF& a, float p, float pe) {
    const float s = DF_ADD(a.hi, p);
    const float bb = DF_SUB(s, a.hi);
    const float e = DF_ADD(DF_SUB(a.hi, DF_SUB(s, bb)), DF_SUB(p, bb));
    a.hi = s;
    a.lo = DF_ADD(a.lo, DF_ADD(e, pe));
}
OVL_HD void acc_prod(AccF& a, float x, float y, float sg = 1.f) {
    const float p = DF_MUL(x, y);
    const float pe = DF_FMA(x, y, -p);
    acc_add(a, sg * p, sg * pe);
}
// Pair addition for the block and sequence sums of AccF values (TwoSum of the leading parts, the
// trailing parts and the rounding error added in FP32)
OVL_HD AccF accf_add(AccF a, AccF b) {
    const float s = DF_ADD(a.hi, b.hi);
    const float bb = DF_SUB(s, a.hi);
    const float e = DF_ADD(DF_SUB(a.hi, DF_SUB(s, bb)), DF_SUB(b.hi, bb));
    AccF r;
    r.hi = s;
    r.lo = DF_ADD(DF_ADD(a.lo, b.lo), e);
    return r;
}
struct AccD {
    double v = 0.0;
};
__device__ __forceinline__ void acc_prod(AccD& a, double x, double y, double sg = 1.0) { a.v += sg * x * y; }

template <class A, class R>
__device__ __forceinline__ void acc_cdot(A* a, cx<R> x, cx<R> y) {  // += conj(x) y
    acc_prod(a[0], x.r, y.r);
    acc_prod(a[0], x.i, y.i);
    acc_prod(a[1], x.r, y.i);
    acc_prod(a[1], x.i, y.r, R(-1));
}
template <class A, class R>
__device__ __forceinline__ void acc_norm2(A& a, cx<R> x) {
    acc_prod(a, x.r, x.r);
    acc_prod(a, x.i, x.i);
}

}  // namespace ovl
