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

}  // namespace ovl
