// Device templates of the Wilson stencil shared by the stencil kernels and the
// persistent Krylov kernels: hop coefficients, the eight hops of one direction
// (spin projection, SU(3) multiply, reconstruction; Sec. 1, Eq. 1.2), and
// component access in the FP64 / FP32 device layouts.
#pragma once

#include "df32.cuh"
#include "ovl_kernels.h"

namespace ovl {

template <class R> struct VecT;
template <> struct VecT<double> { using T = double2; };
template <> struct VecT<float> { using T = float4; };
template <> struct VecT<df> { using T = dfc; };

template <int LF> struct LinkReal { using R = float; };
template <> struct LinkReal<LINK_F64> { using R = double; };
template <> struct LinkReal<LINK_DF> { using R = df; };

template <int LF, class R>
__device__ __forceinline__ void load_link_any(const void* U, int V, int nu, int i, Link<R>& L) {
    if constexpr (LF == LINK_F64) load_link((const double2*)U, V, nu, i, L);
    else if constexpr (LF == LINK_DF) load_link_df((const dfc*)U, V, nu, i, L);
    else if constexpr (LF == LINK_F32_12) load_link12((const float4*)U, V, nu, i, L);
    else load_link18((const float2*)U, V, nu, i, L);
}

// Hop coefficients of one input: -kappa * (e^{+-mu} for time) for the forward
// (T^+) and backward (T^-) hop of each direction.
template <class R> struct HopCoef { R f[4], b[4]; };

template <class R> __host__ HopCoef<R> make_coef(double mu, double kappa) {
    HopCoef<R> h;
    for (int nu = 0; nu < 3; ++nu) h.f[nu] = h.b[nu] = R(-kappa);
    h.f[3] = R(-kappa * exp(mu));
    h.b[3] = R(-kappa * exp(-mu));
    return h;
}

template <bool CG, class P, class R>
__device__ __forceinline__ void load_spinor_any(const P* x, int V, int i, Spinor<R>& p) {
    if constexpr (CG) load_spinor_cg(x, V, i, p);
    else load_spinor(x, V, i, p);
}

// The forward hop (1 + gamma_nu) U_{x,nu} psi(x + nu) of direction NU for NIN inputs
// sharing the link (CG: L2-coherent vector loads, for vectors written by other
// blocks of the same kernel).
template <int NU, int LF, class R, int NIN, bool CG = false>
__device__ __forceinline__ void hop_fwd(const Geom& g, const Coord& c, int i, const void* U,
                                        const typename VecT<R>::T* const (&x)[NIN], Spinor<R> (&acc)[NIN],
                                        const HopCoef<R> (&hc)[NIN]) {
    Link<R> L;
    Spinor<R> p;
    Half<R> h, uh;
    const int f = neighbour(g, c, NU, +1);
    const R ph = (NU == 3 && c.x[3] == g.L[3] - 1) ? R(g.bc_t) : R(1);
    load_link_any<LF>(U, g.V, NU, i, L);
#pragma unroll
    for (int n = 0; n < NIN; ++n) {
        load_spinor_any<CG>(x[n], g.V, f, p);
        project<NU, +1>(p, h);
        mul_link(L, h, uh);
        recon_acc<NU, +1>(acc[n], uh, hc[n].f[NU] * ph);
    }
}

// The backward hop (1 - gamma_nu) U_{x-nu,nu}^dag psi(x - nu).
template <int NU, int LF, class R, int NIN, bool CG = false>
__device__ __forceinline__ void hop_bwd(const Geom& g, const Coord& c, int i, const void* U,
                                        const typename VecT<R>::T* const (&x)[NIN], Spinor<R> (&acc)[NIN],
                                        const HopCoef<R> (&hc)[NIN]) {
    Link<R> L;
    Spinor<R> p;
    Half<R> h, uh;
    const int b = neighbour(g, c, NU, -1);
    const R ph = (NU == 3 && c.x[3] == 0) ? R(g.bc_t) : R(1);
    load_link_any<LF>(U, g.V, NU, b, L);
#pragma unroll
    for (int n = 0; n < NIN; ++n) {
        load_spinor_any<CG>(x[n], g.V, b, p);
        project<NU, -1>(p, h);
        mul_link_dag(L, h, uh);
        recon_acc<NU, -1>(acc[n], uh, hc[n].b[NU] * ph);
    }
}

// Both hops of direction NU.
template <int NU, int LF, class R, int NIN, bool CG = false>
__device__ __forceinline__ void hops_dir(const Geom& g, const Coord& c, int i, const void* U,
                                         const typename VecT<R>::T* const (&x)[NIN], Spinor<R> (&acc)[NIN],
                                         const HopCoef<R> (&hc)[NIN]) {
    hop_fwd<NU, LF, R, NIN, CG>(g, c, i, U, x, acc, hc);
    hop_bwd<NU, LF, R, NIN, CG>(g, c, i, U, x, acc, hc);
}

// One of the eight hops, h = 0..7: direction h & 3, forward for h < 4 (uniform per warp).
template <int LF, class R, int NIN, bool CG = false>
__device__ __forceinline__ void one_hop(int h, const Geom& g, const Coord& c, int i, const void* U,
                                        const typename VecT<R>::T* const (&x)[NIN], Spinor<R> (&acc)[NIN],
                                        const HopCoef<R> (&hc)[NIN]) {
    switch (h) {
        case 0: hop_fwd<0, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        case 1: hop_fwd<1, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        case 2: hop_fwd<2, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        case 3: hop_fwd<3, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        case 4: hop_bwd<0, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        case 5: hop_bwd<1, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        case 6: hop_bwd<2, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
        default: hop_bwd<3, LF, R, NIN, CG>(g, c, i, U, x, acc, hc); break;
    }
}

// x times a unit: i x if imag, negated if neg (exact: no multiplication)
// a + b; for double-float an intermediate sum without renormalisation (df_add_lazy)
template <class R>
__device__ __forceinline__ cx<R> add_lazy(const cx<R>& a, const cx<R>& b) {
    return a + b;
}

template <class R>
__device__ __forceinline__ cx<R> unit_mul(cx<R> x, bool imag, bool neg) {
    const cx<R> y = imag ? mk(-x.i, x.r) : x;
    return neg ? -y : y;
}

// Hop h = 0..7 (direction nu = h & 3, forward for h < 4) with nu and the sign as warp-uniform
// runtime values: the spin projection of (1 +- gamma_nu) is written as selects and sign flips, so
// every warp of a direction-split block runs the same instructions (one copy of the hop in the
// instruction cache instead of eight).  Same arithmetic as hop_fwd / hop_bwd up to the half
// spinor: out = coefficient x U (or U^dag) x (projected half spinor) of the neighbour; the full
// four-spin contribution is hop_spin(h, sp, out.h[0], out.h[1]).
template <int LF, class R, int NIN>
__device__ __forceinline__ void hop_half_uniform(int h, const Geom& g, const Coord& c, int i, const void* U,
                                                 const typename VecT<R>::T* const (&x)[NIN], Half<R> (&out)[NIN],
                                                 const HopCoef<R> (&hc)[NIN]) {
    const int nu = h & 3;
    const bool fwd = h < 4;
    int y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        int v = c.x[d];
        if (d == nu) {
            v += fwd ? 1 : -1;
            if (v == g.L[d]) v = 0;
            if (v < 0) v = g.L[d] - 1;
        }
        y[d] = v;
    }
    const int nb = internal_index(g, y);
    const bool edge = fwd ? (c.x[3] == g.L[3] - 1) : (c.x[3] == 0);
    const R ph = (nu == 3 && edge) ? R(g.bc_t) : R(1);
    Link<R> L;
    load_link_any<LF>(U, g.V, nu, fwd ? i : nb, L);
    // (1 + S gamma_nu), S = +1 forward, -1 backward, chiral basis: upper spins
    // h0 = p0 + u0 p[2 or 3], h1 = p1 + u1 p[3 or 2]
    const bool hi2 = nu >= 2, im = (nu & 1) == 0;
    const bool n0 = (nu == 3) ? !fwd : fwd;
    const bool n1 = (nu == 0) ? fwd : !fwd;
#pragma unroll
    for (int n = 0; n < NIN; ++n) {
        Spinor<R> p;
        load_spinor(x[n], g.V, nb, p);
        Half<R> hh, uh;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            hh.h[0][a] = add_lazy(p.s[0][a], unit_mul(hi2 ? p.s[2][a] : p.s[3][a], im, n0));
            hh.h[1][a] = add_lazy(p.s[1][a], unit_mul(hi2 ? p.s[3][a] : p.s[2][a], im, n1));
        }
        if (fwd) mul_link(L, hh, uh);
        else mul_link_dag(L, hh, uh);
        const R cf = (fwd ? (nu == 3 ? hc[n].f[3] : hc[n].f[0]) : (nu == 3 ? hc[n].b[3] : hc[n].b[0])) * ph;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out[n].h[0][a] = cf * uh.h[0][a];
            out[n].h[1][a] = cf * uh.h[1][a];
        }
    }
}

// Spin sp of hop h's contribution rebuilt from its half spinor (h0, h1): the upper spins are h0,
// h1, the lower ones +-h or +-i h of one of them (the (1 +- gamma_nu) structure in the chiral
// basis).  With h and sp compile-time constants this is a select of a component and a sign.
template <class R>
__device__ __forceinline__ cx<R> hop_spin(int h, int sp, const cx<R>& h0, const cx<R>& h1) {
    const int nu = h & 3;
    const bool fwd = h < 4;
    const bool hi2 = nu >= 2, im = (nu & 1) == 0;
    const bool nA = !fwd;
    const bool nB = (nu == 0 || nu == 3) ? !fwd : fwd;
    if (sp == 0) return h0;
    if (sp == 1) return h1;
    if (sp == 2) return unit_mul(hi2 ? h0 : h1, im, nA);
    return unit_mul(hi2 ? h1 : h0, im, nB);
}

// The hopping term of site i for NIN inputs (CG: L2-coherent vector loads, for vectors written by
// other blocks of the same kernel).
template <int LF, class R, int NIN, bool CG = false>
__device__ __forceinline__ void apply_site(const Geom& g, int i, const void* U,
                                           const typename VecT<R>::T* const (&x)[NIN], Spinor<R> (&acc)[NIN],
                                           const HopCoef<R> (&hc)[NIN]) {
    const Coord c = site_coord(g, i);
#pragma unroll
    for (int n = 0; n < NIN; ++n)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[n].s[s][a] = mk(R(0), R(0));
    hops_dir<0, LF, R, NIN, CG>(g, c, i, U, x, acc, hc);
    hops_dir<1, LF, R, NIN, CG>(g, c, i, U, x, acc, hc);
    hops_dir<2, LF, R, NIN, CG>(g, c, i, U, x, acc, hc);
    hops_dir<3, LF, R, NIN, CG>(g, c, i, U, x, acc, hc);
}

// add the diagonal term and apply gamma5 = diag(1, 1, -1, -1)
template <class R>
__device__ __forceinline__ void finish_site(Spinor<R>& acc, const Spinor<R>& self, bool g5) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> z = acc.s[s][a] + self.s[s][a];
            acc.s[s][a] = (g5 && s >= 2) ? -z : z;
        }
}

template <class R> __device__ __forceinline__ cx<R> ld_comp(const typename VecT<R>::T* x, int V, int i, int q);
template <> __device__ inline cx<double> ld_comp<double>(const double2* x, int V, int i, int q) {
    const double2 v = __ldg(x + (size_t)q * V + i);
    return mk(v.x, v.y);
}
template <> __device__ inline cx<float> ld_comp<float>(const float4* x, int V, int i, int q) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(x) + ((size_t)(q >> 1) * V + i) * 2 + (q & 1));
    return mk(v.x, v.y);
}
template <class R> __device__ __forceinline__ void st_comp(typename VecT<R>::T* x, int V, int i, int q, cx<R> z);
// L2-coherent component load
template <class R> __device__ __forceinline__ cx<R> ld_comp_cg(const typename VecT<R>::T* x, int V, int i, int q);
template <> __device__ inline cx<double> ld_comp_cg<double>(const double2* x, int V, int i, int q) {
    const double2 v = __ldcg(x + (size_t)q * V + i);
    return mk(v.x, v.y);
}
template <> __device__ inline cx<float> ld_comp_cg<float>(const float4* x, int V, int i, int q) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(x) + ((size_t)(q >> 1) * V + i) * 2 + (q & 1));
    return mk(v.x, v.y);
}
template <> __device__ inline cx<df> ld_comp_cg<df>(const dfc* x, int V, int i, int q) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(x) + (size_t)q * V + i);
    return mk(df(v.x, v.y), df(v.z, v.w));
}
template <> __device__ inline void st_comp<df>(dfc* x, int V, int i, int q, cx<df> z) {
    x[(size_t)q * V + i] = c2dfc(z);
}
template <> __device__ inline void st_comp<double>(double2* x, int V, int i, int q, cx<double> z) {
    x[(size_t)q * V + i] = make_double2(z.r, z.i);
}
template <> __device__ inline void st_comp<float>(float4* x, int V, int i, int q, cx<float> z) {
    reinterpret_cast<float2*>(x)[((size_t)(q >> 1) * V + i) * 2 + (q & 1)] = make_float2(z.r, z.i);
}


}  // namespace ovl
