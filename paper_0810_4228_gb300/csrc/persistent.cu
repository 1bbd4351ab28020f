// Persistent forms of the two passes of the mixed-precision two-sided Lanczos
// solve (Sec. 4, Eq. 4.2; two-pass procedure of Sec. 5).
//
// On lattices that hold a few thousand sites per SM the per-step kernels are
// bound by launch gaps and dependent-load latency, not by work.  Here one
// cooperative launch runs all k steps.  Every block owns fixed 32-site tiles
// for the whole solve and keeps their own-site state on chip (shared memory):
// the current and previous basis vectors and t = A v_i, s = A^dag w_i (pass 1),
// or v_i, v_{i-1} and the accumulating y (pass 2).  Only the neighbours of the
// stencil are read from global memory (through L2, since other blocks wrote
// them), and only the new basis vectors are written.
//
// Pass 1 meets the other blocks at two bounded grid barriers per step: after
// the per-block partial sums of alpha = w^dag t and |t|^2 (and of the
// re-projection coefficients L^dag t, R^dag s), and after those of
// w^^dag v^, |v^|^2, |w^|^2.  In-block sums use exact FP32 products with
// compensated (pair) accumulation; the cross-block sums and all recurrence
// scalars are FP64 and formed by a single warp -- GB300's FP64 pipe is narrow,
// so scalar algebra repeated by every warp would cost more than the stencil.  Every block adds the per-block partials
// in the same fixed order, so all blocks hold bit-identical coefficients.
// Pass 2 regenerates the basis in FP64 with one barrier per step.  The barriers
// count arrivals on a counter zeroed before each launch.
#include <algorithm>

#include "stencil_impl.cuh"

namespace ovl {

static constexpr int PT = 32;        // sites per tile
static constexpr int PW1 = 8;        // pass 1: warps per block, one hop (4 directions x fwd/bwd) each
static constexpr int PW2 = 4;        // pass 2: warps per block, both hops of one direction each
static constexpr int PMAX_TPB = 8;   // tiles per block held on chip
static constexpr int PMAX_M = 64;    // deflated vectors handled by re-projection
static constexpr long long PSPIN = 20000000;

// In-block sums of FP32 products carried as unevaluated pairs hi + lo: every product enters
// exactly (p = a b rounded, e = fma(a, b, -p) its error) and every addition keeps its rounding
// error (Knuth's TwoSum), so the block partials carry about twice FP32's precision while the
// work stays on the FP32 pipe.  The _rn intrinsics keep the compiler from contracting the
// error-free transformations into fused operations.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += a * b (sg = +1) or acc -= a * b (sg = -1)
__device__ __forceinline__ void ff_fma(ff& acc, float a, float b, float sg = 1.f) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    float s, e;
    two_sum(acc.hi, sg * p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, sg * pe));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return ff{s, __fadd_rn(__fadd_rn(a.lo, b.lo), e)};
}

// acc += conj(a) b  (re into acc[0], im into acc[1])
__device__ __forceinline__ void ff_cdot(ff* acc, cx<float> a, cx<float> b) {
    ff_fma(acc[0], a.r, b.r);
    ff_fma(acc[0], a.i, b.i);
    ff_fma(acc[1], a.r, b.i);
    ff_fma(acc[1], a.i, b.r, -1.f);
}

__device__ __forceinline__ void ff_norm2(ff& acc, cx<float> a) {
    ff_fma(acc, a.r, a.r);
    ff_fma(acc, a.i, a.i);
}

// Block sum of NQ pair-valued partials per thread (warp trees of pairs, then lane q of warp 0
// adds the warps' pairs for value q in a fixed order); the block's sums go to part[q] as pairs.
// redf: NW * NQ float2.
template <int NQ, int NW>
__device__ __forceinline__ void block_reduce_ff(ff (&v)[NQ], float2* redf, float2* part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ff u;
            u.hi = __shfl_xor_sync(0xffffffffu, v[q].hi, o);
            u.lo = __shfl_xor_sync(0xffffffffu, v[q].lo, o);
            v[q] = ff_add(v[q], u);
        }
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) redf[wid * NQ + q] = make_float2(v[q].hi, v[q].lo);
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        ff s{redf[q].x, redf[q].y};
#pragma unroll
        for (int w = 1; w < NW; ++w) s = ff_add(s, ff{redf[w * NQ + q].x, redf[w * NQ + q].y});
        part[q] = make_float2(s.hi, s.lo);
    }
    __syncthreads();
}

// Called by one full warp: out[q] = sum over blocks b < G of the pairs part[b * stride + q], q < nq,
// added as pairs in a fixed order (identical in every block) and rounded to FP64 at the end.
__device__ __forceinline__ void warp_sum_partials(const float2* part, int stride, int nq, int G, double* out) {
    const int lane = threadIdx.x & 31;
    if (nq <= 4) {
        const int q = lane >> 3, j = lane & 7;
        ff a0{0.f, 0.f}, a1{0.f, 0.f};
        if (q < nq) {
            int b = j;
#pragma unroll 4
            for (; b + 8 < G; b += 16) {
                const float2 x0 = __ldcg(part + (size_t)b * stride + q);
                const float2 x1 = __ldcg(part + (size_t)(b + 8) * stride + q);
                a0 = ff_add(a0, ff{x0.x, x0.y});
                a1 = ff_add(a1, ff{x1.x, x1.y});
            }
            if (b < G) {
                const float2 x0 = __ldcg(part + (size_t)b * stride + q);
                a0 = ff_add(a0, ff{x0.x, x0.y});
            }
        }
        ff acc = ff_add(a0, a1);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            ff u;
            u.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
            u.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
            acc = ff_add(acc, u);
        }
        if (j == 0 && q < nq) out[q] = (double)acc.hi + (double)acc.lo;
    } else {
        for (int q = 0; q < nq; ++q) {
            ff acc{0.f, 0.f};
            for (int b = lane; b < G; b += 32) {
                const float2 x = __ldcg(part + (size_t)b * stride + q);
                acc = ff_add(acc, ff{x.x, x.y});
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ff u;
                u.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
                u.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
                acc = ff_add(acc, u);
            }
            if (lane == 0) out[q] = (double)acc.hi + (double)acc.lo;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ cx<float> down(cx<double> z) { return mk((float)z.r, (float)z.i); }

struct P1Args {
    const float4* U;
    float4* v[3];
    float4* w[3];
    KState* ks;
    double2* alpha;
    double2* beta;
    double2* gamma;
    const float2* R32;  // re-projection vectors (FP32 device layout as float2 arrays)
    const float2* L32;
    int m;
    float2* partA;       // [G][4 + 4m] pair-valued block partials
    float2* partC;       // [G][4]
    unsigned int* bar;
    HopCoef<float> hv, hw;
    Geom g;
    int k;
    int ntiles;
    int tpb;
    long long spin;          // polls before a barrier wait gives up (sets ks->timeout)
    unsigned int unreach;    // added to every barrier target: 1 makes every wait run out (timeout tests)
};

// pass-1 scalars shared by the block (written by warp 0)
struct P1Shared {
    cx<float> cs[2];             // scales of the current v~, w~ (t = sv A v~, s = sw A^dag w~)
    cx<float> ca[2];             // alpha sv, conj(alpha) sw
    cx<float> cp[2];             // gamma_{i-1} svp, conj(beta_{i-1}) swp
    cx<float> pq[2][PMAX_M];     // re-projection coefficients p = L^dag t, q = R^dag s
    int done;
};

// Own-site state: slot 0/1 the current and previous vector (alternating), slot 2 t (vw = 0) and
// s (vw = 1).
__device__ __forceinline__ int st_idx(int jt, int slot, int vw, int site, int q) {
    return (((jt * 3 + slot) * 2 + vw) * PT + site) * 12 + q;
}

__global__ void __launch_bounds__(32 * PW1) k_pass1_persistent(P1Args a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<float>* dirpart = reinterpret_cast<cx<float>*>(smraw);   // [PW1][2][PT][12]
    cx<float>* st = dirpart + PW1 * 2 * PT * 12;                  // [tpb][3][2][PT][12]
    __shared__ float2 redf[PW1 * 4];
    __shared__ double coef[4 + 4 * PMAX_M];
    __shared__ double oc[4];
    __shared__ P1Shared sh;
    KState* ks = a.ks;
    int* err = &ks->timeout;
    if (ks->done || ks->status) return;
    const Geom g = a.g;
    const int G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // epilogue / recurrence thread: components q = 3 sp .. 3 sp + 2 of t (vw = 0) or s (vw = 1) at `site`
    const int site = tid >> 3, sp = (tid >> 1) & 3, vw = tid & 1;
    const int m = a.m;
    const int NA = 4 + 4 * m;
    // recurrence state in FP64, meaningful in warp 0 lane 0
    cx<double> sv = d2c(ks->sv), sw = d2c(ks->sw), svp = d2c(ks->svp), swp = d2c(ks->swp);
    cx<double> beta_prev = mk(0.0, 0.0), gamma_prev = mk(0.0, 0.0);
    double anorm2 = ks->anorm * ks->anorm;
    int kused = 0, bd = -1;
    unsigned int nbar = 0;

    // own-site start vectors into slot 0, zero previous vectors
    {
        int jt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
            const int ii = tile * PT + site;
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                const int q = 3 * sp + c3;
                cx<float> x = mk(0.f, 0.f);
                if (ii < g.V) x = ld_comp_cg<float>(vw ? a.w[0] : a.v[0], g.V, ii, q);
                st[st_idx(jt, 0, vw, site, q)] = x;
                st[st_idx(jt, 1, vw, site, q)] = mk(0.f, 0.f);
            }
        }
    }
    if (tid == 0) {
        sh.cs[0] = down(sv);
        sh.cs[1] = down(sw);
        sh.done = 0;
    }
    __syncthreads();

    for (int i = 0; i < a.k; ++i) {
        const int cur = i & 1, prv = cur ^ 1;
        const float4* vi = a.v[i % 3];
        const float4* wi = a.w[i % 3];
        // ---- phase A: t = sv A v~_i, s = sw A^dag w~_i on the own tiles
        ff pa[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int jt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
            {
                const int i0 = tile * PT + lane;
                Spinor<float> acc[2];
#pragma unroll
                for (int n = 0; n < 2; ++n)
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[n].s[s][c] = mk(0.f, 0.f);
                if (i0 < g.V) {
                    const Coord c = site_coord(g, i0);
                    const float4* const xs[2] = {vi, wi};
                    const HopCoef<float> hcs[2] = {a.hv, a.hw};
                    one_hop<LINK_F32_12, float, 2, true>(wid, g, c, i0, a.U, xs, acc, hcs);
                }
#pragma unroll
                for (int n = 0; n < 2; ++n)
#pragma unroll
                    for (int q = 0; q < 12; ++q) dirpart[((wid * 2 + n) * PT + lane) * 12 + q] = acc[n].s[q / 3][q % 3];
            }
            __syncthreads();
            const int ii = tile * PT + site;
            if (ii < g.V) {
                const cx<float> cs = sh.cs[vw];
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    const int q = 3 * sp + c3;
                    cx<float> z = st[st_idx(jt, cur, vw, site, q)];
#pragma unroll
                    for (int w8 = 0; w8 < PW1; ++w8) z = z + dirpart[((w8 * 2 + vw) * PT + site) * 12 + q];
                    if (sp >= 2) z = -z;
                    z = cs * z;
                    st[st_idx(jt, 2, vw, site, q)] = z;
                    if (vw == 0) {
                        ff_cdot(pa, st[st_idx(jt, cur, 1, site, q)], z);
                        ff_norm2(pa[2], z);
                    }
                }
            }
            __syncthreads();
        }
        // per-block partials of w~^dag t and |t|^2 (FP32 in-block, FP64 across warps)
        block_reduce_ff<3, PW1>(pa, redf, a.partA + (size_t)blockIdx.x * NA);
        // re-projection partials p_j = l_j^dag t (vw = 0 threads), q_j = r_j^dag s (vw = 1)
        for (int j = 0; j < m; ++j) {
            ff pr[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            int jt2 = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt2) {
                const int ii = tile * PT + site;
                if (ii >= g.V) continue;
                const float4* basis =
                    reinterpret_cast<const float4*>((vw ? a.R32 : a.L32) + (size_t)j * 12 * g.V);
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    const int q = 3 * sp + c3;
                    ff_cdot(pr + 2 * vw, ld_comp<float>(basis, g.V, ii, q), st[st_idx(jt2, 2, vw, site, q)]);
                }
            }
            // p_j at 4 + 2j, q_j at 4 + 2m + 2j: reduce into the block's slots 4 + 4j.. and move
            block_reduce_ff<4, PW1>(pr, redf, a.partA + (size_t)blockIdx.x * NA + 4 + 4 * j);
        }
        grid_barrier_mono(a.bar, (unsigned)G * (++nbar) + a.unreach, err, 1, a.spin);
        if (*(volatile int*)err) return;
        // ---- scalars (warp 0): alpha_i, the recurrence coefficients of phase C
        if (wid == 0) {
            warp_sum_partials(a.partA, NA, 3, G, coef);
            if (m > 0) warp_sum_partials(a.partA + 4, NA, 4 * m, G, coef + 4);
            if (lane == 0) {
                const cx<double> alpha = cdot(sw, mk(coef[0], coef[1]));
                anorm2 = fmax(anorm2, coef[2]);
                kused = i + 1;
                if (blockIdx.x == 0) a.alpha[i] = c2d(alpha);
                sh.ca[0] = down(alpha * sv);
                sh.ca[1] = down(conj(alpha) * sw);
                sh.cp[0] = down(i > 0 ? gamma_prev * svp : mk(0.0, 0.0));
                sh.cp[1] = down(i > 0 ? conj(beta_prev) * swp : mk(0.0, 0.0));
            }
            for (int j = lane; j < m; j += 32) {
                sh.pq[0][j] = mk((float)coef[4 + 4 * j], (float)coef[4 + 4 * j + 1]);
                sh.pq[1][j] = mk((float)coef[4 + 4 * j + 2], (float)coef[4 + 4 * j + 3]);
            }
        }
        if (i == a.k - 1) break;
        __syncthreads();
        // ---- phase C: the recurrence on the own sites (Eq. 4.2), reductions for beta, gamma
        ff pc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float4* const xn = vw ? a.w[(i + 1) % 3] : a.v[(i + 1) % 3];
        const cx<float> ca = sh.ca[vw], cp = sh.cp[vw];
        jt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
            const int ii = tile * PT + site;
            const bool ok = ii < g.V;
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                const int q = 3 * sp + c3;
                cx<float> z = mk(0.f, 0.f);
                if (ok) {
                    z = st[st_idx(jt, 2, vw, site, q)] - ca * st[st_idx(jt, cur, vw, site, q)];
                    if (i > 0) z = z - cp * st[st_idx(jt, prv, vw, site, q)];
                    if (m > 0) {
                        const float2* basis = vw ? a.L32 : a.R32;
                        for (int j = 0; j < m; ++j)
                            z = z - sh.pq[vw][j] *
                                        ld_comp<float>(reinterpret_cast<const float4*>(basis + (size_t)j * 12 * g.V),
                                                       g.V, ii, q);
                    }
                    st_comp<float>(xn, g.V, ii, q, z);
                    st[st_idx(jt, prv, vw, site, q)] = z;
                }
                // w^^dag v^ on the vw = 1 thread, with v^ from its partner lane
                const float pr_ = __shfl_xor_sync(0xffffffffu, z.r, 1);
                const float pi_ = __shfl_xor_sync(0xffffffffu, z.i, 1);
                if (vw) {
                    ff_cdot(pc, z, mk(pr_, pi_));
                    ff_norm2(pc[3], z);
                } else {
                    ff_norm2(pc[2], z);
                }
            }
        }
        block_reduce_ff<4, PW1>(pc, redf, a.partC + (size_t)blockIdx.x * 4);
        grid_barrier_mono(a.bar, (unsigned)G * (++nbar) + a.unreach, err, 1, a.spin);
        if (*(volatile int*)err) return;
        if (wid == 0) {
            warp_sum_partials(a.partC, 4, 4, G, oc);
            if (lane == 0) {
                const double nv2 = oc[2], nw2 = oc[3];
                const cx<double> delta = mk(oc[0], oc[1]);
                int dn = 0;
                if (nv2 <= 1e-26 * fmax(anorm2, 1e-300)) {
                    dn = 1;  // lucky breakdown: |v^| <= 1e-13 max |A v_i|
                } else if (norm2(delta) <= 1e-28 * nv2 * nw2) {
                    dn = 1;  // serious breakdown: |w^^dag v^| <= 1e-14 |v^| |w^|
                    bd = i + 1;
                } else {
                    const double rnv = rsqrt(nv2), nv = nv2 * rnv;
                    const cx<double> gm = mk(oc[0] * rnv, oc[1] * rnv);
                    beta_prev = mk(nv, 0.0);
                    gamma_prev = gm;
                    if (blockIdx.x == 0) {
                        a.beta[i] = c2d(beta_prev);
                        a.gamma[i] = c2d(gm);
                    }
                    svp = sv;
                    swp = sw;
                    sv = mk(rnv, 0.0);
                    sw = (1.0 / norm2(gm)) * gm;  // 1 / conj(gm)
                    sh.cs[0] = down(sv);
                    sh.cs[1] = down(sw);
                }
                sh.done = dn;
            }
        }
        __syncthreads();
        if (sh.done) break;
    }
    if (blockIdx.x == 0 && tid == 0) {
        ks->kused = kused;
        ks->done = 1;
        ks->anorm = sqrt(anorm2);
        if (bd >= 0) ks->bdstep = bd;
        ks->sv = c2d(sv);
        ks->sw = c2d(sw);
        ks->svp = c2d(svp);
        ks->swp = c2d(swp);
    }
}

// Per-step coefficients of the regeneration, formed once: v_{i+1} = ib (A v_i) - a' v_i - g' v_{i-1},
// ib = 1 / beta_i, a' = ib alpha_i, g' = ib gamma_{i-1}; y += c_{i+1} v_{i+1}.  Stored in the
// precision of the pass (double2, or double-float dfc).
template <class VT> struct RegenCoef {
    VT ib, a, g, c;
};
__device__ __forceinline__ void put(double2& o, cx<double> z) { o = c2d(z); }
__device__ __forceinline__ void put(dfc& o, cx<double> z) { o = c2dfc(mk(df(z.r), df(z.i))); }
__device__ __forceinline__ cx<double> get(const double2& v) { return d2c(v); }
__device__ __forceinline__ cx<df> get(const dfc& v) { return dfc2c(v); }

template <class VT>
__global__ void k_pass2_coef(const KState* ks, const double2* alpha, const double2* beta, const double2* gamma,
                             const double2* c, RegenCoef<VT>* out, int kmax, unsigned int* bar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) bar[0] = 0u;  // arrival counter of the pass-2 barriers
    if (i + 1 >= kmax || i + 1 >= ks->kused) return;
    const cx<double> ib = cdiv(mk(1.0, 0.0), d2c(beta[i]));
    RegenCoef<VT> r;
    put(r.ib, ib);
    put(r.a, ib * d2c(alpha[i]));
    put(r.g, i > 0 ? ib * d2c(gamma[i - 1]) : mk(0.0, 0.0));
    put(r.c, d2c(c[i + 1]));
    out[i] = r;
}

template <class R> struct P2Args {
    const void* U;
    void* v[3];
    double2* y;
    const KState* ks;
    const void* cf;
    unsigned int* bar;
    int* err;
    HopCoef<R> hc[1];
    Geom g;
    int ntiles;
};

// FP64 (R = double) or double-float (R = df) pass-2 state: slots 0/1 alternate as v_i and v_{i-1},
// slot 2 accumulates y
__device__ __forceinline__ int st2_idx(int jt, int slot, int site, int q) { return ((jt * 3 + slot) * PT + site) * 12 + q; }

template <class R> __device__ __forceinline__ cx<R> from_f64(double2 v);
template <> __device__ __forceinline__ cx<double> from_f64<double>(double2 v) { return d2c(v); }
template <> __device__ __forceinline__ cx<df> from_f64<df>(double2 v) { return d2df(v); }
__device__ __forceinline__ double2 to_f64(cx<double> z) { return c2d(z); }
__device__ __forceinline__ double2 to_f64(cx<df> z) { return df2d(z); }

// regeneration v_{i+1} = ((A - alpha_i) v_i - gamma_{i-1} v_{i-1}) / beta_i, y += c_{i+1} v_{i+1} (Sec. 5)
template <class R, int LF>
__global__ void __launch_bounds__(32 * PW2) k_pass2_persistent(P2Args<R> a) {
    using VT = typename VecT<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R>* dirpart = reinterpret_cast<cx<R>*>(smraw);  // [PW2][PT][12]
    cx<R>* st = dirpart + PW2 * PT * 12;               // [tpb][3][PT][12]
    if (a.ks->status || a.ks->timeout) return;  // (pass 1 gave up: the same decision in every block)
    const int kused = a.ks->kused;
    const Geom g = a.g;
    const int G = gridDim.x;
    const int tid = threadIdx.x, site = tid >> 2, sp = tid & 3;
    const int lane = tid & 31, wid = tid >> 5;
    const RegenCoef<VT>* cfs = reinterpret_cast<const RegenCoef<VT>*>(a.cf);
    {
        int jt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
            const int ii = tile * PT + site;
            const bool ok = ii < g.V;
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                const int q = 3 * sp + c3;
                st[st2_idx(jt, 0, site, q)] = ok ? ld_comp_cg<R>((const VT*)a.v[0], g.V, ii, q) : mk(R(0), R(0));
                st[st2_idx(jt, 1, site, q)] = mk(R(0), R(0));
                st[st2_idx(jt, 2, site, q)] = ok ? from_f64<R>(__ldcg(a.y + (size_t)q * g.V + ii)) : mk(R(0), R(0));
            }
        }
    }
    __syncthreads();
    RegenCoef<VT> cf;
    if (kused > 1) cf = cfs[0];
    unsigned int nbar = 0;
    for (int i = 0; i + 1 < kused; ++i) {
        const int cur = i & 1, prv = cur ^ 1;
        const VT* vi = (const VT*)a.v[i % 3];
        VT* vn = (VT*)a.v[(i + 1) % 3];
        const cx<R> ib = get(cf.ib), al = get(cf.a), gm = get(cf.g), cc = get(cf.c);
        if (i + 2 < kused) cf = cfs[i + 1];  // next step's coefficients, loaded ahead
        int jt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
            {
                const int i0 = tile * PT + lane;
                Spinor<R> acc[1];
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[0].s[s][c] = mk(R(0), R(0));
                if (i0 < g.V) {
                    const Coord c = site_coord(g, i0);
                    const VT* const xs[1] = {vi};
                    switch (wid) {
                        case 0: hops_dir<0, LF, R, 1, true>(g, c, i0, a.U, xs, acc, a.hc); break;
                        case 1: hops_dir<1, LF, R, 1, true>(g, c, i0, a.U, xs, acc, a.hc); break;
                        case 2: hops_dir<2, LF, R, 1, true>(g, c, i0, a.U, xs, acc, a.hc); break;
                        default: hops_dir<3, LF, R, 1, true>(g, c, i0, a.U, xs, acc, a.hc); break;
                    }
                }
#pragma unroll
                for (int q = 0; q < 12; ++q) dirpart[(wid * PT + lane) * 12 + q] = acc[0].s[q / 3][q % 3];
            }
            __syncthreads();
            const int ii = tile * PT + site;
            if (ii < g.V) {
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    const int q = 3 * sp + c3;
                    const cx<R> self = st[st2_idx(jt, cur, site, q)];
                    cx<R> z = self;
#pragma unroll
                    for (int w4 = 0; w4 < PW2; ++w4) z = z + dirpart[(w4 * PT + site) * 12 + q];
                    if (sp >= 2) z = -z;
                    z = ib * z - al * self;
                    if (i > 0) z = z - gm * st[st2_idx(jt, prv, site, q)];
                    st_comp<R>(vn, g.V, ii, q, z);
                    st[st2_idx(jt, prv, site, q)] = z;
                    st[st2_idx(jt, 2, site, q)] = st[st2_idx(jt, 2, site, q)] + cc * z;
                }
            }
            __syncthreads();
        }
        if (i + 2 < kused) {
            grid_barrier_mono(a.bar, (unsigned)G * (++nbar), a.err, 1, PSPIN);
            if (*(volatile int*)a.err) return;
        }
    }
    int jt = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
        const int ii = tile * PT + site;
        if (ii >= g.V) continue;
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
            const int q = 3 * sp + c3;
            a.y[(size_t)q * g.V + ii] = to_f64(st[st2_idx(jt, 2, site, q)]);
        }
    }
}

static int persistent_grid(int ntiles, int num_sms) { return std::max(1, std::min(ntiles, num_sms)); }

static size_t pass1_smem(int tpb) { return sizeof(cx<float>) * ((size_t)PW1 * 2 * PT * 12 + (size_t)tpb * 3 * 2 * PT * 12); }
static size_t pass2_smem(int tpb) { return 16 * ((size_t)PW2 * PT * 12 + (size_t)tpb * 3 * PT * 12); }

bool persistent_ok(const Geom& g, int num_sms) {
    // own-site state of every tile of a block fits in shared memory
    const int ntiles = (g.V + PT - 1) / PT;
    const int tpb = (ntiles + num_sms - 1) / num_sms;
    return tpb <= PMAX_TPB;
}

int launch_pass1_persistent(const float4* U12, float4* const v[3], float4* const w[3], KState* ks, double2* alpha,
                            double2* beta, double2* gamma, const float2* R32, const float2* L32, int m, double mu,
                            double kappa, int k, double* partials, unsigned int* bar, const Geom& g, int num_sms,
                            cudaStream_t st, long long spin, int unreachable) {
    if (m > PMAX_M) return -1;
    P1Args a;
    a.spin = spin > 0 ? spin : PSPIN;
    a.unreach = unreachable ? 1u : 0u;
    a.U = U12;
    for (int q = 0; q < 3; ++q) a.v[q] = v[q], a.w[q] = w[q];
    a.ks = ks;
    a.alpha = alpha;
    a.beta = beta;
    a.gamma = gamma;
    a.R32 = R32;
    a.L32 = L32;
    a.m = m;
    a.ntiles = (g.V + PT - 1) / PT;
    const int G = persistent_grid(a.ntiles, num_sms);
    a.tpb = (a.ntiles + G - 1) / G;
    if (a.tpb > PMAX_TPB) return -1;
    a.partA = reinterpret_cast<float2*>(partials);
    a.partC = a.partA + (size_t)G * (4 + 4 * m);
    a.bar = bar;
    a.hv = make_coef<float>(mu, kappa);
    a.hw = make_coef<float>(-mu, kappa);
    a.g = g;
    a.k = k;
    static unsigned long long attr_dev = 0;
    if (first_use_on_device(attr_dev))
        cudaFuncSetAttribute(k_pass1_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pass1_smem(PMAX_TPB));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(32 * PW1);
    cfg.dynamicSmemBytes = pass1_smem(a.tpb);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_pass1_persistent, a);
}

template <class R, int LF>
static int launch_p2(P2Args<R> a, HopCoef<R> hc, int G, int tpb, cudaStream_t st) {
    a.hc[0] = hc;
    static unsigned long long attr_dev = 0;
    if (first_use_on_device(attr_dev))
        cudaFuncSetAttribute(k_pass2_persistent<R, LF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pass2_smem(PMAX_TPB));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(32 * PW2);
    cfg.dynamicSmemBytes = pass2_smem(tpb);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_pass2_persistent<R, LF>, a);
}

int launch_pass2_persistent(const double2* U64, const float4* Udf, double2* const v[3], double2* y, const KState* ks,
                            const double2* alpha, const double2* beta, const double2* gamma, const double2* c,
                            double2* coef_work, int kmax, double mu, double kappa, unsigned int* bar, int* err,
                            const Geom& g, int num_sms, cudaStream_t st) {
    const bool dfm = Udf != nullptr;
    const int ntiles = (g.V + PT - 1) / PT;
    const int G = persistent_grid(ntiles, num_sms);
    const int tpb = (ntiles + G - 1) / G;
    auto fill = [&](auto& a) {
        a.U = dfm ? (const void*)Udf : (const void*)U64;
        for (int q = 0; q < 3; ++q) a.v[q] = v[q];
        a.y = y;
        a.ks = ks;
        a.cf = coef_work;
        a.bar = bar;
        a.err = err;
        a.g = g;
        a.ntiles = ntiles;
    };
    if (tpb > PMAX_TPB) return -1;
    if (dfm) {
        k_pass2_coef<dfc><<<(kmax + 127) / 128, 128, 0, st>>>(ks, alpha, beta, gamma, c,
                                                              reinterpret_cast<RegenCoef<dfc>*>(coef_work), kmax, bar);
        launch_f64_to_df(v[0], (size_t)12 * g.V, st);
        P2Args<df> a;
        fill(a);
        return launch_p2<df, LINK_DF>(a, make_coef<df>(mu, kappa), G, tpb, st);
    }
    k_pass2_coef<double2><<<(kmax + 127) / 128, 128, 0, st>>>(ks, alpha, beta, gamma, c,
                                                               reinterpret_cast<RegenCoef<double2>*>(coef_work), kmax,
                                                               bar);
    P2Args<double> a;
    fill(a);
    return launch_p2<double, LINK_F64>(a, make_coef<double>(mu, kappa), G, tpb, st);
}

}  // namespace ovl
