// Batched two-sided Lanczos solves: several right-hand sides on several gauge
// configurations (lattices of different sizes) in one sequence of launches,
// captured once as a CUDA graph.
//
// A sequence is one (configuration, right-hand side) pair.  Each batched kernel
// covers every sequence in one launch: its blocks are a concatenation of
// per-sequence block ranges (a device table maps a block to its sequence), so
// lattices of any size share the GPU in every step.  Reductions are per
// sequence: block partials and a ticket counter of their own, the last block
// of a sequence sums its partials in a fixed order and sets the coefficients
// (Sec. 4, Eq. 4.2).  A finished sequence (lucky breakdown, k reached) skips
// the rest of its work uniformly.  The links of a configuration are read by all
// of its right-hand sides in the same step and stay in L2 between them.
//
// Mixed precision (OVL_MIXED): pass 1 in FP32 with 12-real links (in-block sums
// of exact FP32 products in compensated pairs), pass 2 regenerates the basis
// from the pass-1 coefficients and accumulates y (Sec. 5) in double-float
// arithmetic (df32.cuh; native FP64 with OVL_PASS2_F64).  Otherwise
// FP64 throughout: one pass with the basis stored and the combination
// y = sum_i c_i v_i at the end, or, with OVL_TWO_PASS or when the basis would
// exceed 32 GiB, an FP64 pass 1 followed by the FP64 regeneration pass.
#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ctx.h"
#include "stencil_impl.cuh"

namespace ovl {

struct BSeq {
    Geom g;
    size_t n;                 // 12 V
    const void* U;            // pass-1 links: FP32-12 (float4) or FP64 (double2)
    const double2* U64;       // FP64 links (regeneration)
    const void* Udf;          // double-float links (regeneration of mixed solves)
    const int* nbr;           // [8][V] neighbour table of the lattice (regeneration)
    void* v[3];               // pass-1 ring (FP32 float4 pairs or FP64); unused with a stored basis
    void* w[3];
    void* t;
    void* s;
    double2* V;               // FP64 one-pass: stored basis, k + 1 vectors (else null)
    double2* r[3];            // FP64 regeneration ring (two-pass)
    double2* y;
    KState* ks;
    double2* alpha;
    double2* beta;
    double2* gamma;
    double2* cvec;
    double2* vscale;
    double2* part;            // [nblk][4] block partials of the batched kernels
    unsigned int* cnt;        // ticket of this sequence
    int blk0[3], nblk[3];     // block range in the pass-1 launches, per site-block shape (64, 128, 256 sites)
    int tile0, ntile;         // tile range in the tiled launches (tiles of TT sites)
};

namespace {

// pass-1 site-block shapes (sites = threads per block), picked per batch by the autotuner
constexpr int NSHAPE = 3;
constexpr int SHAPE_SITES[NSHAPE] = {64, 128, 256};
constexpr int TT = 32;   // sites per tile of the direction-split kernels (one warp per direction)

template <class R> struct BVec;
template <> struct BVec<float> { using T = float4; };
template <> struct BVec<double> { using T = double2; };

template <class R> struct AccOf;
template <> struct AccOf<float> { using T = AccF; };
template <> struct AccOf<double> { using T = AccD; };

// accf_add(AccF, AccF), the pair addition of the block and sequence sums, is in df32.cuh
__device__ __forceinline__ AccF acc_shfl(AccF a, int o) {
    AccF r;
    r.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    r.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    return r;
}
__device__ __forceinline__ AccD accf_add(AccD a, AccD b) {
    AccD r;
    r.v = a.v + b.v;
    return r;
}
__device__ __forceinline__ AccD acc_shfl(AccD a, int o) {
    AccD r;
    r.v = __shfl_xor_sync(0xffffffffu, a.v, o);
    return r;
}
__device__ __forceinline__ double2 acc_store(AccF a) { return make_double2((double)a.hi, (double)a.lo); }
__device__ __forceinline__ double2 acc_store(AccD a) { return make_double2(a.v, 0.0); }
__device__ __forceinline__ AccF acc_load(double2 v, AccF) {
    AccF r;
    r.hi = (float)v.x;
    r.lo = (float)v.y;
    return r;
}
__device__ __forceinline__ AccD acc_load(double2 v, AccD) {
    AccD r;
    r.v = v.x;
    return r;
}

// Per-sequence reduction of NQ accumulators (in their own arithmetic: compensated FP32 pairs for FP32
// data, FP64 otherwise): warp trees, the block's warps in a fixed order into part[local], then the
// last block of the sequence (ticket) adds the partials of its nblk blocks in a fixed order.
// Returns true in the last block; out[] (FP64) is valid in thread 0 there.
template <int NQ, int NW, class A>
__device__ bool seq_reduce(A (&v)[NQ], double2* part, unsigned int* cnt, int local, int nblk, double (&out)[NQ]) {
    __shared__ double2 red[NQ][NW];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        A x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = accf_add(x, acc_shfl(x, o));
        if (lane == 0) red[q][wid] = acc_store(x);
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        A sacc = acc_load(red[q][0], A());
        for (int w = 1; w < NW; ++w) sacc = accf_add(sacc, acc_load(red[q][w], A()));
        part[(size_t)local * 4 + q] = acc_store(sacc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(cnt, 1u);
        last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // one warp per value (a warp takes several when the block has fewer warps than values): lanes
    // over the blocks, then the warp tree (fixed order)
    for (int qv = wid; qv < NQ; qv += NW) {
        A acc = acc_load(make_double2(0.0, 0.0), A());
        for (int b = lane; b < nblk; b += 32) acc = accf_add(acc, acc_load(__ldcg(&part[(size_t)b * 4 + qv]), A()));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = accf_add(acc, acc_shfl(acc, o));
        if (lane == 0) red[qv][0] = acc_store(acc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < NQ; ++q) out[q] = red[q][0].x + red[q][0].y;
        *cnt = 0u;
    }
    return true;
}

// Programmatic dependent launch: the batched kernels of one solve follow each other on one
// stream and are launched with programmatic stream serialisation, so a kernel's blocks may be
// scheduled while the previous kernel drains.  Each kernel waits here (full completion and memory
// visibility of the previous grid) before it reads anything the previous kernel wrote, and lets
// the next kernel be scheduled once all of its own blocks have started.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class R>
__device__ __forceinline__ void* vslot(const BSeq& q, int j, bool wvec) {
    if (!wvec && q.V) return q.V + (size_t)j * q.n;
    return wvec ? q.w[j % 3] : q.v[j % 3];
}

// t = sv A v~_i, s = sw A^dag w~_i at every site of every running sequence; alpha_i = w_i^dag t.
// The grid's y index splits the two stencils (y = 0: t and the alpha partials; y = 1: s), so a
// thread carries one accumulator spinor instead of two (fewer registers: more warps per SM).
// The last step's s (i = klast) is not used, so the y = 1 blocks may skip it once the sequence
// is marked done.
// The FP32 form is compiled for 768 resident threads per SM (at most 80 registers): measured on the
// 48-sequence batch, pass 1 137.1 -> 134.3 ms (64-site blocks) and 145.4 -> 134.7 ms (128).
template <int LF, class R, int SH>
__global__ void __launch_bounds__(SHAPE_SITES[SH], LF == LINK_F64 ? 1 : 768 / SHAPE_SITES[SH]) k_b_pair(
    const BSeq* __restrict__ S, const int* __restrict__ bseq, int i, int klast, HopCoef<R> hv, HopCoef<R> hw) {
    using VT = typename BVec<R>::T;
    const BSeq& q = S[bseq[blockIdx.x]];  // set-up data, not written by the solve
    KState* ks = q.ks;
    pdl_wait_and_release();
    if (ks->done || ks->status) return;
    constexpr int BT = SHAPE_SITES[SH];
    const int local = blockIdx.x - q.blk0[SH];
    const int site = local * BT + threadIdx.x;
    const VT* vi = (const VT*)vslot<R>(q, i, false);
    const VT* wi = (const VT*)vslot<R>(q, i, true);
    if (blockIdx.y == 1) {  // s = sw A^dag w~
        if (site < q.g.V) {
            const cx<R> sw = mk((R)ks->sw.x, (R)ks->sw.y);
            const VT* const xs[1] = {wi};
            const HopCoef<R> hcs[1] = {hw};
            Spinor<R> acc[1], self;
            apply_site<LF, R, 1>(q.g, site, q.U, xs, acc, hcs);
            load_spinor(wi, q.g.V, site, self);
            finish_site(acc[0], self, true);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[0].s[sp][c] = sw * acc[0].s[sp][c];
            store_spinor((VT*)q.s, q.g.V, site, acc[0]);
        }
        return;
    }
    typename AccOf<R>::T a[3];
    if (site < q.g.V) {
        const cx<R> sv = mk((R)ks->sv.x, (R)ks->sv.y);
        const VT* const xs[1] = {vi};
        const HopCoef<R> hcs[1] = {hv};
        Spinor<R> acc[1], self;
        apply_site<LF, R, 1>(q.g, site, q.U, xs, acc, hcs);
        load_spinor(vi, q.g.V, site, self);
        finish_site(acc[0], self, true);
        load_spinor(wi, q.g.V, site, self);  // w~ at the own site: alpha = conj(sw) w~^dag t
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[0].s[sp][c] = sv * acc[0].s[sp][c];
                acc_cdot(a, self.s[sp][c], acc[0].s[sp][c]);
                acc_norm2(a[2], acc[0].s[sp][c]);
            }
        store_spinor((VT*)q.t, q.g.V, site, acc[0]);
    }
    double o[3];
    if (seq_reduce<3, BT / 32>(a, q.part, q.cnt, local, q.nblk[SH], o) && threadIdx.x == 0) {
        const cx<double> alpha = cdot(d2c(ks->sw), mk(o[0], o[1]));  // conj(sw) w~^dag t
        q.alpha[i] = c2d(alpha);
        ks->anorm = fmax(ks->anorm, sqrt(o[2]));
        ks->kused = i + 1;
        if (i >= klast) ks->done = 1;
    }
}

// 16-byte chunks of a device-layout vector: FP32 float4 = two complex, FP64 double2 = one
template <class R> struct Chunk;
template <> struct Chunk<float> {
    static constexpr int N = 6, P = 2;
    static __device__ __forceinline__ void split(const float4 v, cx<float> (&z)[2]) {
        z[0] = mk(v.x, v.y);
        z[1] = mk(v.z, v.w);
    }
    static __device__ __forceinline__ float4 join(const cx<float> (&z)[2]) {
        return make_float4(z[0].r, z[0].i, z[1].r, z[1].i);
    }
};
template <> struct Chunk<double> {
    static constexpr int N = 12, P = 1;
    static __device__ __forceinline__ void split(const double2 v, cx<double> (&z)[1]) { z[0] = mk(v.x, v.y); }
    static __device__ __forceinline__ double2 join(const cx<double> (&z)[1]) { return make_double2(z[0].r, z[0].i); }
};

// v^ = t - alpha v_i - gamma_{i-1} v_{i-1}, w^ = s - conj(alpha) w_i - conj(beta_{i-1}) w_{i-1};
// w^^dag v^, |v^|^2, |w^|^2 -> beta_i, gamma_i, the scales, breakdown checks (Eq. 4.2).  Element by
// element: one 16-byte chunk of each operand at a time (few registers, many warps per SM).
// The FP32 form is compiled for 1536 resident threads per SM (at most 40 registers): measured on the
// 48-sequence batch, pass 1 134.9 -> 130.9 ms (128-site blocks).
template <class R, int SH>
__global__ void __launch_bounds__(SHAPE_SITES[SH], sizeof(R) == 4 ? 1536 / SHAPE_SITES[SH] : 1)
    k_b_lstep(const BSeq* __restrict__ S, const int* __restrict__ bseq, int i) {
    using VT = typename BVec<R>::T;
    using CH = Chunk<R>;
    constexpr int P = CH::P;
    const BSeq& q = S[bseq[blockIdx.x]];  // set-up data, not written by the solve
    KState* ks = q.ks;
    pdl_wait_and_release();
    if (ks->done || ks->status) return;
    __shared__ cx<R> cf[4];
    if (threadIdx.x == 0) {
        const cx<double> a = d2c(q.alpha[i]);
        const cx<double> ca = a * d2c(ks->sv), da = conj(a) * d2c(ks->sw);
        const cx<double> cg = i > 0 ? d2c(q.gamma[i - 1]) * d2c(ks->svp) : mk(0.0, 0.0);
        const cx<double> db = i > 0 ? conj(d2c(q.beta[i - 1])) * d2c(ks->swp) : mk(0.0, 0.0);
        cf[0] = mk((R)ca.r, (R)ca.i);
        cf[1] = mk((R)da.r, (R)da.i);
        cf[2] = mk((R)cg.r, (R)cg.i);
        cf[3] = mk((R)db.r, (R)db.i);
    }
    __syncthreads();
    constexpr int BT = SHAPE_SITES[SH];
    const int local = blockIdx.x - q.blk0[SH];
    const int site = local * BT + threadIdx.x;
    typename AccOf<R>::T a[4];
    if (site < q.g.V) {
        const size_t V = (size_t)q.g.V;
        const VT* tp = (const VT*)q.t;
        const VT* sp_ = (const VT*)q.s;
        const VT* vp = (const VT*)vslot<R>(q, i, false);
        const VT* wp = (const VT*)vslot<R>(q, i, true);
        const VT* vmp = (const VT*)vslot<R>(q, i > 0 ? i - 1 : i, false);
        const VT* wmp = (const VT*)vslot<R>(q, i > 0 ? i - 1 : i, true);
        VT* vn = (VT*)vslot<R>(q, i + 1, false);
        VT* wn = (VT*)vslot<R>(q, i + 1, true);
        const cx<R> c0 = cf[0], c1 = cf[1], c2 = cf[2], c3 = cf[3];
#pragma unroll 2
        for (int ch = 0; ch < CH::N; ++ch) {
            const size_t e = (size_t)ch * V + site;
            cx<R> t[P], s[P], vv[P], ww[P], vm[P], wm[P];
            CH::split(__ldg(tp + e), t);
            CH::split(__ldg(sp_ + e), s);
            CH::split(__ldg(vp + e), vv);
            CH::split(__ldg(wp + e), ww);
            if (i > 0) {
                CH::split(__ldg(vmp + e), vm);
                CH::split(__ldg(wmp + e), wm);
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                cx<R> x = t[p] - c0 * vv[p];
                cx<R> y = s[p] - c1 * ww[p];
                if (i > 0) {
                    x = x - c2 * vm[p];
                    y = y - c3 * wm[p];
                }
                t[p] = x;
                s[p] = y;
                acc_cdot(a, y, x);
                acc_norm2(a[2], x);
                acc_norm2(a[3], y);
            }
            vn[e] = CH::join(t);
            wn[e] = CH::join(s);
        }
    }
    double o[4];
    if (seq_reduce<4, BT / 32>(a, q.part, q.cnt, local, q.nblk[SH], o) && threadIdx.x == 0) {
        const double nv = sqrt(o[2]), nw = sqrt(o[3]);
        const cx<double> delta = mk(o[0], o[1]);
        if (nv <= 1e-13 * fmax(ks->anorm, 1e-300)) {
            ks->done = 1;  // lucky breakdown
        } else if (sqrt(norm2(delta)) <= 1e-14 * nv * nw) {
            ks->done = 1;  // serious breakdown
            ks->bdstep = i + 1;
        } else {
            const cx<double> gm = mk(o[0] / nv, o[1] / nv);
            q.beta[i] = make_double2(nv, 0.0);
            q.gamma[i] = c2d(gm);
            ks->svp = ks->sv;
            ks->swp = ks->sw;
            ks->sv = make_double2(1.0 / nv, 0.0);
            ks->sw = c2d(cdiv(mk(1.0, 0.0), conj(gm)));
            q.vscale[i + 1] = ks->sv;
        }
    }
}

// ---- persistent batched pass 1 (all sites of the batch resident at once) ----------------------
// One cooperative launch runs the whole FP32 pass 1 of every sequence: one thread per site, blocks
// of BP1_T sites, each block within one sequence.  Per step: phase A, t = sv A v~_i and
// s = sw A^dag w~_i at the own site (kept in registers), block partials of w~^dag t and |t|^2;
// the sequence's blocks meet at a bounded barrier (a monotonic counter per sequence); every block
// sums the sequence's partials in the same fixed order, so all of them hold the same alpha_i;
// phase C, the recurrence of Eq. 4.2 at the own site (v^, w^ stored: the neighbours' next
// stencil reads them), partials of w^^dag v^, |v^|^2, |w^|^2; second barrier; every block forms
// beta_i, gamma_i, the scales and the breakdown decisions, identically.  Sequences finish
// independently.  Vector loads go through L2 (.cg): the ring slots are rewritten during the launch.
constexpr int BP1_T = 128;
constexpr long long BP1_SPIN = 20000000;  // polls before a barrier wait gives up (sets ks->timeout)

struct BP1Args {
    const BSeq* S;
    const int* bseq;      // block -> sequence (blocks of BP1_T sites: the pass-1 shape 1 tables)
    unsigned int* bar;    // one barrier counter per sequence, zero at launch
    int k;
    HopCoef<float> hv, hw;
};

// Block sum of NQ compensated pairs into part[local * 4 + q] (warp trees, then the warps in order).
template <int NQ>
__device__ __forceinline__ void bp1_block_partial(AccF (&v)[NQ], double2* part, int local) {
    __shared__ double2 red[NQ][BP1_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        AccF x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = accf_add(x, acc_shfl(x, o));
        if (lane == 0) red[q][wid] = acc_store(x);
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        AccF sacc = acc_load(red[q][0], AccF());
        for (int w = 1; w < BP1_T / 32; ++w) sacc = accf_add(sacc, acc_load(red[q][w], AccF()));
        part[(size_t)local * 4 + q] = acc_store(sacc);
    }
}

// The sequence's sums of NQ values over its nblk block partials, in a fixed order (lanes over the
// blocks, then the warp tree), one warp per value; out (shared) is valid in all threads on return.
template <int NQ>
__device__ __forceinline__ void bp1_seq_sum(const double2* part, int nblk, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int qv = wid; qv < NQ; qv += BP1_T / 32) {
        AccF acc = acc_load(make_double2(0.0, 0.0), AccF());
        for (int b = lane; b < nblk; b += 32) acc = accf_add(acc, acc_load(__ldcg(&part[(size_t)b * 4 + qv]), AccF()));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = accf_add(acc, acc_shfl(acc, o));
        if (lane == 0) {
            const double2 r = acc_store(acc);
            out[qv] = r.x + r.y;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ cx<float> f32c(cx<double> z) { return mk((float)z.r, (float)z.i); }

struct BP1Scalars {
    cx<double> sv, sw, svp, swp, beta_prev, gamma_prev;
    double anorm;
    int kused, bd;
};

template <int LF>
__global__ void __launch_bounds__(BP1_T, 3) k_bp1(BP1Args a) {
    const int sidx = a.bseq[blockIdx.x];
    const BSeq& q = a.S[sidx];
    KState* ks = q.ks;
    if (ks->done || ks->status) return;  // the whole sequence leaves (written before this launch)
    __shared__ cx<float> cs[2];          // sv, sw of the current step
    __shared__ cx<float> cc[4];          // alpha sv, conj(alpha) sw, gamma_{i-1} svp, conj(beta_{i-1}) swp
    __shared__ double osum[4];
    __shared__ int sdone;
    const int local = blockIdx.x - q.blk0[1], nblk = q.nblk[1];
    const int site = local * BP1_T + threadIdx.x;
    const bool ok = site < q.g.V;
    const int V = q.g.V;
    unsigned int* bar = a.bar + sidx;
    int* err = &ks->timeout;
    double2* partA = q.part;
    double2* partC = q.part + (size_t)nblk * 4;
    // recurrence scalars in FP64, meaningful in thread 0 (identical in every block of the sequence)
    // recurrence scalars in FP64, used by thread 0 only (shared: no registers in the other threads)
    __shared__ BP1Scalars sc;
    if (threadIdx.x == 0) {
        sc.sv = d2c(ks->sv), sc.sw = d2c(ks->sw), sc.svp = d2c(ks->svp), sc.swp = d2c(ks->swp);
        sc.beta_prev = mk(0.0, 0.0), sc.gamma_prev = mk(0.0, 0.0);
        sc.anorm = ks->anorm;
        sc.kused = 0, sc.bd = -1;
        cs[0] = f32c(sc.sv);
        cs[1] = f32c(sc.sw);
    }
    __syncthreads();
    unsigned int nb = 0;
    for (int i = 0; i < a.k; ++i) {
        const float4* vi = (const float4*)q.v[i % 3];
        const float4* wi = (const float4*)q.w[i % 3];
        // ---- phase A
        AccF pa[3];
        Spinor<float> t, s;
        if (ok) {
            const float4* const xs[2] = {vi, wi};
            const HopCoef<float> hcs[2] = {a.hv, a.hw};
            Spinor<float> acc[2], self[2];
            apply_site<LF, float, 2, true>(q.g, site, q.U, xs, acc, hcs);
            load_spinor_cg(vi, V, site, self[0]);
            load_spinor_cg(wi, V, site, self[1]);
            finish_site(acc[0], self[0], true);
            finish_site(acc[1], self[1], true);
            t = acc[0];
            s = acc[1];
            const cx<float> fsv = cs[0], fsw = cs[1];
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    t.s[sp][c] = fsv * t.s[sp][c];
                    s.s[sp][c] = fsw * s.s[sp][c];
                    acc_cdot(pa, self[1].s[sp][c], t.s[sp][c]);
                    acc_norm2(pa[2], t.s[sp][c]);
                }
        }
        bp1_block_partial<3>(pa, partA, local);
        grid_barrier_mono(bar, (unsigned)nblk * (++nb), err, 1, BP1_SPIN);
        if (*(volatile int*)err) return;
        bp1_seq_sum<3>(partA, nblk, osum);
        if (threadIdx.x == 0) {
            const cx<double> alpha = cdot(sc.sw, mk(osum[0], osum[1]));  // conj(sw) w~^dag t
            sc.anorm = fmax(sc.anorm, sqrt(osum[2]));
            sc.kused = i + 1;
            if (local == 0) q.alpha[i] = c2d(alpha);
            cc[0] = f32c(alpha * sc.sv);
            cc[1] = f32c(conj(alpha) * sc.sw);
            cc[2] = f32c(i > 0 ? sc.gamma_prev * sc.svp : mk(0.0, 0.0));
            cc[3] = f32c(i > 0 ? conj(sc.beta_prev) * sc.swp : mk(0.0, 0.0));
        }
        if (i == a.k - 1) break;
        __syncthreads();
        // ---- phase C: v^ = t - alpha v_i - gamma_{i-1} v_{i-1}, w^ likewise (Eq. 4.2)
        AccF pc[4];
        if (ok) {
            const cx<float> ca = cc[0], da = cc[1], cg = cc[2], db = cc[3];
            Spinor<float> vv, ww, vm, wm;
            load_spinor_cg(vi, V, site, vv);
            load_spinor_cg(wi, V, site, ww);
            if (i > 0) {
                load_spinor_cg((const float4*)q.v[(i + 2) % 3], V, site, vm);
                load_spinor_cg((const float4*)q.w[(i + 2) % 3], V, site, wm);
            }
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cx<float> x = t.s[sp][c] - ca * vv.s[sp][c];
                    cx<float> y = s.s[sp][c] - da * ww.s[sp][c];
                    if (i > 0) {
                        x = x - cg * vm.s[sp][c];
                        y = y - db * wm.s[sp][c];
                    }
                    t.s[sp][c] = x;
                    s.s[sp][c] = y;
                    acc_cdot(pc, y, x);
                    acc_norm2(pc[2], x);
                    acc_norm2(pc[3], y);
                }
            store_spinor((float4*)q.v[(i + 1) % 3], V, site, t);
            store_spinor((float4*)q.w[(i + 1) % 3], V, site, s);
        }
        bp1_block_partial<4>(pc, partC, local);
        grid_barrier_mono(bar, (unsigned)nblk * (++nb), err, 1, BP1_SPIN);
        if (*(volatile int*)err) return;
        bp1_seq_sum<4>(partC, nblk, osum);
        if (threadIdx.x == 0) {
            const double nv = sqrt(osum[2]), nw = sqrt(osum[3]);
            const cx<double> delta = mk(osum[0], osum[1]);
            int dn = 0;
            if (nv <= 1e-13 * fmax(sc.anorm, 1e-300)) {
                dn = 1;  // lucky breakdown
            } else if (sqrt(norm2(delta)) <= 1e-14 * nv * nw) {
                dn = 1;  // serious breakdown
                sc.bd = i + 1;
            } else {
                const cx<double> gm = mk(osum[0] / nv, osum[1] / nv);
                sc.beta_prev = mk(nv, 0.0);
                sc.gamma_prev = gm;
                sc.svp = sc.sv;
                sc.swp = sc.sw;
                sc.sv = mk(1.0 / nv, 0.0);
                sc.sw = cdiv(mk(1.0, 0.0), conj(gm));
                if (local == 0) {
                    q.beta[i] = make_double2(nv, 0.0);
                    q.gamma[i] = c2d(gm);
                    q.vscale[i + 1] = c2d(sc.sv);
                }
                cs[0] = f32c(sc.sv);
                cs[1] = f32c(sc.sw);
            }
            sdone = dn;
        }
        __syncthreads();
        if (sdone) break;
    }
    if (local == 0 && threadIdx.x == 0) {
        ks->kused = sc.kused;
        ks->done = 1;
        ks->anorm = sc.anorm;
        if (sc.bd >= 0) ks->bdstep = sc.bd;
        ks->sv = c2d(sc.sv);
        ks->sw = c2d(sc.sw);
        ks->svp = c2d(sc.svp);
        ks->swp = c2d(sc.swp);
    }
}

// Regeneration (Sec. 5): r_{i+1} = ((A - alpha_i) r_i - gamma_{i-1} r_{i-1}) / beta_i, y += c_{i+1} r_{i+1},
// in FP64 (R = double) or double-float (R = df; ring and y converted beforehand).  One block per
// 32-site tile of a sequence: warp h applies hop h (direction-uniform code) to the tile's sites, the
// eight partial sums meet in shared memory, and 128 threads (site, spin) finish three components each.
template <class R> __device__ __forceinline__ cx<R> cvt_coef(cx<double> z);
template <> __device__ __forceinline__ cx<double> cvt_coef<double>(cx<double> z) { return z; }
template <> __device__ __forceinline__ cx<df> cvt_coef<df>(cx<double> z) { return mk(df(z.r), df(z.i)); }

// Hop h of the double-float regeneration at site i, written straight to out[0..6) (the half
// spinor, spins 0 and 1, colours 0..2, times the hop coefficient): spin row by spin row, the
// neighbour's two spin components that row needs are projected and the link applied row by row (U)
// or column by column (U^dag), so that only one projected row, one link row and two accumulators
// are live at a time (few registers: six blocks per SM with little spilling; measured on the
// 48-sequence batch, pass 2 317.9 -> 305.2 ms against projecting both rows first).  The link is
// read once per spin row (the second time from L1).  The operations and their order per output are
// those of hop_half_uniform with mul_link / mul_link_dag, so the results are the same.
__device__ __forceinline__ void hop_half_rows_df(int h, const Geom& g, const int* __restrict__ nbr, int i,
                                                 const dfc* __restrict__ U, const dfc* __restrict__ x,
                                                 const HopCoef<df>& hc, cx<df>* __restrict__ out) {
    const int nu = h & 3;
    const bool fwd = h < 4;
    // neighbour and boundary phase from the lattice's table (no coordinate arithmetic per hop)
    const int ne = __ldg(nbr + (size_t)h * g.V + i);
    const int nb = ne < 0 ? ~ne : ne;
    const df ph = ne < 0 ? df(-1) : df(1);
    const bool hi2 = nu >= 2, im = (nu & 1) == 0;
    const bool n0 = (nu == 3) ? !fwd : fwd;
    const bool n1 = (nu == 0) ? fwd : !fwd;
    const float4* xv = reinterpret_cast<const float4*>(x);
    const size_t V = (size_t)g.V;
    auto ldx = [&](int q) {
        const float4 v = __ldg(xv + (size_t)q * V + nb);
        return mk(df(v.x, v.y), df(v.z, v.w));
    };
    const df cf = (fwd ? (nu == 3 ? hc.f[3] : hc.f[0]) : (nu == 3 ? hc.b[3] : hc.b[0])) * ph;
    const float4* uv = reinterpret_cast<const float4*>(U) + (size_t)nu * 9 * V + (fwd ? i : nb);
    // spin rows one after the other: the projected row sp (three colours) and one link row at a
    // time (the link read twice, from L1 the second time): fewer live registers
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        cx<df> hs[3];
        const bool nn = sp == 0 ? n0 : n1;
        const int so = hi2 ? 2 + sp : 3 - sp;
#pragma unroll
        for (int a = 0; a < 3; ++a) hs[a] = add_lazy(ldx(3 * sp + a), unit_mul(ldx(3 * so + a), im, nn));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<df> u[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 v = __ldg(uv + (size_t)(fwd ? 3 * a + k : 3 * k + a) * V);
                u[k] = mk(df(v.x, v.y), df(v.z, v.w));
            }
            dfacc re, imv;
            if (fwd) {
                dfacc_first(re, u[0].r, hs[0].r, false);
                dfacc_add(re, u[0].i, hs[0].i, true);
                dfacc_first(imv, u[0].r, hs[0].i, false);
                dfacc_add(imv, u[0].i, hs[0].r, false);
#pragma unroll
                for (int k = 1; k < 3; ++k) {
                    dfacc_add(re, u[k].r, hs[k].r, false);
                    dfacc_add(re, u[k].i, hs[k].i, true);
                    dfacc_add(imv, u[k].r, hs[k].i, false);
                    dfacc_add(imv, u[k].i, hs[k].r, false);
                }
            } else {
                dfacc_first(re, u[0].r, hs[0].r, false);
                dfacc_add(re, u[0].i, hs[0].i, false);
                dfacc_first(imv, u[0].r, hs[0].i, false);
                dfacc_add(imv, u[0].i, hs[0].r, true);
#pragma unroll
                for (int k = 1; k < 3; ++k) {
                    dfacc_add(re, u[k].r, hs[k].r, false);
                    dfacc_add(re, u[k].i, hs[k].i, false);
                    dfacc_add(imv, u[k].r, hs[k].i, false);
                    dfacc_add(imv, u[k].i, hs[k].r, true);
                }
            }
            out[3 * sp + a] = cf * mk(dfacc_value(re), dfacc_value(imv));
        }
    }
}

template <class R, int LF, int MINB>
__global__ void __launch_bounds__(8 * TT, MINB) k_b_regen(const BSeq* __restrict__ S, const int* __restrict__ tseq, int i,
                                                    HopCoef<R> hc) {
    using VT = typename VecT<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R>(*dirpart)[TT][6] = reinterpret_cast<cx<R>(*)[TT][6]>(smraw);  // [8][TT][2 spins x 3 colours]
    __shared__ cx<R> cf[4];
    const BSeq& q = S[tseq[blockIdx.x]];  // set-up data, not written by the solve
    const KState* ks = q.ks;
    pdl_wait_and_release();
    if (ks->status || i + 1 >= ks->kused) return;
    if (threadIdx.x == 0) {
        const cx<double> ib = cdiv(mk(1.0, 0.0), d2c(q.beta[i]));
        cf[0] = cvt_coef<R>(ib);
        cf[1] = cvt_coef<R>(ib * d2c(q.alpha[i]));
        cf[2] = cvt_coef<R>(i > 0 ? ib * d2c(q.gamma[i - 1]) : mk(0.0, 0.0));
        cf[3] = cvt_coef<R>(d2c(q.cvec[i + 1]));
    }
    const int tile = blockIdx.x - q.tile0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const VT* ri = (const VT*)q.r[i % 3];
    const void* U = LF == LINK_DF ? q.Udf : (const void*)q.U64;
    {
        // warp wid: hop wid of the tile's 32 sites, kept as its half spinor
        const int i0 = tile * TT + lane;
        if (i0 < q.g.V) {
            if constexpr (LF == LINK_DF) {
                hop_half_rows_df(wid, q.g, q.nbr, i0, (const dfc*)U, (const dfc*)ri, hc, dirpart[wid][lane]);
            } else {
                const Coord c = site_coord(q.g, i0);
                const VT* const xs[1] = {ri};
                const HopCoef<R> hcs[1] = {hc};
                Half<R> hp[1];
                hop_half_uniform<LF, R, 1>(wid, q.g, c, i0, U, xs, hp, hcs);
#pragma unroll
                for (int c6 = 0; c6 < 6; ++c6) dirpart[wid][lane][c6] = hp[0].h[c6 / 3][c6 % 3];
            }
        }
    }
    __syncthreads();
    // epilogue: 256 threads (site, part), components part and part + 8 (< 12)
    const int site = threadIdx.x >> 3, part = threadIdx.x & 7;
    const int ii = tile * TT + site;
    if (ii >= q.g.V) return;
    const VT* rm = (const VT*)q.r[(i + 2) % 3];
    VT* rn = (VT*)q.r[(i + 1) % 3];
    VT* y = (VT*)q.y;
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
        const int c = part + 8 * c2;
        if (c >= 12) break;
        const cx<R> self = ld_comp_cg<R>(ri, q.g.V, ii, c);
        cx<R> z = self;
        const int sp = c / 3, a = c % 3;
#pragma unroll
        for (int w = 0; w < 8; ++w) z = add_lazy(z, hop_spin<R>(w, sp, dirpart[w][site][a], dirpart[w][site][3 + a]));
        if (c >= 6) z = -z;  // gamma5: spins 2, 3
        z = mk(cf[0].r * z.r, cf[0].r * z.i) - cf[1] * self;  // 1 / beta_i is real
        if (i > 0) z = z - cf[2] * ld_comp_cg<R>(rm, q.g.V, ii, c);
        st_comp<R>(rn, q.g.V, ii, c, z);
        st_comp<R>(y, q.g.V, ii, c, ld_comp_cg<R>(y, q.g.V, ii, c) + cf[3] * z);
    }
}

// The regeneration step for two sequences of the same lattice per block (work entry: the two
// sequences, the tile, whether the second one exists): each hop warp loads the link and computes
// the neighbour index once and runs the two sequences' double-float products as independent chains
// (twice the work in flight per warp); the epilogue spreads the 2 x 32 sites x 12 components over
// the 256 threads, three each.  Same arithmetic per sequence as k_b_regen.
template <class R, int LF, int MINB>
__global__ void __launch_bounds__(8 * TT, MINB) k_b_regen2(const BSeq* __restrict__ S, const int4* __restrict__ work,
                                                     int i, HopCoef<R> hc) {
    using VT = typename VecT<R>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R>(*dirpart)[8][TT][6] = reinterpret_cast<cx<R>(*)[8][TT][6]>(smraw);  // [2][8][TT][6]
    __shared__ cx<R> cf[2][4];
    const int4 wk = work[blockIdx.x];  // set-up data, not written by the solve
    const BSeq& qa = S[wk.x];
    const BSeq& qb = S[wk.y];
    const bool two = wk.w != 0;
    pdl_wait_and_release();
    const bool la = !(qa.ks->status || i + 1 >= qa.ks->kused);
    const bool lb = two && !(qb.ks->status || i + 1 >= qb.ks->kused);
    if (!la && !lb) return;
    if (threadIdx.x < 2 && (threadIdx.x == 0 || two)) {
        const BSeq& q = threadIdx.x ? qb : qa;
        const cx<double> ib = cdiv(mk(1.0, 0.0), d2c(q.beta[i]));
        cf[threadIdx.x][0] = cvt_coef<R>(ib);
        cf[threadIdx.x][1] = cvt_coef<R>(ib * d2c(q.alpha[i]));
        cf[threadIdx.x][2] = cvt_coef<R>(i > 0 ? ib * d2c(q.gamma[i - 1]) : mk(0.0, 0.0));
        cf[threadIdx.x][3] = cvt_coef<R>(d2c(q.cvec[i + 1]));
    }
    const int tile = wk.z;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Geom& g = qa.g;
    const VT* ra = (const VT*)qa.r[i % 3];
    const VT* rb = two ? (const VT*)qb.r[i % 3] : ra;
    const void* U = LF == LINK_DF ? qa.Udf : (const void*)qa.U64;
    {
        const int i0 = tile * TT + lane;
        if (i0 < g.V) {
            if constexpr (LF == LINK_DF) {
                hop_half_rows_df(wid, g, qa.nbr, i0, (const dfc*)U, (const dfc*)ra, hc, dirpart[0][wid][lane]);
                hop_half_rows_df(wid, g, qa.nbr, i0, (const dfc*)U, (const dfc*)rb, hc, dirpart[1][wid][lane]);
            } else {
                const Coord c = site_coord(g, i0);
                const VT* const xs[2] = {ra, rb};
                const HopCoef<R> hcs[2] = {hc, hc};
                Half<R> hp[2];
                hop_half_uniform<LF, R, 2>(wid, g, c, i0, U, xs, hp, hcs);
#pragma unroll
                for (int c6 = 0; c6 < 6; ++c6) {
                    dirpart[0][wid][lane][c6] = hp[0].h[c6 / 3][c6 % 3];
                    dirpart[1][wid][lane][c6] = hp[1].h[c6 / 3][c6 % 3];
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) {
        const int task = threadIdx.x + rr * 8 * TT;
        const int sq = task / (TT * 12), rem = task % (TT * 12);
        const int site = rem / 12, c = rem % 12;
        if (sq ? !lb : !la) continue;
        const BSeq& q = sq ? qb : qa;
        const int ii = tile * TT + site;
        if (ii >= g.V) continue;
        const VT* ri = sq ? rb : ra;
        const VT* rm = (const VT*)q.r[(i + 2) % 3];
        VT* rn = (VT*)q.r[(i + 1) % 3];
        VT* y = (VT*)q.y;
        const cx<R> self = ld_comp_cg<R>(ri, g.V, ii, c);
        cx<R> z = self;
        const int sp = c / 3, a = c % 3;
#pragma unroll
        for (int w = 0; w < 8; ++w)
            z = add_lazy(z, hop_spin<R>(w, sp, dirpart[sq][w][site][a], dirpart[sq][w][site][3 + a]));
        if (c >= 6) z = -z;  // gamma5: spins 2, 3
        z = mk(cf[sq][0].r * z.r, cf[sq][0].r * z.i) - cf[sq][1] * self;  // 1 / beta_i is real
        if (i > 0) z = z - cf[sq][2] * ld_comp_cg<R>(rm, g.V, ii, c);
        st_comp<R>(rn, g.V, ii, c, z);
        st_comp<R>(y, g.V, ii, c, ld_comp_cg<R>(y, g.V, ii, c) + cf[sq][3] * z);
    }
}

}  // namespace
}  // namespace ovl

// ------------------------------------------------------------------ host side --
struct ovl_batch {
    std::vector<ovl_ctx*> ctx;
    std::vector<int> nrhs;
    std::vector<int> seq_ctx;   // context of each sequence
    int nseq = 0;
    int kcap = 0;
    int mode = -1;              // 1 mixed, 0 FP64 one pass (basis stored), 2 FP64 two pass
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;
    // device memory
    void* mem = nullptr;
    size_t mem_bytes = 0;
    ovl::BSeq* dseq = nullptr;
    int* dbseq[ovl::NSHAPE] = {nullptr, nullptr, nullptr};
    int* dtseq = nullptr;
    int4* dpair = nullptr;         // regeneration work of two sequences per block: (a, b, tile, two)
    int npair_blocks = 0;
    unsigned int* pbar = nullptr;  // per-sequence barrier counters of the persistent pass 1
    int bp1_fit = -1;              // persistent pass 1 fits the GPU (-1: not yet determined)
    int nblocks[ovl::NSHAPE] = {0, 0, 0};
    int ntiles = 0;
    // autotuned launch shapes: pass-1 site-block shape, blocks per SM of the regeneration kernel
    int shape = 1;
    int regen_minb = 3;
    int regen_pair = 0;         // 1: two sequences of one lattice per regeneration block
    bool tuned = false;
    bool pinned = false;        // shapes set by ovl_batch_set_tuning: never retuned
    bool tune_cached = false;   // the shapes came from the tuning cache (no timing)
    int tuned_mode = -1;
    std::vector<ovl::BSeq> hseq;
    std::vector<double2*> b64, bR, bL, pq;
    ovl::KState* ks = nullptr;
    double2 *alpha = nullptr, *beta = nullptr, *gamma = nullptr, *cvec = nullptr, *vscale = nullptr;
    double2* inner = nullptr;
    size_t inner_stride = 0;
    double* qpart = nullptr;
    size_t qpart_stride = 0;
    unsigned int* qcnt = nullptr;
    double* part = nullptr;      // scratch of the per-sequence prologue kernels (pro_off[s] doubles in)
    std::vector<size_t> pro_off;
    std::vector<int> pro_m;      // deflation sizes the prologue scratch was laid out for
    unsigned int* counter = nullptr;
    // the sequences' prologues run on side streams (graph branches), joined before pass 1
    static constexpr int NSIDE = 4;
    cudaStream_t side[NSIDE] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[NSIDE] = {nullptr, nullptr, nullptr, nullptr};
    double2* stage = nullptr;    // host transfers
    // per-phase profile (OVL_PROFILE): pass 1, inner sign, pass 2 / combination
    double prof_ms[3] = {0.0, 0.0, 0.0};
    int prof_n = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // graph
    cudaGraphExec_t exec = nullptr;
    int g_k = -1, g_flags = 0;
    std::vector<int> g_m;  // deflation size of every context when the graph was captured
    double g_mu = 0, g_kappa = 0;
    std::string err;
};

namespace {

int bfail(ovl_batch* b, int code, const std::string& m) {
    if (b) b->err = m;
    return code;
}

void bfree(ovl_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    if (b->mem) cudaFree(b->mem);
    b->mem = nullptr;
    b->mem_bytes = 0;
    b->mode = -1;
}

// Carve the batch's device memory for mode (1 mixed, 0 FP64 one pass, 2 FP64 two pass) and Krylov size kmax.
int balloc(ovl_batch* b, int mode, int kmax) {
    if (b->mem && b->mode == mode && b->kcap >= kmax) return OVL_OK;
    bfree(b);
    const int ns = b->nseq;
    const size_t kk = (size_t)kmax + 2;
    const size_t inner_stride = std::max(ovl::inner_work_elems(kmax, 0), ovl::inner_work_elems(kmax, 1));
    const size_t qpart_stride = 8192;
    // byte sizes, every piece 256-aligned
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t total = 0;
    std::vector<size_t> seq_bytes(ns);
    int nblocks[ovl::NSHAPE] = {0, 0, 0}, ntiles = 0;
    for (int s = 0; s < ns; ++s) {
        const ovl_ctx* c = b->ctx[b->seq_ctx[s]];
        const size_t n = c->n;
        // partials: the most blocks of a pass-1 shape, or two sets for the persistent pass 1
        const int nblk = std::max((c->g.V + ovl::SHAPE_SITES[0] - 1) / ovl::SHAPE_SITES[0],
                                  2 * ((c->g.V + ovl::BP1_T - 1) / ovl::BP1_T));
        for (int h = 0; h < ovl::NSHAPE; ++h) nblocks[h] += (c->g.V + ovl::SHAPE_SITES[h] - 1) / ovl::SHAPE_SITES[h];
        ntiles += (c->g.V + ovl::TT - 1) / ovl::TT;
        size_t z = 0;
        z += 4 * al(n * sizeof(double2));                        // b, bR, bL, y
        z += 3 * al(n * sizeof(double2));                        // regeneration ring
        if (mode == 1) z += 8 * al(n * sizeof(float2));          // FP32 v, w rings, t, s
        else if (mode == 0) z += (kk + 5) * al(n * sizeof(double2));  // FP64 basis, w ring, t, s
        else z += 8 * al(n * sizeof(double2));                  // FP64 v, w rings, t, s
        z += al((size_t)nblk * 4 * sizeof(double2)) + al(128 * sizeof(double2));  // partials, pq
        seq_bytes[s] = z;
        total += z;
    }
    // prologue scratch per sequence: the two-stage projections' partials (m vectors x blocks,
    // complex) or the deflation split's grid sum (4 values x at most 512 blocks)
    // two sequences of one lattice per regeneration block (the sources of a context are consecutive)
    std::vector<int4> ptable;
    {
        int s0 = 0;
        for (size_t j = 0; j < b->ctx.size(); ++j) {
            const int nt = (b->ctx[j]->g.V + ovl::TT - 1) / ovl::TT;
            for (int r = 0; r < b->nrhs[j]; r += 2) {
                const int sa = s0 + r, two = r + 1 < b->nrhs[j];
                const int sb = two ? sa + 1 : sa;
                for (int t = 0; t < nt; ++t) ptable.push_back(make_int4(sa, sb, t, two));
            }
            s0 += b->nrhs[j];
        }
    }
    std::vector<size_t> pro_off(ns + 1, 0);
    std::vector<int> pro_m(ns, 0);
    for (int s = 0; s < ns; ++s) {
        const ovl_ctx* c = b->ctx[b->seq_ctx[s]];
        pro_m[s] = c->m;
        const size_t need = std::max<size_t>((size_t)2 * std::max(c->m, 1) * ovl::multidot_blocks(c->n), 2048);
        pro_off[s + 1] = pro_off[s] + ((need + 31) & ~(size_t)31);
    }
    total += al(ns * sizeof(ovl::KState)) + 5 * al(ns * kk * sizeof(double2)) +
             al((size_t)ns * inner_stride * sizeof(double2)) + al((size_t)ns * qpart_stride * sizeof(double)) +
             al(ns * 64 * sizeof(unsigned int)) + al(ns * sizeof(ovl::BSeq)) + al(nblocks[0] * sizeof(int)) +
             al(nblocks[1] * sizeof(int)) + al(nblocks[2] * sizeof(int)) +
             al(ntiles * sizeof(int)) + al(ns * sizeof(unsigned int)) + al(ptable.size() * sizeof(int4)) +
             al(pro_off[ns] * sizeof(double)) + al(64 * sizeof(unsigned int));
    if (cudaMalloc(&b->mem, total) != cudaSuccess) {
        b->mem = nullptr;
        return bfail(b, OVL_ENOMEM, "batch workspace");
    }
    b->mem_bytes = total;
    char* p = (char*)b->mem;
    auto take = [&](size_t bytes) { char* r = p; p += al(bytes); return (void*)r; };
    b->ks = (ovl::KState*)take(ns * sizeof(ovl::KState));
    b->alpha = (double2*)take(ns * kk * sizeof(double2));
    b->beta = (double2*)take(ns * kk * sizeof(double2));
    b->gamma = (double2*)take(ns * kk * sizeof(double2));
    b->cvec = (double2*)take(ns * kk * sizeof(double2));
    b->vscale = (double2*)take(ns * kk * sizeof(double2));
    b->inner = (double2*)take((size_t)ns * inner_stride * sizeof(double2));
    b->inner_stride = inner_stride;
    b->qpart = (double*)take((size_t)ns * qpart_stride * sizeof(double));
    b->qpart_stride = qpart_stride;
    b->qcnt = (unsigned int*)take(ns * 64 * sizeof(unsigned int));
    b->dseq = (ovl::BSeq*)take(ns * sizeof(ovl::BSeq));
    for (int h = 0; h < ovl::NSHAPE; ++h) b->dbseq[h] = (int*)take(nblocks[h] * sizeof(int));
    b->dtseq = (int*)take(ntiles * sizeof(int));
    b->pbar = (unsigned int*)take(ns * sizeof(unsigned int));
    b->dpair = (int4*)take(ptable.size() * sizeof(int4));
    b->npair_blocks = (int)ptable.size();
    b->part = (double*)take(pro_off[ns] * sizeof(double));
    b->pro_off = pro_off;
    b->pro_m = pro_m;
    b->counter = (unsigned int*)take(64 * sizeof(unsigned int));
    b->hseq.assign(ns, ovl::BSeq());
    b->b64.assign(ns, nullptr), b->bR.assign(ns, nullptr), b->bL.assign(ns, nullptr), b->pq.assign(ns, nullptr);
    std::vector<int> table[ovl::NSHAPE], ttable;
    ttable.reserve(ntiles);
    int blk0[ovl::NSHAPE] = {0, 0, 0}, tile0 = 0;
    for (int s = 0; s < ns; ++s) {
        ovl_ctx* c = b->ctx[b->seq_ctx[s]];
        const size_t n = c->n;
        ovl::BSeq& q = b->hseq[s];
        std::memset(&q, 0, sizeof(q));
        q.g = c->g;
        q.n = n;
        q.U = mode == 1 ? (const void*)c->U12 : (const void*)c->U64;
        q.U64 = c->U64;
        q.Udf = c->Udf;
        q.nbr = c->nbr;
        b->b64[s] = (double2*)take(n * sizeof(double2));
        b->bR[s] = (double2*)take(n * sizeof(double2));
        b->bL[s] = (double2*)take(n * sizeof(double2));
        q.y = (double2*)take(n * sizeof(double2));
        for (int j = 0; j < 3; ++j) q.r[j] = (double2*)take(n * sizeof(double2));
        if (mode == 1) {
            for (int j = 0; j < 3; ++j) q.v[j] = take(n * sizeof(float2)), q.w[j] = take(n * sizeof(float2));
            q.t = take(n * sizeof(float2));
            q.s = take(n * sizeof(float2));
            q.V = nullptr;
        } else if (mode == 0) {
            q.V = (double2*)take(kk * n * sizeof(double2));
            for (int j = 0; j < 3; ++j) q.w[j] = take(n * sizeof(double2)), q.v[j] = nullptr;
            q.t = take(n * sizeof(double2));
            q.s = take(n * sizeof(double2));
        } else {
            for (int j = 0; j < 3; ++j) q.v[j] = take(n * sizeof(double2)), q.w[j] = take(n * sizeof(double2));
            q.t = take(n * sizeof(double2));
            q.s = take(n * sizeof(double2));
            q.V = nullptr;
        }
        q.ks = b->ks + s;
        q.alpha = b->alpha + s * kk;
        q.beta = b->beta + s * kk;
        q.gamma = b->gamma + s * kk;
        q.cvec = b->cvec + s * kk;
        q.vscale = b->vscale + s * kk;
        for (int h = 0; h < ovl::NSHAPE; ++h) q.nblk[h] = (c->g.V + ovl::SHAPE_SITES[h] - 1) / ovl::SHAPE_SITES[h];
        q.part = (double2*)take((size_t)std::max(q.nblk[0], 2 * q.nblk[1]) * 4 * sizeof(double2));
        b->pq[s] = (double2*)take(128 * sizeof(double2));
        q.cnt = b->qcnt + s;  // the inner quadrature's counters follow at qcnt + nseq
        for (int h = 0; h < ovl::NSHAPE; ++h) {
            q.blk0[h] = blk0[h];
            for (int j = 0; j < q.nblk[h]; ++j) table[h].push_back(s);
            blk0[h] += q.nblk[h];
        }
        q.ntile = (c->g.V + ovl::TT - 1) / ovl::TT;
        q.tile0 = tile0;
        for (int j = 0; j < q.ntile; ++j) ttable.push_back(s);
        tile0 += q.ntile;
    }
    for (int h = 0; h < ovl::NSHAPE; ++h) b->nblocks[h] = blk0[h];
    b->ntiles = tile0;
    if (cudaMemcpy(b->dseq, b->hseq.data(), ns * sizeof(ovl::BSeq), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dbseq[0], table[0].data(), table[0].size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dbseq[1], table[1].data(), table[1].size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dbseq[2], table[2].data(), table[2].size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dtseq, ttable.data(), ttable.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dpair, ptable.data(), ptable.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->qcnt, 0, ns * 64 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(b->counter, 0, 64 * sizeof(unsigned int)) != cudaSuccess) {
        bfree(b);
        return bfail(b, OVL_ECUDA, "batch set-up copies");
    }
    b->mode = mode;
    b->kcap = kmax;
    return OVL_OK;
}

// Launch with programmatic stream serialisation (see pdl_wait_and_release).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

// The whole FP32 pass 1 as one cooperative launch when all of the batch's sites fit the GPU at once.
bool bp1_fits(ovl_batch* b) {
    if (b->bp1_fit < 0) {
        int per_sm = 0, nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ovl::k_bp1<ovl::LINK_F32_12>, ovl::BP1_T, 0);
        b->bp1_fit = (per_sm > 0 && b->nblocks[1] <= per_sm * nsm) ? 1 : 0;
    }
    return b->bp1_fit == 1;
}

int launch_bp1(ovl_batch* b, int k, double mu, double kappa, cudaStream_t st) {
    if (cudaMemsetAsync(b->pbar, 0, b->nseq * sizeof(unsigned int), st) != cudaSuccess) return OVL_ECUDA;
    ovl::BP1Args a;
    a.S = b->dseq;
    a.bseq = b->dbseq[1];
    a.bar = b->pbar;
    a.k = k;
    a.hv = ovl::make_coef<float>(mu, kappa);
    a.hw = ovl::make_coef<float>(-mu, kappa);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->nblocks[1]);
    cfg.blockDim = dim3(ovl::BP1_T);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ovl::k_bp1<ovl::LINK_F32_12>, a) == cudaSuccess ? OVL_OK : OVL_ECUDA;
}

// One pass-1 step of every sequence with site-block shape SH.
template <int SH>
void pass1_step(ovl_batch* b, int i, int k, double mu, double kappa, bool mixed, cudaStream_t st) {
    const int nb = b->nblocks[SH], T = ovl::SHAPE_SITES[SH];
    const ovl::BSeq* S = b->dseq;
    const int* tab = b->dbseq[SH];
    if (mixed) {
        launch_pdl(ovl::k_b_pair<ovl::LINK_F32_12, float, SH>, dim3(nb, 2), T, 0, st, S, tab, i, k - 1,
                   ovl::make_coef<float>(mu, kappa), ovl::make_coef<float>(-mu, kappa));
        if (i + 1 < k) launch_pdl(ovl::k_b_lstep<float, SH>, nb, T, 0, st, S, tab, i);
    } else {
        launch_pdl(ovl::k_b_pair<ovl::LINK_F64, double, SH>, dim3(nb, 2), T, 0, st, S, tab, i, k - 1,
                   ovl::make_coef<double>(mu, kappa), ovl::make_coef<double>(-mu, kappa));
        if (i + 1 < k) launch_pdl(ovl::k_b_lstep<double, SH>, nb, T, 0, st, S, tab, i);
    }
}

// One regeneration step of every sequence, blocks-per-SM bound MINB (one or two sequences per block).
template <int MINB>
void regen_step(ovl_batch* b, int i, double mu, double kappa, bool dfm, cudaStream_t st) {
    const size_t smr = (size_t)8 * ovl::TT * 6 * 16;
    static unsigned long long attr_dev = 0;
    if (ovl::first_use_on_device(attr_dev)) {
        cudaFuncSetAttribute(ovl::k_b_regen<ovl::df, ovl::LINK_DF, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smr);
        cudaFuncSetAttribute(ovl::k_b_regen<double, ovl::LINK_F64, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
        cudaFuncSetAttribute(ovl::k_b_regen2<ovl::df, ovl::LINK_DF, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smr));
        cudaFuncSetAttribute(ovl::k_b_regen2<double, ovl::LINK_F64, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smr));
    }
    const ovl::BSeq* S = b->dseq;
    if (b->regen_pair) {
        if (dfm)
            launch_pdl(ovl::k_b_regen2<ovl::df, ovl::LINK_DF, MINB>, b->npair_blocks, 8 * ovl::TT, 2 * smr, st, S,
                       (const int4*)b->dpair, i, ovl::make_coef<ovl::df>(mu, kappa));
        else
            launch_pdl(ovl::k_b_regen2<double, ovl::LINK_F64, MINB>, b->npair_blocks, 8 * ovl::TT, 2 * smr, st, S,
                       (const int4*)b->dpair, i, ovl::make_coef<double>(mu, kappa));
        return;
    }
    const int* tab = b->dtseq;
    if (dfm)
        launch_pdl(ovl::k_b_regen<ovl::df, ovl::LINK_DF, MINB>, b->ntiles, 8 * ovl::TT, smr, st, S, tab, i,
                   ovl::make_coef<ovl::df>(mu, kappa));
    else
        launch_pdl(ovl::k_b_regen<double, ovl::LINK_F64, MINB>, b->ntiles, 8 * ovl::TT, smr, st, S, tab, i,
                   ovl::make_coef<double>(mu, kappa));
}

// Everything between the packed sources and the unpacked results, on stream st.
int enqueue_batch(ovl_batch* b, int k, double mu, double kappa, int flags, cudaStream_t st) {
    if (k > b->kcap) return bfail(b, OVL_EINVAL, "k exceeds the batch workspace");
    const bool mixed = b->mode == 1;
    const bool twopass = b->mode != 0;
    const int ns = b->nseq;
    const bool prof = (flags & OVL_PROFILE) != 0;
    // prologue of every sequence (deflation split, start vectors): independent, so they run on
    // side streams forked from st and joined before pass 1 (parallel branches of the graph)
    const int nside = std::min(ns, ovl_batch::NSIDE);
    if (!b->ev_fork) {
        if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
            return bfail(b, OVL_ECUDA, "prologue events");
        for (int j = 0; j < ovl_batch::NSIDE; ++j)
            if (cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_join[j], cudaEventDisableTiming) != cudaSuccess)
                return bfail(b, OVL_ECUDA, "prologue streams");
    }
    cudaEventRecord(b->ev_fork, st);
    for (int j = 0; j < nside; ++j) cudaStreamWaitEvent(b->side[j], b->ev_fork, 0);
    for (int s = 0; s < ns; ++s) {
        cudaStream_t ss = b->side[s % nside];
        ovl_ctx* c = b->ctx[b->seq_ctx[s]];
        const ovl::BSeq& q = b->hseq[s];
        const size_t n = q.n;
        double* part = b->part + b->pro_off[s];
        unsigned int* cnt = b->qcnt + 2 * ns + s;  // zero between uses (the last block resets it)
        ovl::launch_state_init(q.ks, ss);
        const int m = c->m;
        if (m > 0) {
            ovl::launch_multidot(c->L, n, m, b->b64[s], b->pq[s], 0, part, n, ss);
            ovl::launch_multidot(c->R, n, m, b->b64[s], b->pq[s] + m, 0, part, n, ss);
        }
        ovl::launch_deflate_split(b->b64[s], c->R, c->L, c->lam, m, b->pq[s], b->bR[s], b->bL[s], q.y, q.ks,
                                  q.vscale, part, cnt, n, ss);
        if (mixed) {
            ovl::launch_native_f64_to_f32(b->bR[s], q.v[0], q.g, 1, ss);
            ovl::launch_native_f64_to_f32(b->bL[s], q.w[0], q.g, 1, ss);
        } else {
            cudaMemcpyAsync(q.V ? (void*)q.V : q.v[0], b->bR[s], n * sizeof(double2), cudaMemcpyDeviceToDevice, ss);
            cudaMemcpyAsync(q.w[0], b->bL[s], n * sizeof(double2), cudaMemcpyDeviceToDevice, ss);
        }
    }
    for (int j = 0; j < nside; ++j) {
        cudaEventRecord(b->ev_join[j], b->side[j]);
        cudaStreamWaitEvent(st, b->ev_join[j], 0);
    }
    // pass 1 (all sequences per launch): one persistent launch for mixed batches that fit the GPU
    if (prof) cudaEventRecord(b->ev[0], st);
    if (mixed && !(flags & OVL_STEPWISE) && bp1_fits(b)) {
        if (launch_bp1(b, k, mu, kappa, st)) return bfail(b, OVL_ECUDA, "persistent pass-1 launch");
    } else
    for (int i = 0; i < k; ++i) {
        switch (b->shape) {
            case 0: pass1_step<0>(b, i, k, mu, kappa, mixed, st); break;
            case 1: pass1_step<1>(b, i, k, mu, kappa, mixed, st); break;
            default: pass1_step<2>(b, i, k, mu, kappa, mixed, st); break;
        }
    }
    // inner sign of every sequence at once; Roberts' iteration where the quadrature did not settle
    if (prof) cudaEventRecord(b->ev[1], st);
    const size_t kk = (size_t)b->kcap + 2;
    if (ovl::launch_inner_quadrature_batched(ns, b->alpha, b->beta, b->gamma, b->ks, b->cvec, kk, b->inner,
                                             b->inner_stride, b->kcap, b->qpart, b->qpart_stride, b->qcnt + ns, st))
        return bfail(b, OVL_ECUDA, "batched inner sign launch");
    for (int s = 0; s < ns; ++s) {
        ovl_ctx* c = b->ctx[b->seq_ctx[s]];
        const ovl::BSeq& q = b->hseq[s];
        if (ovl::launch_inner_newton(q.alpha, q.beta, q.gamma, nullptr, 0, 1, q.ks, q.cvec,
                                     b->inner + (size_t)s * b->inner_stride, b->inner_stride, b->kcap, c->num_sms, st,
                                     1))
            return bfail(b, OVL_ECUDA, "inner sign fallback launch");
    }
    // combination
    if (prof) cudaEventRecord(b->ev[2], st);
    if (twopass) {
        // mixed: double-float regeneration unless OVL_PASS2_F64 (ring and y converted in place)
        const bool dfm = mixed && !(flags & OVL_PASS2_F64);
        for (int s = 0; s < ns; ++s) {
            const ovl::BSeq& q = b->hseq[s];
            ovl::launch_scale_start(b->bR[s], q.r[0], q.y, q.cvec, q.ks, q.n, st);
            if (dfm) {
                ovl::launch_f64_to_df(q.r[0], q.n, st);
                ovl::launch_f64_to_df(q.y, q.n, st);
            }
        }
        for (int i = 0; i + 1 < k; ++i) {
            switch (b->regen_minb) {
                case 2: regen_step<2>(b, i, mu, kappa, dfm, st); break;
                case 4: regen_step<4>(b, i, mu, kappa, dfm, st); break;
                case 5: regen_step<5>(b, i, mu, kappa, dfm, st); break;
                case 6: regen_step<6>(b, i, mu, kappa, dfm, st); break;
                default: regen_step<3>(b, i, mu, kappa, dfm, st); break;
            }
        }
        if (dfm)
            for (int s = 0; s < ns; ++s) ovl::launch_df_to_f64(b->hseq[s].y, b->hseq[s].n, st);
    } else {
        for (int s = 0; s < ns; ++s) {
            const ovl::BSeq& q = b->hseq[s];
            ovl::launch_combine(q.V, q.n, q.vscale, q.cvec, q.ks, b->kcap, q.y, q.n, st);
        }
    }
    if (prof) cudaEventRecord(b->ev[3], st);
    return cudaGetLastError() == cudaSuccess ? OVL_OK : bfail(b, OVL_ECUDA, "batch launch");
}

// Tuning cache: the chosen shapes per (GPU model, SM count, precision, lattice extents and
// right-hand sides of every context), kept for the process and, when the environment variable
// OVL_TUNE_CACHE names a file, in that file ("key shape minb pair" per line) across processes.
std::mutex g_tune_mu;
std::map<std::string, std::array<int, 3>> g_tune;

std::string tune_key(const ovl_batch* b) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr{};
    cudaGetDeviceProperties(&pr, dev);
    std::string k = std::string(pr.name) + "/" + std::to_string(pr.multiProcessorCount) + "/m" + std::to_string(b->mode);
    for (size_t j = 0; j < b->ctx.size(); ++j) {
        const ovl::Geom& g = b->ctx[j]->g;
        k += "/" + std::to_string(g.L[0]) + "x" + std::to_string(g.L[1]) + "x" + std::to_string(g.L[2]) + "x" +
             std::to_string(g.L[3]) + "r" + std::to_string(b->nrhs[j]);
    }
    for (char& ch : k)
        if (ch == ' ') ch = '_';
    return k;
}

bool tune_lookup(const std::string& key, std::array<int, 3>& out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) {
        const char* path = std::getenv("OVL_TUNE_CACHE");
        if (path && *path) {
            std::ifstream f(path);
            std::string kk;
            int a, m, q;
            while (f >> kk >> a >> m >> q) g_tune[kk] = {a, m, q};
        }
        it = g_tune.find(key);
        if (it == g_tune.end()) return false;
    }
    out = it->second;
    return out[0] >= 0 && out[0] < ovl::NSHAPE && out[1] >= 2 && out[1] <= 6 && (out[2] == 0 || out[2] == 1);
}

void tune_store(const std::string& key, const std::array<int, 3>& v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = v;
    const char* path = std::getenv("OVL_TUNE_CACHE");
    if (path && *path) {
        std::ofstream f(path, std::ios::app);
        f << key << " " << v[0] << " " << v[1] << " " << v[2] << "\n";
    }
}

// Autotuner of the batched kernels' launch shapes (site-block size of the pass-1 kernels, blocks
// per SM of the regeneration kernel): each candidate runs a short eager solve (TUNE_K steps) of the
// whole batch with events around its phases; the fastest pass-1 and regeneration candidates are
// kept for the batch.  The sources must already be packed.
int autotune(ovl_batch* b, double mu, double kappa, int flags, cudaStream_t st) {
    if (b->kcap < 8) return OVL_OK;  // too short to time; the defaults stay until a longer solve
    const int TUNE_K = std::min(24, b->kcap);  // the workspace holds kcap steps
    const int saved_shape = b->shape, saved_minb = b->regen_minb;
    for (cudaEvent_t& e : b->ev)
        if (!e && cudaEventCreate(&e) != cudaSuccess) return bfail(b, OVL_ECUDA, "tuning events");
    // candidates: pass-1 site-block shape, regeneration blocks per SM, sequences per regeneration block
    struct Cand {
        int shape, minb, pair;
    };
    const Cand cands[] = {{0, 3, 0}, {1, 4, 0}, {2, 5, 0}, {1, 6, 0}, {1, 2, 1}, {1, 3, 1}, {1, 4, 1}};
    const int ncand = (int)(sizeof(cands) / sizeof(cands[0]));
    float best1 = 1e30f, best2 = 1e30f;
    int bs = saved_shape, bm = saved_minb, bp = b->regen_pair;
    for (int rep = 0; rep < 2; ++rep)  // the first round warms caches and instruction memory
        for (int c = 0; c < ncand; ++c) {
            b->shape = cands[c].shape;
            b->regen_minb = cands[c].minb;
            b->regen_pair = cands[c].pair;
            const int r = enqueue_batch(b, TUNE_K, mu, kappa, (flags | OVL_PROFILE) & ~OVL_NO_GRAPH, st);
            if (r) return r;
            if (cudaStreamSynchronize(st) != cudaSuccess) return bfail(b, OVL_ECUDA, "tuning solve");
            float t1 = 0.f, t2 = 0.f;
            cudaEventElapsedTime(&t1, b->ev[0], b->ev[1]);
            cudaEventElapsedTime(&t2, b->ev[2], b->ev[3]);
            if (rep == 1) {
                if (t1 < best1) best1 = t1, bs = cands[c].shape;
                if (t2 < best2) best2 = t2, bm = cands[c].minb, bp = cands[c].pair;
            }
        }
    b->shape = bs;
    b->regen_minb = bm;
    b->regen_pair = bp;
    b->tuned = true;
    b->tuned_mode = b->mode;
    if (b->exec) cudaGraphExecDestroy(b->exec);  // a captured graph holds the old shapes
    b->exec = nullptr;
    return OVL_OK;
}

}  // namespace

extern "C" {

int ovl_batch_tuning(const ovl_batch* b, int* pass1_block_sites, int* regen_blocks_per_sm, int* regen_seqs_per_block) {
    if (!b) return OVL_EINVAL;
    if (pass1_block_sites) *pass1_block_sites = ovl::SHAPE_SITES[b->shape];
    if (regen_blocks_per_sm) *regen_blocks_per_sm = b->regen_minb;
    if (regen_seqs_per_block) *regen_seqs_per_block = b->regen_pair ? 2 : 1;
    return b->tuned ? OVL_OK : OVL_ESTATE;
}

int ovl_batch_set_tuning(ovl_batch* b, int pass1_block_sites, int regen_blocks_per_sm, int regen_seqs_per_block) {
    if (!b) return OVL_EINVAL;
    int sh = -1;
    for (int c = 0; c < ovl::NSHAPE; ++c)
        if (ovl::SHAPE_SITES[c] == pass1_block_sites) sh = c;
    if (sh < 0 || regen_blocks_per_sm < 2 || regen_blocks_per_sm > 6 || regen_seqs_per_block < 1 ||
        regen_seqs_per_block > 2)
        return bfail(b, OVL_EINVAL, "unsupported launch shape");
    b->shape = sh;
    b->regen_minb = regen_blocks_per_sm;
    b->regen_pair = regen_seqs_per_block == 2;
    b->tuned = b->pinned = true;
    if (b->exec) cudaGraphExecDestroy(b->exec);  // a captured graph holds the old shapes
    b->exec = nullptr;
    return OVL_OK;
}

int ovl_batch_create(ovl_batch** out, ovl_ctx* const* ctxs, int nctx, const int* nrhs) {
    if (!out || !ctxs || nctx < 1 || !nrhs) return OVL_EINVAL;
    *out = nullptr;
    ovl_batch* b = new ovl_batch();
    for (int j = 0; j < nctx; ++j) {
        if (!ctxs[j] || nrhs[j] < 0) {
            delete b;
            return OVL_EINVAL;
        }
        if (!ctxs[j]->have_gauge) {
            delete b;
            return OVL_ESTATE;
        }
        b->ctx.push_back(ctxs[j]);
        b->nrhs.push_back(nrhs[j]);
        for (int r = 0; r < nrhs[j]; ++r) b->seq_ctx.push_back(j);
    }
    b->nseq = (int)b->seq_ctx.size();
    if (b->nseq == 0) {
        delete b;
        return OVL_EINVAL;
    }
    b->st = ctxs[0]->st;
    *out = b;
    return OVL_OK;
}

int ovl_batch_destroy(ovl_batch* b) {
    if (!b) return OVL_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    else cudaDeviceSynchronize();
    bfree(b);
    if (b->cap_st) cudaStreamDestroy(b->cap_st);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    for (int j = 0; j < ovl_batch::NSIDE; ++j) {
        if (b->side[j]) cudaStreamDestroy(b->side[j]);
        if (b->ev_join[j]) cudaEventDestroy(b->ev_join[j]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
    return OVL_OK;
}

const char* ovl_batch_last_error(const ovl_batch* b) { return b ? b->err.c_str() : "null batch"; }

int ovl_batch_solve(ovl_batch* b, int k, double mu, double kappa, const void* const* bsrc, void* const* out,
                    int flags, ovl_info* info) {
    if (!b || !bsrc || !out || k < 1) return bfail(b, OVL_EINVAL, "bad argument");
    // FP64: the basis is stored when it fits a fixed budget, else the regeneration pass is used
    size_t ntot = 0;
    for (int q = 0; q < b->nseq; ++q) ntot += b->ctx[b->seq_ctx[q]]->n;
    const bool fits = ((size_t)k + 2) * ntot * sizeof(double2) <= ((size_t)32 << 30);
    const int mode = (flags & OVL_MIXED) ? 1 : ((flags & OVL_TWO_PASS) || !fits) ? 2 : 0;
    // a deflation set larger than the prologue scratch was laid out for: lay the workspace out again
    if (b->mem)
        for (int q = 0; q < b->nseq; ++q)
            if (b->ctx[b->seq_ctx[q]]->m > b->pro_m[q]) {
                bfree(b);
                break;
            }
    int r = balloc(b, mode, k);
    if (r) return r;
    for (ovl_ctx* c : b->ctx) {
        if (c->m > 0 && mode == 1 && !c->R32) return bfail(b, OVL_ESTATE, "deflation set not installed");
        if (c->st != b->st) return bfail(b, OVL_EINVAL, "all contexts of a batch must share one stream");
    }
    cudaStream_t st = b->st;
    const bool host = (flags & OVL_HOST) != 0;
    // pack the sources (canonical -> device layout); sources of context j follow one another
    int s = 0;
    for (size_t j = 0; j < b->ctx.size(); ++j) {
        ovl_ctx* c = b->ctx[j];
        const size_t n = c->n, vb = n * sizeof(double2);
        for (int rr = 0; rr < b->nrhs[j]; ++rr, ++s) {
            const double2* src = (const double2*)bsrc[j] + (size_t)rr * n;
            if (host) {
                r = ovl_priv::ensure_base(c);
                if (r) return bfail(b, r, c->err);
                if (cudaMemcpyAsync(c->stage_in, src, vb, cudaMemcpyHostToDevice, st) != cudaSuccess)
                    return bfail(b, OVL_ECUDA, "source copy");
                src = c->stage_in;
            }
            ovl::launch_pack_spinor(src, b->b64[s], 0, c->g, st);
        }
    }
    // launch shapes: timed once per batch on its own data (short eager solves), unless OVL_NO_TUNE
    if (!b->pinned && b->tuned_mode != mode && !(flags & OVL_NO_TUNE)) {
        const std::string key = tune_key(b);
        std::array<int, 3> v;
        if (tune_lookup(key, v)) {  // tuned before for this GPU, batch shape and precision
            b->shape = v[0], b->regen_minb = v[1], b->regen_pair = v[2];
            b->tuned = true;
            b->tuned_mode = b->mode;
            b->tune_cached = true;
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        } else {
            r = autotune(b, mu, kappa, flags, st);
            if (r) return r;
            b->tune_cached = false;
            tune_store(key, {b->shape, b->regen_minb, b->regen_pair});
        }
    }
    // the solve, as a graph captured once per (k, flags, mu, kappa); per-phase events need eager launches
    if (flags & OVL_PROFILE) {
        flags |= OVL_NO_GRAPH;
        for (cudaEvent_t& e : b->ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) return bfail(b, OVL_ECUDA, "profile events");
    }
    const int gflags = flags & (OVL_MIXED | OVL_NO_GRAPH | OVL_TWO_PASS | OVL_PASS2_F64 | OVL_STEPWISE);
    if (flags & OVL_NO_GRAPH) {
        r = enqueue_batch(b, k, mu, kappa, flags, st);
        if (r) return r;
    } else {
        std::vector<int> msig;
        for (const ovl_ctx* c : b->ctx) msig.push_back(c->m);
        if (!b->exec || b->g_k != k || b->g_flags != gflags || b->g_mu != mu || b->g_kappa != kappa ||
            b->g_m != msig) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            if (!b->cap_st && cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking) != cudaSuccess)
                return bfail(b, OVL_ECUDA, "capture stream");
            cudaGraph_t gr = nullptr;
            if (cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, OVL_ECUDA, "begin capture");
            r = enqueue_batch(b, k, mu, kappa, flags, b->cap_st);
            cudaError_t e = cudaStreamEndCapture(b->cap_st, &gr);
            if (r) {
                if (gr) cudaGraphDestroy(gr);
                return r;
            }
            if (e != cudaSuccess) return bfail(b, OVL_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->exec, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) {
                b->exec = nullptr;
                return bfail(b, OVL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            }
            b->g_k = k, b->g_flags = gflags, b->g_mu = mu, b->g_kappa = kappa;
            b->g_m = msig;
        }
        if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return bfail(b, OVL_ECUDA, "graph launch");
    }
    // unpack: out = y, or D_ov b = b + gamma5 y with OVL_OVERLAP
    s = 0;
    for (size_t j = 0; j < b->ctx.size(); ++j) {
        ovl_ctx* c = b->ctx[j];
        const size_t n = c->n, vb = n * sizeof(double2);
        for (int rr = 0; rr < b->nrhs[j]; ++rr, ++s) {
            const double2* src = (const double2*)bsrc[j] + (size_t)rr * n;
            double2* dst = (double2*)out[j] + (size_t)rr * n;
            const bool ov = (flags & OVL_OVERLAP) != 0;
            if (host) {
                if (ov && cudaMemcpyAsync(c->stage_in, src, vb, cudaMemcpyHostToDevice, st) != cudaSuccess)
                    return bfail(b, OVL_ECUDA, "source copy");
                ovl::launch_unpack_spinor(b->hseq[s].y, 0, c->stage_out, ov ? c->stage_in : nullptr, ov ? 1 : 0, c->g,
                                          st);
                if (cudaMemcpyAsync(dst, c->stage_out, vb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                    return bfail(b, OVL_ECUDA, "result copy");
            } else {
                ovl::launch_unpack_spinor(b->hseq[s].y, 0, dst, ov ? src : nullptr, ov ? 1 : 0, c->g, st);
            }
        }
    }
    std::vector<ovl::KState> ks(b->nseq);
    if (cudaMemcpyAsync(ks.data(), b->ks, b->nseq * sizeof(ovl::KState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return bfail(b, OVL_ECUDA, std::string("batch solve: ") + cudaGetErrorString(cudaGetLastError()));
    if (flags & OVL_PROFILE) {
        for (int j = 0; j < 3; ++j) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, b->ev[j], b->ev[j + 1]);
            b->prof_ms[j] += ms;
        }
        b->prof_n += 1;
    }
    int worst = OVL_OK;
    for (int q = 0; q < b->nseq; ++q) {
        if (info) {
            info[q].k_used = ks[q].kused;
            info[q].breakdown_step = ks[q].bdstep;
            info[q].inner_iters = ks[q].inner_iters;
            info[q].inner_method = ks[q].inner_method;
            info[q].bperp_norm = ks[q].nR;
            info[q].inner_err = ks[q].inner_err;
        }
        int code = OVL_OK;
        if (ks[q].timeout) code = OVL_ETIMEOUT;
        else if (ks[q].status) code = ks[q].status;
        else if (ks[q].bdstep >= 0) code = OVL_EBREAKDOWN;
        if (code && !worst) {
            worst = code;
            b->err = "sequence " + std::to_string(q) + " failed";
        }
    }
    return worst;
}

int ovl_batch_profile(ovl_batch* b, double* ms3, int* nsolves, int reset) {
    if (!b) return OVL_EINVAL;
    if (ms3)
        for (int j = 0; j < 3; ++j) ms3[j] = b->prof_ms[j];
    if (nsolves) *nsolves = b->prof_n;
    if (reset) {
        for (int j = 0; j < 3; ++j) b->prof_ms[j] = 0.0;
        b->prof_n = 0;
    }
    return OVL_OK;
}

int ovl_sign_krylov_batched(ovl_ctx* const* ctxs, int nctx, const int* nrhs, int k, double mu, double kappa,
                            const void* const* b, void* const* out, int flags, ovl_info* info) {
    ovl_batch* bt = nullptr;
    int r = ovl_batch_create(&bt, ctxs, nctx, nrhs);
    if (r) return r;
    r = ovl_batch_solve(bt, k, mu, kappa, b, out, flags | OVL_NO_GRAPH, info);
    if (r && ctxs[0]) ctxs[0]->err = bt->err;
    ovl_batch_destroy(bt);
    return r;
}

}  // extern "C"
