// Arnoldi (Sec. 2, Eq. 2.2-2.6; with LR deflation Sec. 3, Eq. 3.4) with the basis V_k stored as
// double-float pairs and the classical Gram-Schmidt (applied twice) evaluated in double-float
// arithmetic on the FP32 pipe.
//
// Step j of the Arnoldi relation A V_j = V_{j+1} H_j:  t = A v_j (FP64 stencil on the FP64 copy of
// v_j), h1 = V^dag t, t -= V h1, h2 = V^dag t, t -= V h2, H[0..j, j] = h1 + h2,
// H[j+1, j] = |t|, v_{j+1} = t / |t|.  The two passes over the stored basis per Gram-Schmidt sweep
// are the whole cost of the method at large k (Sec. 5); with FP64 arithmetic they run at the FP64
// issue rate, which on this GPU is far below what HBM delivers for 16 bytes per complex element.
// Double-float values (hi + lo, about 48 significant bits) take the same 16 bytes per complex
// element and their products and sums run on the FP32 pipe, so the sweeps become bandwidth
// bound.  The coefficients h, H and the inner sign stay FP64; every product enters its sum through
// the exact FMA split (dfacc), and every sum of per-lane, per-warp and per-block partials is
// deterministic (fixed order).
#include "ovl_kernels.h"
#include "df32.cuh"

namespace ovl {

static constexpr int AD_T = 256;    // threads per block
static constexpr int AD_W = AD_T / 32;
static constexpr int AD_CH = 1024;  // elements of x per block in the many-vector dot

__device__ __forceinline__ float4 to_f4(cx<df> z) { return make_float4(z.r.hi, z.r.lo, z.i.hi, z.i.lo); }
__device__ __forceinline__ cx<df> from_f4(float4 v) { return mk(df(v.x, v.y), df(v.z, v.w)); }

// sum over the 32 lanes of a warp (butterfly; every lane ends with the same value)
__device__ __forceinline__ df warp_sum_df(df a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const df b(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
        a = a + b;
    }
    return a;
}

// ------------------------------------------------------------------ helpers --
// xdf = x (FP64 -> double-float split), n complex values
__global__ void k_adf_todf(const double2* __restrict__ x, float4* __restrict__ xdf, const KState* ks, size_t n) {
    if (ks->done || ks->status) return;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        xdf[e] = to_f4(d2df(x[e]));
}

// v_1 = x / |x| (|x| = nR from the deflation split): the double-float split into V_0 and its
// exact FP64 value (hi + lo fits a double) into x64, the stencil's input of step 0
__global__ void k_adf_start(const double2* __restrict__ x, float4* __restrict__ v, double2* __restrict__ x64,
                            const KState* ks, size_t n) {
    if (ks->status || ks->nR == 0.0) return;
    const double s = 1.0 / ks->nR;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 a = x[e];
        const cx<df> z = d2df(make_double2(a.x * s, a.y * s));
        v[e] = to_f4(z);
        x64[e] = df2d(z);
    }
}

// ---------------------------------------------------------- many-vector dot --
// The update sweep streams the basis from HBM with one 16-byte load per lane and a chain of
// dependent double-float operations behind it, so a warp has about one load in flight; L2
// prefetches a fixed distance ahead (no registers held) keep more bytes in flight per SM.
static constexpr int AD_PFV = 4;   // update: vectors (of this warp) ahead
__device__ __forceinline__ void prefetch_l2(const float4* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// 16-byte asynchronous global -> shared copies (completion waited for per thread with
// cp.async.wait_group, a hardware wait)
__device__ __forceinline__ void cp_async16(float4* smem, const float4* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// re + i im += conj(v) x
__device__ __forceinline__ void adf_dot_term(dfacc& re, dfacc& im, const cx<df>& v, const cx<df>& xx) {
    dfacc_add(re, v.r, xx.r, false);
    dfacc_add(re, v.i, xx.i, false);
    dfacc_add(im, v.r, xx.i, false);
    dfacc_add(im, v.i, xx.r, true);
}
// re + i im += h v
__device__ __forceinline__ void adf_axpy_term(dfacc& re, dfacc& im, const cx<df>& h, const cx<df>& v) {
    dfacc_add(re, h.r, v.r, false);
    dfacc_add(re, h.i, v.i, true);
    dfacc_add(im, h.r, v.i, false);
    dfacc_add(im, h.i, v.r, false);
}

// stage 1, grid (chunks, vector groups): block (c, g) stages elements [c*AD_CH, (c+1)*AD_CH) of
// x in shared memory; warp w forms the partial dots V_l^dag x over that chunk for
// l = g*vpb + w, g*vpb + w + AD_W, ... < min(nvec, (g+1)*vpb).  The warp streams its
// (vector, tile of AD_SUB elements) pieces through two shared-memory tiles: the copy of the next
// tile is in flight while the current one is summed, so every warp keeps 4 KB of the basis in
// flight instead of one 16-byte load per lane.
static constexpr int AD_SUB = 256;
static size_t adf_dot_smem() { return sizeof(float4) * ((size_t)AD_CH + (size_t)AD_W * 2 * AD_SUB); }

__global__ void __launch_bounds__(AD_T) k_adf_dot(const float4* __restrict__ V, size_t ld, int nvec, int vpb,
                                                  const float4* __restrict__ x, double2* __restrict__ part,
                                                  size_t n, const KState* ks) {
    extern __shared__ float4 adf_sm[];
    float4* xs = adf_sm;
    if (ks->done || ks->status) return;
    const size_t base = (size_t)blockIdx.x * AD_CH;
    const int lim = (int)(n - base < (size_t)AD_CH ? n - base : (size_t)AD_CH);
    for (int q = threadIdx.x; q < lim; q += AD_T) xs[q] = x[base + q];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* wb = adf_sm + AD_CH + (size_t)wid * 2 * AD_SUB;
    const int l0 = blockIdx.y * vpb + wid;
    const int l1 = min(nvec, blockIdx.y * vpb + vpb);
    const int nv = l0 < l1 ? (l1 - l0 + AD_W - 1) / AD_W : 0;
    const int ntile = (lim + AD_SUB - 1) / AD_SUB;
    const int total = nv * ntile;
    // each lane copies (and later reads) the elements lane, lane + 32, ... of a tile
    auto issue = [&](int it) {
        const int a = it / ntile, si = it - a * ntile;
        const float4* src = V + (size_t)(l0 + a * AD_W) * ld + base + (size_t)si * AD_SUB;
        float4* dst = wb + (it & 1) * AD_SUB;
        const int cnt = min(AD_SUB, lim - si * AD_SUB);
        for (int u = lane; u < cnt; u += 32) cp_async16(dst + u, src + u);
        cp_async_commit();
    };
    if (total > 0) issue(0);
    dfacc re = {0.f, 0.f}, im = {0.f, 0.f};
    for (int it = 0; it < total; ++it) {
        if (it + 1 < total) {
            issue(it + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const int a = it / ntile, si = it - a * ntile;
        const float4* cur = wb + (it & 1) * AD_SUB;
        const float4* xt = xs + si * AD_SUB;
        const int cnt = min(AD_SUB, lim - si * AD_SUB);
        if (si == 0) {
            re = {0.f, 0.f};
            im = {0.f, 0.f};
        }
#pragma unroll 4
        for (int u = lane; u < cnt; u += 32) adf_dot_term(re, im, from_f4(cur[u]), from_f4(xt[u]));
        if (si == ntile - 1) {
            const df sr = warp_sum_df(dfacc_value(re)), si2 = warp_sum_df(dfacc_value(im));
            if (lane == 0)
                part[(size_t)(l0 + a * AD_W) * gridDim.x + blockIdx.x] = make_double2(sr.to_double(), si2.to_double());
        }
        __syncwarp();  // this tile's buffer receives the copy issued two iterations on
    }
}

// stage 2: one warp per vector sums its block partials in FP64 (fixed order); h in FP64 and as a
// double-float split for the update kernels
__global__ void k_adf_dot_reduce(const double2* __restrict__ part, int nblk, int nvec, double2* __restrict__ h,
                                 float4* __restrict__ hdf, const KState* ks) {
    if (ks->done || ks->status) return;
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= nvec) return;
    double re = 0.0, im = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = part[(size_t)l * nblk + b];
        re += v.x;
        im += v.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) {
        h[l] = make_double2(re, im);
        hdf[l] = to_f4(d2df(make_double2(re, im)));
    }
}

// ------------------------------------------------------- many-vector update --
// Block = 32 consecutive elements (lane) x AD_W warps; warp w sums c_l V_l[e] over l = w, w + AD_W,
// ... < nvec, the warps' sums are added in shared memory in warp order.
__device__ __forceinline__ void adf_lincomb(const float4* __restrict__ V, size_t ld, int nvec,
                                            const float4* __restrict__ c, size_t e, bool in, int wid, int lane,
                                            float4 (&red)[AD_W][32], cx<df>& sum) {
    dfacc re = {0.f, 0.f}, im = {0.f, 0.f};
    if (in) {
#pragma unroll 4
        for (int l = wid; l < nvec; l += AD_W) {
            if ((lane & 7) == 0 && l + AD_PFV * AD_W < nvec)  // one lane per 128-byte line
                prefetch_l2(V + (size_t)(l + AD_PFV * AD_W) * ld + e);
            adf_axpy_term(re, im, from_f4(__ldg(c + l)), from_f4(__ldg(V + (size_t)l * ld + e)));
        }
    }
    red[wid][lane] = make_float4(re.s, re.e, im.s, im.e);
    __syncthreads();
    if (wid == 0) {
        df sr = df_fast2sum(red[0][lane].x, red[0][lane].y), si = df_fast2sum(red[0][lane].z, red[0][lane].w);
#pragma unroll
        for (int w = 1; w < AD_W; ++w) {
            const float4 p = red[w][lane];
            sr = sr + df_fast2sum(p.x, p.y);
            si = si + df_fast2sum(p.z, p.w);
        }
        sum = mk(sr, si);
    }
}

struct ArnoldiFinDf {
    double2* H;
    int ldH;
    const double2* h1;
    const double2* h2;
    int j;
    int jlast;
    double bdtol;  // lucky breakdown when H[j+1, j] <= bdtol * (largest column norm of H so far)
};

// x -= sum_l h_l V_l (x double-float, in place).  fin = 1 (second pass of step j): also |x|^2 over
// the grid, and the last block writes H[0..j, j] = h1 + h2, H[j+1, j] = |x|, kused = j + 1 and
// marks the solve done on a lucky breakdown or at j = jlast.
__global__ void __launch_bounds__(AD_T) k_adf_update(const float4* __restrict__ V, size_t ld, int nvec,
                                                     const float4* __restrict__ hdf, float4* __restrict__ x,
                                                     size_t n, KState* ks, int fin, ArnoldiFinDf af,
                                                     double* partials, unsigned int* counter) {
    __shared__ float4 red[AD_W][32];
    __shared__ double rsm[32];
    if (ks->done || ks->status) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t ntile = (n + 31) / 32;
    double part[1] = {0.0};
    for (size_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const size_t e = tile * 32 + lane;
        const bool in = e < n;
        cx<df> s;
        adf_lincomb(V, ld, nvec, hdf, e, in, wid, lane, red, s);
        if (wid == 0 && in) {
            const cx<df> xv = from_f4(x[e]);
            const cx<df> z = mk(xv.r - s.r, xv.i - s.i);
            x[e] = to_f4(z);
            const double2 zd = df2d(z);
            part[0] += zd.x * zd.x + zd.y * zd.y;
        }
        __syncthreads();  // red is reused by the next tile
    }
    if (!fin) return;
    double out[1];
    if (grid_sum_last<1>(part, partials, counter, out, rsm)) {
        const int j = af.j;
        double hh = 0.0;
        for (int r = threadIdx.x; r <= j; r += blockDim.x) {
            const double2 a = af.h1[r], b = af.h2[r];
            const double2 v = make_double2(a.x + b.x, a.y + b.y);
            af.H[r + (size_t)j * af.ldH] = v;
            hh += v.x * v.x + v.y * v.y;
        }
        double hv[1] = {hh};
        block_sum<1>(hv, rsm);
        if (threadIdx.x == 0) {
            const double hn = sqrt(out[0]);
            af.H[(j + 1) + (size_t)j * af.ldH] = make_double2(hn, 0.0);
            const double colnorm = sqrt(hv[0] + out[0]);
            if (colnorm > ks->anorm) ks->anorm = colnorm;
            ks->kused = j + 1;
            ks->red[0] = make_double2(hn, 0.0);
            if (hn <= af.bdtol * fmax(ks->anorm, 1e-300) || j == af.jlast) ks->done = 1;
        }
    }
}

// v_{j+1} = t / |t| in place (double-float), and its exact FP64 value into x64 (the next step's
// stencil input); skipped after the last step or a lucky breakdown
__global__ void k_adf_normalize(float4* __restrict__ t, double2* __restrict__ x64, const KState* ks, size_t n) {
    if (ks->done || ks->status) return;
    const df inv(1.0 / ks->red[0].x);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const cx<df> z = from_f4(t[e]);
        const cx<df> v = mk(z.r * inv, z.i * inv);
        t[e] = to_f4(v);
        x64[e] = df2d(v);
    }
}

// c_l as double-float splits for l < kused
__global__ void k_adf_coef(const double2* __restrict__ c, float4* __restrict__ cdf, const KState* ks) {
    if (ks->status) return;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ks->kused; l += gridDim.x * blockDim.x)
        cdf[l] = to_f4(d2df(c[l]));
}

// y += sum_{l < kused} c_l V_l (Eq. 2.6), y FP64
__global__ void __launch_bounds__(AD_T) k_adf_combine(const float4* __restrict__ V, size_t ld,
                                                      const float4* __restrict__ cdf, const KState* ks,
                                                      double2* __restrict__ y, size_t n) {
    __shared__ float4 red[AD_W][32];
    if (ks->status) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t e = (size_t)blockIdx.x * 32 + lane;
    const bool in = e < n;
    cx<df> s;
    adf_lincomb(V, ld, ks->kused, cdf, e, in, wid, lane, red, s);
    if (wid == 0 && in) {
        const double2 a = y[e], d = df2d(s);
        y[e] = make_double2(a.x + d.x, a.y + d.y);
    }
}

// ================================================== low-synch Arnoldi: delayed CGS2 ==
// Classical Gram-Schmidt applied twice with the second pass delayed by one step (the "DCGS2" of the
// low-synchronisation Gram-Schmidt literature: Swirydowicz, Langou, Ananthan, Yang and Thomas,
// Numer. Linear Algebra Appl. 28 (2021); Bielich, Langou, Thomas, Swirydowicz, Yamazaki and Boman,
// Parallel Comput. 112 (2022)), on the double-float basis.  At step j the slots V_0..V_{j-1} hold
// final orthonormal vectors and slot j holds u_j, A v_{j-1} projected once and neither
// re-orthogonalised nor normalised; the stencil has produced w = A u_j (FP64) from its FP64 value.
//  (1) one sweep over V_0..V_j:  c = V_{<j}^dag u_j, rho^2 = u_j^dag u_j, d = V_{<j}^dag w,
//      e = u_j^dag w                                           (k_adf_dot2, k_adf_dot2_reduce)
//  (2) nu^2 = rho^2 - |c|^2 (V_{<j} orthonormal); column j-1 of H becomes final,
//      H[<j, j-1] += c, H[j, j-1] = nu; v_j = (u_j - V_{<j} c) / nu             (k_adf_dcgs)
//  (3) one sweep over V_0..V_{j-1}:  v_j, and u_{j+1} = A v_j - V_{<=j} h = w / nu - V_{<j} d / nu
//      - r v_j with r = (e - c^dag d) / nu^2; the tentative column j of H is
//      h = (d / nu - g, r - c_{j-1}), g = H[<=j, <j] c / nu                      (k_adf_update2)
// because A v_j = (w - A V_{<j} c) / nu = (w - V_{<=j} H[<=j, <j] c) / nu by the Arnoldi relation
// of the final columns: the projection coefficients of A v_j come from the sums of (1) without
// another pass, and the basis is read twice per step instead of four times.  After the last step
// one more dot sweep re-orthogonalises u_k and finishes column k-1.  In exact arithmetic this is
// the Arnoldi process of Sec. 2 (Eq. 2.2-2.3).

static size_t adf_dot2_smem() { return sizeof(float4) * (2 * (size_t)AD_CH + (size_t)AD_W * 2 * AD_SUB); }

// stage 1 of the two-vector dot, grid (chunks, vector groups): V_l^dag x1 and V_l^dag x2 for every
// l < nvec over the block's chunk; x1 is a double-float vector, x2 an FP64 one (split on staging).
// Partials: part[(2 l + q) * gridDim.x + chunk], q = 0 for x1, 1 for x2.
__global__ void __launch_bounds__(AD_T) k_adf_dot2(const float4* __restrict__ V, size_t ld, int nvec, int vpb,
                                                   const float4* __restrict__ x1, const double2* __restrict__ x2,
                                                   double2* __restrict__ part, size_t n, const KState* ks) {
    extern __shared__ float4 adf_sm[];
    float4* xs1 = adf_sm;
    float4* xs2 = adf_sm + AD_CH;
    if (ks->done || ks->status) return;
    const size_t base = (size_t)blockIdx.x * AD_CH;
    const int lim = (int)(n - base < (size_t)AD_CH ? n - base : (size_t)AD_CH);
    for (int q = threadIdx.x; q < lim; q += AD_T) {
        xs1[q] = x1[base + q];
        xs2[q] = to_f4(d2df(x2[base + q]));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* wb = adf_sm + 2 * AD_CH + (size_t)wid * 2 * AD_SUB;
    const int l0 = blockIdx.y * vpb + wid;
    const int l1 = min(nvec, blockIdx.y * vpb + vpb);
    const int nv = l0 < l1 ? (l1 - l0 + AD_W - 1) / AD_W : 0;
    const int ntile = (lim + AD_SUB - 1) / AD_SUB;
    const int total = nv * ntile;
    auto issue = [&](int it) {
        const int a = it / ntile, si = it - a * ntile;
        const float4* src = V + (size_t)(l0 + a * AD_W) * ld + base + (size_t)si * AD_SUB;
        float4* dst = wb + (it & 1) * AD_SUB;
        const int cnt = min(AD_SUB, lim - si * AD_SUB);
        for (int u = lane; u < cnt; u += 32) cp_async16(dst + u, src + u);
        cp_async_commit();
    };
    if (total > 0) issue(0);
    dfacc re1 = {0.f, 0.f}, im1 = {0.f, 0.f}, re2 = {0.f, 0.f}, im2 = {0.f, 0.f};
    for (int it = 0; it < total; ++it) {
        if (it + 1 < total) {
            issue(it + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const int a = it / ntile, si = it - a * ntile;
        const float4* cur = wb + (it & 1) * AD_SUB;
        const int cnt = min(AD_SUB, lim - si * AD_SUB);
        if (si == 0) re1 = im1 = re2 = im2 = {0.f, 0.f};
#pragma unroll 4
        for (int u = lane; u < cnt; u += 32) {
            const cx<df> v = from_f4(cur[u]);
            adf_dot_term(re1, im1, v, from_f4(xs1[si * AD_SUB + u]));
            adf_dot_term(re2, im2, v, from_f4(xs2[si * AD_SUB + u]));
        }
        if (si == ntile - 1) {
            const df s1r = warp_sum_df(dfacc_value(re1)), s1i = warp_sum_df(dfacc_value(im1));
            const df s2r = warp_sum_df(dfacc_value(re2)), s2i = warp_sum_df(dfacc_value(im2));
            if (lane == 0) {
                const size_t l = (size_t)(l0 + a * AD_W);
                part[(2 * l) * gridDim.x + blockIdx.x] = make_double2(s1r.to_double(), s1i.to_double());
                part[(2 * l + 1) * gridDim.x + blockIdx.x] = make_double2(s2r.to_double(), s2i.to_double());
            }
        }
        __syncwarp();  // this tile's buffer receives the copy issued two iterations on
    }
}

// stage 2: one warp per (vector, operand) sums its chunk partials in FP64 (fixed order):
// h1[l] = V_l^dag x1, h2[l] = V_l^dag x2
__global__ void k_adf_dot2_reduce(const double2* __restrict__ part, int nblk, int nvec, double2* __restrict__ h1,
                                  double2* __restrict__ h2, const KState* ks) {
    if (ks->done || ks->status) return;
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= 2 * nvec) return;
    double re = 0.0, im = 0.0;
    for (int b = lane; b < nblk; b += 32) {
        const double2 v = part[(size_t)p * nblk + b];
        re += v.x;
        im += v.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) ((p & 1) ? h2 : h1)[p >> 1] = make_double2(re, im);
}

// (2): one block.  h1 = (c, rho^2) and h2 = (d, e) of step j (h2 unused when fin).  Finishes
// column j-1 of H (j >= 1), decides a lucky breakdown (nu <= bdtol |H|), and for the update writes
// cdf = c, qdf = d / nu (double-float), ks->red[1] = (1 / nu, nu), ks->red[2] = r.  fin = 1 after
// the last step (j = k): only column k-1 is finished and the solve is marked done.  fin = 2 at the
// end of a restart cycle: column k-1 is finished, cdf = c and ks->red[1] are written for the next
// cycle's start vector (u_k - V c) / nu, and the solve goes on unless the Krylov space is invariant.
__global__ void __launch_bounds__(1024) k_adf_dcgs(double2* __restrict__ H, int ldH, const double2* __restrict__ h1,
                                                   const double2* __restrict__ h2, float4* __restrict__ cdf,
                                                   float4* __restrict__ qdf, KState* ks, int j, int fin,
                                                   double bdtol) {
    __shared__ double red[4 * 32];  // block_sum<4>: 32 doubles per value
    __shared__ double s_nu;
    __shared__ int s_stop;
    if (ks->done || ks->status) return;
    // |c|^2, c^dag d, |H[<j, j-1] + c|^2
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = threadIdx.x; l < j; l += blockDim.x) {
        const double2 c = h1[l];
        acc[0] += c.x * c.x + c.y * c.y;
        if (!fin) {
            const double2 d = h2[l];
            acc[1] += c.x * d.x + c.y * d.y;
            acc[2] += c.x * d.y - c.y * d.x;
        }
        const double2 hv = H[l + (size_t)(j - 1) * ldH];
        const double hr = hv.x + c.x, hi = hv.y + c.y;
        acc[3] += hr * hr + hi * hi;
    }
    block_sum<4>(acc, red);
    if (threadIdx.x == 0) {
        const double rho2 = h1[j].x;
        const double nu2 = rho2 - acc[0];
        const double nu = nu2 > 0.0 ? sqrt(nu2) : 0.0;
        int stop = 0;
        if (j >= 1) {
            H[j + (size_t)(j - 1) * ldH] = make_double2(nu, 0.0);
            const double colnorm = sqrt(acc[3] + nu * nu);
            if (colnorm > ks->anorm) ks->anorm = colnorm;
            ks->kused = j;
            if (fin == 1 || nu <= bdtol * fmax(ks->anorm, 1e-300)) stop = 1;  // last column, or K_j invariant
        } else if (!(nu > 0.0)) {
            stop = 1;  // zero start vector (cannot happen after the deflation split's check)
        }
        if (stop) {
            ks->done = 1;
        } else {
            const double inu = 1.0 / nu;
            ks->red[1] = make_double2(inu, nu);
            if (!fin) {  // r = (e - c^dag d) / nu^2
                const double2 e = h2[j];
                ks->red[2] = make_double2((e.x - acc[1]) * inu * inu, (e.y - acc[2]) * inu * inu);
            }
        }
        s_nu = nu;
        s_stop = stop;
    }
    __syncthreads();
    const double inu = s_stop ? 0.0 : 1.0 / s_nu;
    for (int l = threadIdx.x; l < j; l += blockDim.x) {
        const double2 c = h1[l];
        const double2 hv = H[l + (size_t)(j - 1) * ldH];
        H[l + (size_t)(j - 1) * ldH] = make_double2(hv.x + c.x, hv.y + c.y);
        if (!s_stop) {
            cdf[l] = to_f4(d2df(c));
            if (!fin) {
                const double2 d = h2[l];
                qdf[l] = to_f4(d2df(make_double2(d.x * inu, d.y * inu)));
            }
        }
    }
}

// (3): per element e, over the final vectors V_0..V_{j-1}: s1 = sum_l c_l V_l[e], s2 = sum_l
// (d_l / nu) V_l[e]; then v_j = (u_j - s1) / nu into slot j (in place of u_j) and u_{j+1} =
// w / nu - s2 - r v_j into slot j + 1 and, as FP64, into x64 (the next stencil's input).  Blocks
// 0..j also write the tentative column j of H: H[i, j] = d_i / nu - g_i (i < j), r - c_{j-1}
// (i = j), g_i = sum_{l >= i-1} H[i, l] c_l / nu (upper Hessenberg rows of the final columns).
__global__ void __launch_bounds__(AD_T) k_adf_update2(const float4* __restrict__ V, size_t ld, int j,
                                                      const float4* __restrict__ cdf, const float4* __restrict__ qdf,
                                                      float4* __restrict__ uj, float4* __restrict__ unext,
                                                      const double2* __restrict__ w, double2* __restrict__ x64,
                                                      double2* __restrict__ H, int ldH, const double2* __restrict__ h1,
                                                      const double2* __restrict__ h2, size_t n, KState* ks) {
    __shared__ float4 red1[AD_W][32];
    __shared__ float4 red2[AD_W][32];
    if (ks->done || ks->status) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double2 sc = ks->red[1];
    const double inu = sc.x;
    const double2 r = ks->red[2];
    if ((int)blockIdx.x <= j && wid == 0) {
        const int i = blockIdx.x;
        double gr = 0.0, gi = 0.0;
        for (int l = max(i - 1, 0) + lane; l < j; l += 32) {
            const double2 hv = H[i + (size_t)l * ldH], c = h1[l];
            gr += hv.x * c.x - hv.y * c.y;
            gi += hv.x * c.y + hv.y * c.x;
        }
        gr = warp_sum(gr) * inu;
        gi = warp_sum(gi) * inu;
        if (lane == 0) {
            double2 hv;
            if (i < j) {
                const double2 d = h2[i];
                hv = make_double2(d.x * inu - gr, d.y * inu - gi);
            } else {
                const double2 cl = j > 0 ? h1[j - 1] : make_double2(0.0, 0.0);
                hv = make_double2(r.x - cl.x, r.y - cl.y);
            }
            H[i + (size_t)j * ldH] = hv;
        }
    }
    const df dinu(inu);
    const cx<df> rr = d2df(r);
    const size_t ntile = (n + 31) / 32;
    for (size_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const size_t e = tile * 32 + lane;
        const bool in = e < n;
        dfacc a1r = {0.f, 0.f}, a1i = {0.f, 0.f}, a2r = {0.f, 0.f}, a2i = {0.f, 0.f};
        if (in) {
#pragma unroll 4
            for (int l = wid; l < j; l += AD_W) {
                if ((lane & 7) == 0 && l + AD_PFV * AD_W < j)  // one lane per 128-byte line
                    prefetch_l2(V + (size_t)(l + AD_PFV * AD_W) * ld + e);
                const cx<df> v = from_f4(__ldg(V + (size_t)l * ld + e));
                adf_axpy_term(a1r, a1i, from_f4(__ldg(cdf + l)), v);
                adf_axpy_term(a2r, a2i, from_f4(__ldg(qdf + l)), v);
            }
        }
        red1[wid][lane] = make_float4(a1r.s, a1r.e, a1i.s, a1i.e);
        red2[wid][lane] = make_float4(a2r.s, a2r.e, a2i.s, a2i.e);
        __syncthreads();
        if (wid == 0 && in) {
            df s1r = df_fast2sum(red1[0][lane].x, red1[0][lane].y), s1i = df_fast2sum(red1[0][lane].z, red1[0][lane].w);
            df s2r = df_fast2sum(red2[0][lane].x, red2[0][lane].y), s2i = df_fast2sum(red2[0][lane].z, red2[0][lane].w);
#pragma unroll
            for (int q = 1; q < AD_W; ++q) {
                const float4 p1 = red1[q][lane], p2 = red2[q][lane];
                s1r = s1r + df_fast2sum(p1.x, p1.y);
                s1i = s1i + df_fast2sum(p1.z, p1.w);
                s2r = s2r + df_fast2sum(p2.x, p2.y);
                s2i = s2i + df_fast2sum(p2.z, p2.w);
            }
            const cx<df> u = from_f4(uj[e]);
            const cx<df> vj = mk((u.r - s1r) * dinu, (u.i - s1i) * dinu);
            const cx<df> ww = d2df(w[e]);
            const cx<df> rv = rr * vj;
            const cx<df> un = mk(ww.r * dinu - s2r - rv.r, ww.i * dinu - s2i - rv.i);
            uj[e] = to_f4(vj);
            unext[e] = to_f4(un);
            x64[e] = df2d(un);
        }
        __syncthreads();  // red1, red2 are reused by the next tile
    }
}

// ======================================================== restarted Arnoldi ==
// Arnoldi restarted every m steps (Eiermann and Ernst, SIAM J. Numer. Anal. 44 (2006)): cycle c
// runs m delayed-CGS2 steps on the double-float basis slots 0..m from the start vector in slot 0,
// writing its Hessenberg block into the accumulated matrix at rows and columns c m ..; the block's
// subdiagonal entry H[m, m-1] is the coupling to the next cycle.  After the cycle the inner sign of
// the accumulated K x K matrix gives c_K = |b_perp| sgn(H_K) e_1, of which the rows of cycle c
// multiply its basis: y += V_c c_K[c m ..].  The next cycle starts from v_m = (u_m - V c) / nu.
// Cycle bookkeeping in the state record: red[4].x = K (columns finished so far), red[5] = (steps of
// this cycle, stopped); a lucky breakdown stops the process after that cycle's combination.
__global__ void k_rs_begin(KState* ks, int cyc) {
    if (ks->status) return;
    if (cyc == 0) {  // a source the deflation split left empty (done already) stops the process
        ks->red[4] = make_double2(0.0, 0.0);
        ks->red[5] = make_double2(0.0, ks->done ? 1.0 : 0.0);
    }
    ks->done = ks->red[5].y != 0.0 ? 1 : 0;
    ks->kused = 0;
}

// after the cycle's last Gram-Schmidt: K += steps of this cycle; kused = K for the inner sign
__global__ void k_rs_mid(KState* ks) {
    if (ks->status) return;
    const int local = ks->red[5].y != 0.0 ? 0 : ks->kused;
    const int K = (int)ks->red[4].x + local;
    ks->red[4] = make_double2((double)K, 0.0);
    ks->red[5].x = (double)local;
    ks->kused = K;
}

// double-float combination coefficients of this cycle: cdf[l] = c[off + l], l < steps
__global__ void k_rs_coef(const double2* __restrict__ c, float4* __restrict__ cdf, const KState* ks, int off) {
    if (ks->status) return;
    const int local = (int)ks->red[5].x;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < local; l += gridDim.x * blockDim.x)
        cdf[l] = to_f4(d2df(c[off + l]));
}

// y += sum_{l < steps} cdf_l V_l (y FP64)
__global__ void __launch_bounds__(AD_T) k_rs_combine(const float4* __restrict__ V, size_t ld,
                                                     const float4* __restrict__ cdf, const KState* ks,
                                                     double2* __restrict__ y, size_t n) {
    __shared__ float4 red[AD_W][32];
    if (ks->status) return;
    const int local = (int)ks->red[5].x;
    if (local <= 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t e = (size_t)blockIdx.x * 32 + lane;
    const bool in = e < n;
    cx<df> s;
    adf_lincomb(V, ld, local, cdf, e, in, wid, lane, red, s);
    if (wid == 0 && in) {
        const double2 a = y[e], d = df2d(s);
        y[e] = make_double2(a.x + d.x, a.y + d.y);
    }
}

// the next cycle's start vector v_0 = (u_m - V_{<m} c) / nu into slot 0 (each element is read and
// written by its own block) and its FP64 value into x64; after the last cycle, a lucky breakdown
// or an earlier stop, the process is marked stopped and done instead
__global__ void __launch_bounds__(AD_T) k_rs_restart(float4* __restrict__ V, size_t ld, int m,
                                                     const float4* __restrict__ cdf, double2* __restrict__ x64,
                                                     KState* ks, size_t n, int last) {
    __shared__ float4 red[AD_W][32];
    if (ks->status) return;
    if (ks->done || ks->red[5].y != 0.0 || last) {  // the same decision in every block
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ks->red[5].y = 1.0;
            ks->done = 1;
        }
        return;
    }
    const df inu(ks->red[1].x);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t ntile = (n + 31) / 32;
    for (size_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const size_t e = tile * 32 + lane;
        const bool in = e < n;
        cx<df> s;
        adf_lincomb(V, ld, m, cdf, e, in, wid, lane, red, s);
        if (wid == 0 && in) {
            const cx<df> u = from_f4(V[(size_t)m * ld + e]);
            const cx<df> v = mk((u.r - s.r) * inu, (u.i - s.i) * inu);
            V[e] = to_f4(v);
            x64[e] = df2d(v);
        }
        __syncthreads();  // red is reused by the next tile
    }
}

// ---------------------------------------------------------------- launchers --
// the update kernel's grid: one block per 32 elements up to AD_MAXB blocks (its norm partials,
// one double per block, must fit the solve's partials buffer of at least 2^16 doubles)
static constexpr unsigned AD_MAXB = 16384;
static unsigned adf_update_grid(size_t n) {
    const size_t t = (n + 31) / 32;
    return (unsigned)(t < AD_MAXB ? (t ? t : 1) : AD_MAXB);
}

static int adf_grid(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 1024 ? (b ? b : 1) : 1024);
}

void launch_adf_todf(const double2* x, float4* xdf, const KState* ks, size_t n, cudaStream_t st) {
    k_adf_todf<<<adf_grid(n), 256, 0, st>>>(x, xdf, ks, n);
}

void launch_adf_start(const double2* x, float4* v, double2* x64, const KState* ks, size_t n, cudaStream_t st) {
    k_adf_start<<<adf_grid(n), 256, 0, st>>>(x, v, x64, ks, n);
}

int adf_dot_blocks(size_t n) { return (int)((n + AD_CH - 1) / AD_CH); }

void launch_adf_dot(const float4* V, size_t ld, int nvec, const float4* x, double2* h, float4* hdf,
                    double* partials, size_t n, int num_sms, const KState* ks, cudaStream_t st) {
    if (nvec <= 0) return;
    const int nchunk = adf_dot_blocks(n);
    // vectors per warp: about eight blocks per SM in total (four waves of the two that fit an SM with
    // their 80 KB of shared memory), at least one vector per warp
    const long long target = 8ll * (num_sms > 0 ? num_sms : 1);
    long long vpw = ((long long)nvec * nchunk + (long long)AD_W * target - 1) / ((long long)AD_W * target);
    if (vpw < 1) vpw = 1;
    const int vpb = (int)(vpw * AD_W);
    const int ngroup = (nvec + vpb - 1) / vpb;
    double2* part = reinterpret_cast<double2*>(partials);
    static unsigned long long attr_dev = 0;
    if (first_use_on_device(attr_dev))
        cudaFuncSetAttribute(k_adf_dot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adf_dot_smem());
    k_adf_dot<<<dim3(nchunk, ngroup), AD_T, adf_dot_smem(), st>>>(V, ld, nvec, vpb, x, part, n, ks);
    k_adf_dot_reduce<<<(nvec + 7) / 8, 256, 0, st>>>(part, nchunk, nvec, h, hdf, ks);
}

void launch_adf_update(const float4* V, size_t ld, int nvec, const float4* hdf, float4* x, size_t n, KState* ks,
                       double* partials, unsigned int* counter, cudaStream_t st) {
    if (nvec <= 0) return;
    ArnoldiFinDf af = {nullptr, 0, nullptr, nullptr, 0, 0, 0.0};
    k_adf_update<<<adf_update_grid(n), AD_T, 0, st>>>(V, ld, nvec, hdf, x, n, ks, 0, af, partials, counter);
}

void launch_adf_update_fin(const float4* V, size_t ld, int nvec, const float4* hdf, float4* x, double2* H, int ldH,
                           const double2* h1, const double2* h2, int j, int jlast, double* partials,
                           unsigned int* counter, KState* ks, size_t n, cudaStream_t st) {
    // double-float sweeps leave a residual of about 2^-46 |A v_j| where the Krylov space is
    // exhausted (FP64: 2^-53), so the breakdown test sits at 1e-11 instead of FP64's 1e-13
    ArnoldiFinDf af = {H, ldH, h1, h2, j, jlast, 1e-11};
    k_adf_update<<<adf_update_grid(n), AD_T, 0, st>>>(V, ld, nvec, hdf, x, n, ks, 1, af, partials, counter);
}

void launch_adf_normalize(float4* t, double2* x64, const KState* ks, size_t n, cudaStream_t st) {
    k_adf_normalize<<<adf_grid(n), 256, 0, st>>>(t, x64, ks, n);
}

void launch_adf_dot2(const float4* V, size_t ld, int nvec, const float4* x1, const double2* x2, double2* h1,
                     double2* h2, double* partials, size_t n, int num_sms, const KState* ks, cudaStream_t st) {
    if (nvec <= 0) return;
    const int nchunk = adf_dot_blocks(n);
    const long long target = 8ll * (num_sms > 0 ? num_sms : 1);
    long long vpw = ((long long)nvec * nchunk + (long long)AD_W * target - 1) / ((long long)AD_W * target);
    if (vpw < 1) vpw = 1;
    const int vpb = (int)(vpw * AD_W);
    const int ngroup = (nvec + vpb - 1) / vpb;
    double2* part = reinterpret_cast<double2*>(partials);
    static unsigned long long attr_dev = 0;
    if (first_use_on_device(attr_dev))
        cudaFuncSetAttribute(k_adf_dot2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adf_dot2_smem());
    k_adf_dot2<<<dim3(nchunk, ngroup), AD_T, adf_dot2_smem(), st>>>(V, ld, nvec, vpb, x1, x2, part, n, ks);
    k_adf_dot2_reduce<<<(2 * nvec + 7) / 8, 256, 0, st>>>(part, nchunk, nvec, h1, h2, ks);
}

void launch_adf_dcgs(double2* H, int ldH, const double2* h1, const double2* h2, float4* cdf, float4* qdf, KState* ks,
                     int j, int fin, cudaStream_t st) {
    // double-float sweeps: the lucky-breakdown threshold of the double-float CGS2 path (1e-11)
    k_adf_dcgs<<<1, 1024, 0, st>>>(H, ldH, h1, h2, cdf, qdf, ks, j, fin, 1e-11);
}

void launch_adf_update2(const float4* V, size_t ld, int j, const float4* cdf, const float4* qdf, float4* uj,
                        float4* unext, const double2* w, double2* x64, double2* H, int ldH, const double2* h1,
                        const double2* h2, size_t n, KState* ks, cudaStream_t st) {
    unsigned grid = adf_update_grid(n);
    if (grid < (unsigned)j + 1) grid = (unsigned)j + 1;  // blocks 0..j each write one row of column j
    k_adf_update2<<<grid, AD_T, 0, st>>>(V, ld, j, cdf, qdf, uj, unext, w, x64, H, ldH, h1, h2, n, ks);
}

void launch_rs_begin(KState* ks, int cyc, cudaStream_t st) { k_rs_begin<<<1, 1, 0, st>>>(ks, cyc); }
void launch_rs_mid(KState* ks, cudaStream_t st) { k_rs_mid<<<1, 1, 0, st>>>(ks); }
void launch_rs_combine(const float4* V, size_t ld, const double2* c, int off, float4* cdf, const KState* ks, int m,
                       double2* y, size_t n, cudaStream_t st) {
    k_rs_coef<<<(m + 255) / 256 > 0 ? (m + 255) / 256 : 1, 256, 0, st>>>(c, cdf, ks, off);
    k_rs_combine<<<(unsigned)((n + 31) / 32), AD_T, 0, st>>>(V, ld, cdf, ks, y, n);
}
void launch_rs_restart(float4* V, size_t ld, int m, const float4* cdf, double2* x64, KState* ks, size_t n, int last,
                       cudaStream_t st) {
    k_rs_restart<<<adf_update_grid(n), AD_T, 0, st>>>(V, ld, m, cdf, x64, ks, n, last);
}

void launch_adf_combine(const float4* V, size_t ld, const double2* c, float4* cdf, const KState* ks, int kmax,
                        double2* y, size_t n, cudaStream_t st) {
    k_adf_coef<<<(kmax + 255) / 256 > 0 ? (kmax + 255) / 256 : 1, 256, 0, st>>>(c, cdf, ks);
    k_adf_combine<<<(unsigned)((n + 31) / 32), AD_T, 0, st>>>(V, ld, cdf, ks, y, n);
}

}  // namespace ovl
