// Wilson stencil kernels: A = gamma5 D_w(mu) and A^dag = gamma5 D_w(-mu)
// (Sec. 1, Eq. 1.1-1.2; the adjoint enters the two-sided Lanczos recurrence of
// Sec. 4, Eq. 4.2), plus the layout conversions at the library boundary.
//
// One thread per lattice site, 128-thread blocks held to 80 registers so that six
// blocks (24 warps) share an SM: the single application is bound by HBM and its
// DRAM traffic is already the algorithmic minimum (links and x read once, y
// written once), so what remains is keeping enough loads in flight.  A block covers a range of checkerboard
// indices for both parities (first half of the block parity 0, second half
// parity 1), so neighbouring sites -- which have the opposite parity -- are
// processed by the same block and their links/spinors are re-read from L1/L2.
// Spinors are stored [component-chunk][site] with 16-byte chunks (double2 for
// FP64, float4 = two complex for FP32): every load of a warp is one 512-byte
// coalesced transaction.  Links are stored [nu][element][site]; the FP32 12-real
// format keeps rows 0 and 1 and rebuilds row 2 = conj(row0 x row1) in registers.
// The e^{+-mu} factors, kappa and the antiperiodic time phase are applied as
// real scalars to the projected half spinor, so links stay in SU(3).
#include <algorithm>
#include <type_traits>

#include "stencil_impl.cuh"

namespace ovl {

__device__ __forceinline__ int site_of_thread(const Geom& g) {
    const int half = blockDim.x >> 1;
    const int par = threadIdx.x >= half;
    const int cb = blockIdx.x * half + (threadIdx.x - par * half);
    return cb < g.Vh ? par * g.Vh + cb : -1;
}

int dslash_grid(const Geom& g, int threads) { return (g.Vh + threads / 2 - 1) / (threads / 2); }

// Row-grouped traversal of the single stencil on large lattices.  With blocks taken in index order
// the sites of hyperplane x0 + 1 come a whole hyperplane (L1 L2 L4 sites, 42 MB of spinors and
// links on 48^3 x 64) after those of x0, and the x0 neighbours and backward links fall out of L2 in
// between and are read from DRAM again (ncu: 1.45 x the algorithmic bytes there, 1.06 x on
// 32^3 x 64).  This grid visits the rows (x0, x1) as: for each group of gx consecutive x1, for
// each x0, the group's rows; blockIdx.x is the block within its row, blockIdx.y the x1 within its
// group, blockIdx.z = group * L0 + x0 (blocks are issued in linear block order: x, then y, then z).
// The x0 neighbours are then gx rows back (7 MB at gx = 8 on 48^3 x 64) and only the rows at a
// group's edges re-read an x1 neighbour.  Each site is still computed by exactly one thread, with
// the same arithmetic: the result is the same to the bit.
struct RowGrid {
    bool ok;
    dim3 grid;
};
static RowGrid row_grid(const Geom& g, int threads) {
    const int half = threads / 2;
    const int row = g.L[2] * g.L4h;  // sites of one parity in a row (x0, x1)
    if (row % half) return {false, dim3(1)};
    int gx = 1;
    for (int d = 1; d <= 16; ++d)
        if (g.L[1] % d == 0) gx = d;
    const long long z = (long long)(g.L[1] / gx) * g.L[0];
    if (z > 65535) return {false, dim3(1)};
    return {true, dim3(row / half, gx, (unsigned)z)};
}

// block bx of nx within its row
__device__ __forceinline__ int site_of_rows(const Geom& g, int bx, int nx) {
    const int half = blockDim.x >> 1;
    const int par = threadIdx.x >= half;
    const int x0 = blockIdx.z % g.L[0];
    const int x1 = (blockIdx.z / g.L[0]) * gridDim.y + blockIdx.y;
    const int cb = ((x0 * g.L[1] + x1) * nx + bx) * half + (threadIdx.x - par * half);
    return par * g.Vh + cb;
}
__device__ __forceinline__ int site_of_thread_rows(const Geom& g) {
    return site_of_rows(g, blockIdx.x, gridDim.x);
}

// --------------------------------------------- direction-split variants --
// For lattices too small to fill the GPU with one thread per site, the four
// directions of a site go to four warps of the same block (warp w computes the
// forward and backward hop of direction w for 32 consecutive sites, so no warp
// diverges); the four partial spinors meet in shared memory, and the 128
// threads then finish (site, spin) pairs: diagonal term, gamma5, scaling and
// the fused epilogue.  Four times the threads, a quarter of the dependent
// loads per thread.
static constexpr int DS_SITES = 32;

// partial spinors of the four directions: smem[dir][input][site][12]
template <int LF, int NIN>
__device__ __forceinline__ void dir_partials(const Geom& g, const void* U,
                                             const typename VecT<typename LinkReal<LF>::R>::T* const (&x)[NIN],
                                             const HopCoef<typename LinkReal<LF>::R> (&hc)[NIN],
                                             cx<typename LinkReal<LF>::R>* sm) {
    using R = typename LinkReal<LF>::R;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * DS_SITES + lane;
    Spinor<R> acc[NIN];
#pragma unroll
    for (int n = 0; n < NIN; ++n)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[n].s[s][a] = mk(R(0), R(0));
    if (i < g.V) {
        const Coord c = site_coord(g, i);
        switch (w) {  // uniform per warp
            case 0: hops_dir<0, LF, R, NIN>(g, c, i, U, x, acc, hc); break;
            case 1: hops_dir<1, LF, R, NIN>(g, c, i, U, x, acc, hc); break;
            case 2: hops_dir<2, LF, R, NIN>(g, c, i, U, x, acc, hc); break;
            default: hops_dir<3, LF, R, NIN>(g, c, i, U, x, acc, hc); break;
        }
    }
#pragma unroll
    for (int n = 0; n < NIN; ++n)
#pragma unroll
        for (int q = 0; q < 12; ++q) sm[((w * NIN + n) * DS_SITES + lane) * 12 + q] = acc[n].s[q / 3][q % 3];
    __syncthreads();
}

// sum of the four direction partials for (site, spin) of this thread, input n
template <class R, int NIN>
__device__ __forceinline__ void dir_sum(const cx<R>* sm, int n, int site, int sp, cx<R> (&o)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<R> z = mk(R(0), R(0));
#pragma unroll
        for (int w = 0; w < 4; ++w) z = z + sm[((w * NIN + n) * DS_SITES + site) * 12 + 3 * sp + a];
        o[a] = z;
    }
}

template <int LF>
__global__ void __launch_bounds__(128) k_dslash_ds(const void* __restrict__ U,
                                                  const typename VecT<typename LinkReal<LF>::R>::T* __restrict__ x,
                                                  typename VecT<typename LinkReal<LF>::R>::T* __restrict__ y,
                                                  HopCoef<typename LinkReal<LF>::R> hc, int g5, const KState* ks,
                                                  Geom g) {
    using R = typename LinkReal<LF>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R>* sm = reinterpret_cast<cx<R>*>(smraw);
    if (ks && (ks->done || ks->status)) return;
    const typename VecT<R>::T* const xs[1] = {x};
    const HopCoef<R> hcs[1] = {hc};
    dir_partials<LF, 1>(g, U, xs, hcs, sm);
    const int site = threadIdx.x >> 2, sp = threadIdx.x & 3;
    const int i = blockIdx.x * DS_SITES + site;
    if (i >= g.V) return;
    cx<R> o[3];
    dir_sum<R, 1>(sm, 0, site, sp, o);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<R> z = o[a] + ld_comp<R>(x, g.V, i, 3 * sp + a);
        if (g5 && sp >= 2) z = -z;
        st_comp<R>(y, g.V, i, 3 * sp + a, z);
    }
}

template <int LF>
__global__ void __launch_bounds__(128) k_dslash_pair_ds(
    const void* __restrict__ U, const typename VecT<typename LinkReal<LF>::R>::T* __restrict__ v,
    const typename VecT<typename LinkReal<LF>::R>::T* __restrict__ w,
    typename VecT<typename LinkReal<LF>::R>::T* __restrict__ t, typename VecT<typename LinkReal<LF>::R>::T* __restrict__ s,
    HopCoef<typename LinkReal<LF>::R> hv, HopCoef<typename LinkReal<LF>::R> hw, KState* ks, double2* alpha, int step,
    int klast, double* partials, unsigned int* counter, Geom g) {
    using R = typename LinkReal<LF>::R;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R>* sm = reinterpret_cast<cx<R>*>(smraw);
    __shared__ double red[96];
    if (ks->done || ks->status) return;
    const double2 sv = ks->sv, sw = ks->sw;
    const typename VecT<R>::T* const xs[2] = {v, w};
    const HopCoef<R> hcs[2] = {hv, hw};
    dir_partials<LF, 2>(g, U, xs, hcs, sm);
    const int site = threadIdx.x >> 2, sp = threadIdx.x & 3;
    const int i = blockIdx.x * DS_SITES + site;
    double part[3] = {0.0, 0.0, 0.0};
    if (i < g.V) {
        cx<R> ov[3], ow[3];
        dir_sum<R, 2>(sm, 0, site, sp, ov);
        dir_sum<R, 2>(sm, 1, site, sp, ow);
        const cx<R> csv = mk(R(sv.x), R(sv.y)), csw = mk(R(sw.x), R(sw.y));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int q = 3 * sp + a;
            const cx<R> wq = ld_comp<R>(w, g.V, i, q);
            cx<R> tv = ov[a] + ld_comp<R>(v, g.V, i, q);
            cx<R> sq = ow[a] + wq;
            if (sp >= 2) {
                tv = -tv;
                sq = -sq;
            }
            tv = csv * tv;
            sq = csw * sq;
            st_comp<R>(t, g.V, i, q, tv);
            st_comp<R>(s, g.V, i, q, sq);
            const cx<double> z = cdot(up(wq), up(tv));
            part[0] += z.r;
            part[1] += z.i;
            part[2] += norm2(up(tv));
        }
    }
    double out[3];
    if (grid_sum_last<3>(part, partials, counter, out, red)) {
        if (threadIdx.x == 0) {
            const cx<double> a = cdot(d2c(sw), mk(out[0], out[1]));
            alpha[step] = c2d(a);
            const double tn = sqrt(out[2]);
            if (tn > ks->anorm) ks->anorm = tn;
            ks->kused = step + 1;
            if (step == klast) ks->done = 1;
        }
    }
}

__global__ void __launch_bounds__(128) k_dslash_regen_ds(const double2* __restrict__ U, const double2* __restrict__ vi,
                                                         const double2* __restrict__ vim1, double2* __restrict__ vip1,
                                                         double2* __restrict__ y, HopCoef<double> hc,
                                                         const KState* ks, const double2* __restrict__ alpha,
                                                         const double2* __restrict__ beta,
                                                         const double2* __restrict__ gamma,
                                                         const double2* __restrict__ c, int step, Geom g) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<double>* sm = reinterpret_cast<cx<double>*>(smraw);
    if (ks->status || step + 1 >= ks->kused) return;
    const double2* const xs[1] = {vi};
    const HopCoef<double> hcs[1] = {hc};
    dir_partials<LINK_F64, 1>(g, U, xs, hcs, sm);
    const int site = threadIdx.x >> 2, sp = threadIdx.x & 3;
    const int i = blockIdx.x * DS_SITES + site;
    if (i >= g.V) return;
    cx<double> o[3];
    dir_sum<double, 1>(sm, 0, site, sp, o);
    const cx<double> a = d2c(alpha[step]);
    const cx<double> ib = cdiv(mk(1.0, 0.0), d2c(beta[step]));
    const cx<double> gm = step > 0 ? d2c(gamma[step - 1]) : mk(0.0, 0.0);
    const cx<double> cc = d2c(c[step + 1]);
#pragma unroll
    for (int q3 = 0; q3 < 3; ++q3) {
        const int q = 3 * sp + q3;
        const size_t e = (size_t)q * g.V + i;
        const cx<double> self = d2c(vi[e]);
        cx<double> z = o[q3] + self;
        if (sp >= 2) z = -z;
        z = z - a * self;
        if (step > 0) z = z - gm * d2c(vim1[e]);
        z = ib * z;
        vip1[e] = c2d(z);
        cx<double> yy = d2c(y[e]);
        cfma(yy, cc, z);
        y[e] = c2d(yy);
    }
}

static size_t ds_smem(int bytes_per_cx, int nin) { return (size_t)4 * nin * DS_SITES * 12 * bytes_per_cx; }
static int ds_grid(const Geom& g) { return (g.V + DS_SITES - 1) / DS_SITES; }

// one thread per site fills the GPU from about this many sites up
static bool use_ds(const Geom& g) { return g.V < 152 * 1024; }

// ------------------------------------------------------------ single apply --
template <int LF, int MINB, bool ROWS>
__global__ void __launch_bounds__(128, MINB) k_dslash(const void* __restrict__ U,
                                                const typename VecT<typename LinkReal<LF>::R>::T* __restrict__ x,
                                                typename VecT<typename LinkReal<LF>::R>::T* __restrict__ y,
                                                HopCoef<typename LinkReal<LF>::R> hc, int g5, const KState* ks,
                                                Geom g) {
    using R = typename LinkReal<LF>::R;
    if (ks && (ks->done || ks->status)) return;
    const int i = ROWS ? site_of_thread_rows(g) : site_of_thread(g);
    if (i < 0) return;
    const typename VecT<R>::T* const xs[1] = {x};
    Spinor<R> acc[1];
    const HopCoef<R> hcs[1] = {hc};
    apply_site<LF, R, 1>(g, i, U, xs, acc, hcs);
    Spinor<R> self;
    load_spinor(x, g.V, i, self);
    finish_site(acc[0], self, g5 != 0);
    store_spinor(y, g.V, i, acc[0]);
}

// blocks per SM of the FP32 single stencil (128 threads each): 6 measured best on GB300 (48^3 x 64:
// 8 gave 4571 -> 3966 GB/s with 12-real links)
#ifndef OVL_DSLASH_F32_MINB
#define OVL_DSLASH_F32_MINB 6
#endif

static int g_ds_mode = -1;  // -1 auto, 0 one thread per site, 1 direction split
void set_dslash_variant(int mode) { g_ds_mode = mode; }
static bool pick_ds(const Geom& g) { return g_ds_mode < 0 ? use_ds(g) : g_ds_mode == 1; }

void launch_dslash(const void* U, int prec, const void* x, void* y, double mu, double kappa, int gamma5,
                   const Geom& g, cudaStream_t st, const KState* ks) {
    if (pick_ds(g)) {
        if (prec == 0)
            k_dslash_ds<LINK_F64><<<ds_grid(g), 128, ds_smem(16, 1), st>>>(U, (const double2*)x, (double2*)y,
                                                                          make_coef<double>(mu, kappa), gamma5, ks, g);
        else if (prec == 1)
            k_dslash_ds<LINK_F32_12><<<ds_grid(g), 128, ds_smem(8, 1), st>>>(U, (const float4*)x, (float4*)y,
                                                                            make_coef<float>(mu, kappa), gamma5, ks, g);
        else
            k_dslash_ds<LINK_F32_18><<<ds_grid(g), 128, ds_smem(8, 1), st>>>(U, (const float4*)x, (float4*)y,
                                                                            make_coef<float>(mu, kappa), gamma5, ks, g);
        return;
    }
    // FP64: four blocks per SM (128 registers; 80 spilled 1.8 KB); FP32: OVL_DSLASH_F32_MINB per SM
    const int T = 128, B = dslash_grid(g, T);
    const RowGrid rg = row_grid(g, T);
    if (prec == 0) {
        if (rg.ok)
            k_dslash<LINK_F64, 4, true><<<rg.grid, T, 0, st>>>(U, (const double2*)x, (double2*)y,
                                                                make_coef<double>(mu, kappa), gamma5, ks, g);
        else
            k_dslash<LINK_F64, 4, false><<<B, T, 0, st>>>(U, (const double2*)x, (double2*)y,
                                                           make_coef<double>(mu, kappa), gamma5, ks, g);
    } else if (prec == 1) {
        if (rg.ok)
            k_dslash<LINK_F32_12, OVL_DSLASH_F32_MINB, true><<<rg.grid, T, 0, st>>>(
                U, (const float4*)x, (float4*)y, make_coef<float>(mu, kappa), gamma5, ks, g);
        else
            k_dslash<LINK_F32_12, OVL_DSLASH_F32_MINB, false><<<B, T, 0, st>>>(
                U, (const float4*)x, (float4*)y, make_coef<float>(mu, kappa), gamma5, ks, g);
    } else {
        if (rg.ok)
            k_dslash<LINK_F32_18, OVL_DSLASH_F32_MINB, true><<<rg.grid, T, 0, st>>>(
                U, (const float4*)x, (float4*)y, make_coef<float>(mu, kappa), gamma5, ks, g);
        else
            k_dslash<LINK_F32_18, OVL_DSLASH_F32_MINB, false><<<B, T, 0, st>>>(
                U, (const float4*)x, (float4*)y, make_coef<float>(mu, kappa), gamma5, ks, g);
    }
}

// -------------------------------------------------------------- pair apply --
// t = sv * gamma5 D_w(mu) v~,  s = sw * gamma5 D_w(-mu) w~,  alpha[step] = w^dag t
// with w = sw w~.  Skipped (uniformly) once the solve is done or failed.
// The two stencils go to two sets of blocks (which = 0: t and the alpha partials; 1: s), so a thread
// carries one accumulator spinor (half the registers: more warps per SM); which is blockIdx.y on a
// one-dimensional grid, the low bit of blockIdx.x on the row-grouped grid.  Only the t blocks take
// part in the reduction.
template <int LF, bool ROWS>
__global__ void __launch_bounds__(128, LF == LINK_F64 ? 2 : OVL_DSLASH_F32_MINB) k_dslash_pair(const void* __restrict__ U,
                                                     const typename VecT<typename LinkReal<LF>::R>::T* __restrict__ v,
                                                     const typename VecT<typename LinkReal<LF>::R>::T* __restrict__ w,
                                                     typename VecT<typename LinkReal<LF>::R>::T* __restrict__ t,
                                                     typename VecT<typename LinkReal<LF>::R>::T* __restrict__ s,
                                                     HopCoef<typename LinkReal<LF>::R> hv,
                                                     HopCoef<typename LinkReal<LF>::R> hw, KState* ks,
                                                     double2* alpha, int step, int klast, double* partials,
                                                     unsigned int* counter, Geom g) {
    using R = typename LinkReal<LF>::R;
    __shared__ double red[3 * 32];  // grid_sum_last<3>: 32 doubles per value
    if (ks->done || ks->status) return;
    const double2 sv = ks->sv, sw = ks->sw;
    const int which = ROWS ? (int)(blockIdx.x & 1u) : (int)blockIdx.y;
    const int i = ROWS ? site_of_rows(g, blockIdx.x >> 1, gridDim.x >> 1) : site_of_thread(g);
    if (which == 1) {  // s = sw A^dag w~
        if (i >= 0) {
            const typename VecT<R>::T* const xs[1] = {w};
            Spinor<R> acc[1], self;
            const HopCoef<R> hcs[1] = {hw};
            apply_site<LF, R, 1>(g, i, U, xs, acc, hcs);
            load_spinor(w, g.V, i, self);
            finish_site(acc[0], self, true);
            const cx<R> csw = mk(R(sw.x), R(sw.y));
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int a = 0; a < 3; ++a) acc[0].s[sp][a] = csw * acc[0].s[sp][a];
            store_spinor(s, g.V, i, acc[0]);
        }
        return;
    }
    // per-thread sums: FP64 for FP64 data; for FP32 data exact FP32 products summed as compensated
    // FP32 pairs (TwoSum) on the FP32 pipe, widened to FP64 for the block and grid sums
    using A = typename std::conditional<sizeof(R) == 4, AccF, AccD>::type;
    A pa[3];
    if (i >= 0) {  // t = sv A v~, partials of w~^dag t and |t|^2
        const typename VecT<R>::T* const xs[1] = {v};
        Spinor<R> acc[1], self;
        const HopCoef<R> hcs[1] = {hv};
        apply_site<LF, R, 1>(g, i, U, xs, acc, hcs);
        load_spinor(v, g.V, i, self);
        finish_site(acc[0], self, true);
        load_spinor(w, g.V, i, self);
        const cx<R> csv = mk(R(sv.x), R(sv.y));
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[0].s[sp][a] = csv * acc[0].s[sp][a];
                acc_cdot(pa, self.s[sp][a], acc[0].s[sp][a]);  // w~^dag t
                acc_norm2(pa[2], acc[0].s[sp][a]);
            }
        store_spinor(t, g.V, i, acc[0]);
    }
    double part[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if constexpr (sizeof(R) == 4) part[j] = (double)pa[j].hi + (double)pa[j].lo;
        else part[j] = pa[j].v;
    }
    double out[3];
    const unsigned nx = ROWS ? gridDim.x >> 1 : gridDim.x;
    const unsigned bx = ROWS ? blockIdx.x >> 1 : blockIdx.x;
    const unsigned blk = ROWS ? bx + nx * (blockIdx.y + gridDim.y * blockIdx.z) : bx;
    const unsigned nblk = ROWS ? nx * gridDim.y * gridDim.z : nx;
    if (grid_sum_last<3>(part, partials, counter, out, red, blk, nblk)) {
        if (threadIdx.x == 0) {
            // alpha = w^dag t = conj(sw) * (w~^dag t)
            cx<double> a = cdot(d2c(sw), mk(out[0], out[1]));
            alpha[step] = c2d(a);
            const double tn = sqrt(out[2]);
            if (tn > ks->anorm) ks->anorm = tn;
            ks->kused = step + 1;
            if (step == klast) ks->done = 1;
        }
    }
}

int dslash_pair_blocks(const Geom& g) { return pick_ds(g) ? ds_grid(g) : dslash_grid(g, 128); }

void launch_dslash_pair(const void* U, int prec, const void* v, const void* w, void* t, void* s, double mu,
                        double kappa, KState* ks, double2* alpha, int step, int klast, double* partials,
                        unsigned int* counter, const Geom& g, cudaStream_t st) {
    const int B = dslash_pair_blocks(g);  // the partial-sum slots the fused reduction writes
    if (pick_ds(g)) {
        static unsigned long long attr_dev = 0;
        if (first_use_on_device(attr_dev))
            cudaFuncSetAttribute(k_dslash_pair_ds<LINK_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ds_smem(16, 2));
        if (prec == 0)
            k_dslash_pair_ds<LINK_F64><<<B, 128, ds_smem(16, 2), st>>>(
                U, (const double2*)v, (const double2*)w, (double2*)t, (double2*)s, make_coef<double>(mu, kappa),
                make_coef<double>(-mu, kappa), ks, alpha, step, klast, partials, counter, g);
        else
            k_dslash_pair_ds<LINK_F32_12><<<B, 128, ds_smem(8, 2), st>>>(
                U, (const float4*)v, (const float4*)w, (float4*)t, (float4*)s, make_coef<float>(mu, kappa),
                make_coef<float>(-mu, kappa), ks, alpha, step, klast, partials, counter, g);
        return;
    }
    // large lattices: the row-grouped block order of the single stencil (same block count, so the
    // same partial-sum slots; the partials are summed in linear block order)
    const int T = 128;
    RowGrid rg = row_grid(g, T);
    rg.grid.x *= 2;  // the two stencils
    const dim3 g1(B, 2);
    if (prec == 0) {
        if (rg.ok)
            k_dslash_pair<LINK_F64, true><<<rg.grid, T, 0, st>>>(
                U, (const double2*)v, (const double2*)w, (double2*)t, (double2*)s, make_coef<double>(mu, kappa),
                make_coef<double>(-mu, kappa), ks, alpha, step, klast, partials, counter, g);
        else
            k_dslash_pair<LINK_F64, false><<<g1, T, 0, st>>>(
                U, (const double2*)v, (const double2*)w, (double2*)t, (double2*)s, make_coef<double>(mu, kappa),
                make_coef<double>(-mu, kappa), ks, alpha, step, klast, partials, counter, g);
    } else {
        if (rg.ok)
            k_dslash_pair<LINK_F32_12, true><<<rg.grid, T, 0, st>>>(
                U, (const float4*)v, (const float4*)w, (float4*)t, (float4*)s, make_coef<float>(mu, kappa),
                make_coef<float>(-mu, kappa), ks, alpha, step, klast, partials, counter, g);
        else
            k_dslash_pair<LINK_F32_12, false><<<g1, T, 0, st>>>(
                U, (const float4*)v, (const float4*)w, (float4*)t, (float4*)s, make_coef<float>(mu, kappa),
                make_coef<float>(-mu, kappa), ks, alpha, step, klast, partials, counter, g);
    }
}

// ------------------------------------------------------ two-pass regeneration --
// v_{i+1} = ((A - alpha_i) v_i - gamma_{i-1} v_{i-1}) / beta_i ;  y += c_{i+1} v_{i+1}
__global__ void __launch_bounds__(256) k_dslash_regen(const double2* __restrict__ U, const double2* __restrict__ vi,
                                                      const double2* __restrict__ vim1, double2* __restrict__ vip1,
                                                      double2* __restrict__ y, HopCoef<double> hc, const KState* ks,
                                                      const double2* __restrict__ alpha,
                                                      const double2* __restrict__ beta,
                                                      const double2* __restrict__ gamma,
                                                      const double2* __restrict__ c, int step, Geom g) {
    if (ks->status || step + 1 >= ks->kused) return;
    const int i = site_of_thread(g);
    if (i < 0) return;
    const double2* const xs[1] = {vi};
    Spinor<double> acc[1];
    const HopCoef<double> hcs[1] = {hc};
    apply_site<LINK_F64, double, 1>(g, i, U, xs, acc, hcs);
    Spinor<double> self;
    load_spinor(vi, g.V, i, self);
    finish_site(acc[0], self, true);
    const cx<double> a = d2c(alpha[step]);
    const cx<double> ib = cdiv(mk(1.0, 0.0), d2c(beta[step]));
    const cx<double> gm = step > 0 ? d2c(gamma[step - 1]) : mk(0.0, 0.0);
    const cx<double> cc = d2c(c[step + 1]);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const size_t e = (size_t)(3 * sp + q) * g.V + i;
            cx<double> z = acc[0].s[sp][q] - a * self.s[sp][q];
            if (step > 0) z = z - gm * d2c(vim1[e]);
            z = ib * z;
            vip1[e] = c2d(z);
            cx<double> yy = d2c(y[e]);
            cfma(yy, cc, z);
            y[e] = c2d(yy);
        }
}

void launch_dslash_regen(const double2* U, const double2* vi, const double2* vim1, double2* vip1, double2* y,
                         double mu, double kappa, const KState* ks, const double2* alpha, const double2* beta,
                         const double2* gamma, const double2* c, int step, const Geom& g, cudaStream_t st) {
    if (pick_ds(g)) {
        k_dslash_regen_ds<<<ds_grid(g), 128, ds_smem(16, 1), st>>>(U, vi, vim1, vip1, y, make_coef<double>(mu, kappa),
                                                                   ks, alpha, beta, gamma, c, step, g);
        return;
    }
    const int T = 128, B = dslash_grid(g, T);
    k_dslash_regen<<<B, T, 0, st>>>(U, vi, vim1, vip1, y, make_coef<double>(mu, kappa), ks, alpha, beta, gamma, c,
                                    step, g);
}

// FP64 device-layout vectors (double2 [12][V]) to the FP32 device layout (float4 [6][V],
// components 2c, 2c+1 in one float4): nvec consecutive vectors of 12V complex each.
__global__ void k_native_f64_to_f32(const double2* __restrict__ x, float4* __restrict__ y, int V, int nvec) {
    const size_t tot = (size_t)nvec * 6 * V;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const size_t vec = e / ((size_t)6 * V);
        const size_t r = e - vec * 6 * V;
        const int c2 = (int)(r / V), i = (int)(r - (size_t)c2 * V);
        const double2* xv = x + vec * 12 * (size_t)V;
        const double2 a = xv[(size_t)(2 * c2) * V + i], b = xv[(size_t)(2 * c2 + 1) * V + i];
        y[vec * 6 * (size_t)V + (size_t)c2 * V + i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}

void launch_native_f64_to_f32(const double2* x, void* y, const Geom& g, int nvec, cudaStream_t st) {
    const size_t tot = (size_t)nvec * 6 * g.V;
    int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
    k_native_f64_to_f32<<<blocks, 256, 0, st>>>(x, (float4*)y, g.V, nvec);
}

// the inverse: FP32 device layout (float4 [6][V]) to the FP64 device layout (double2 [12][V])
__global__ void k_native_f32_to_f64(const float4* __restrict__ x, double2* __restrict__ y, int V, int nvec) {
    const size_t tot = (size_t)nvec * 6 * V;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const size_t vec = e / ((size_t)6 * V);
        const size_t r = e - vec * 6 * V;
        const int c2 = (int)(r / V), i = (int)(r - (size_t)c2 * V);
        const float4 a = x[vec * 6 * (size_t)V + (size_t)c2 * V + i];
        double2* yv = y + vec * 12 * (size_t)V;
        yv[(size_t)(2 * c2) * V + i] = make_double2((double)a.x, (double)a.y);
        yv[(size_t)(2 * c2 + 1) * V + i] = make_double2((double)a.z, (double)a.w);
    }
}

void launch_native_f32_to_f64(const void* x, double2* y, const Geom& g, int nvec, cudaStream_t st) {
    const size_t tot = (size_t)nvec * 6 * g.V;
    int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
    k_native_f32_to_f64<<<blocks, 256, 0, st>>>((const float4*)x, y, g.V, nvec);
}

// Neighbour table: nbr[h][i] = internal index of the neighbour of site i in hop h (h < 4: x + nu,
// h >= 4: x - nu, nu = h & 3), bit-inverted (~index, negative) where the hop crosses the
// antiperiodic time boundary and takes the phase -1.
__global__ void k_build_nbr(int* __restrict__ nbr, Geom g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const Coord c = site_coord(g, i);
    for (int h = 0; h < 8; ++h) {
        const int nu = h & 3;
        const bool fwd = h < 4;
        const int nb = neighbour(g, c, nu, fwd ? +1 : -1);
        const bool edge = nu == 3 && (fwd ? (c.x[3] == g.L[3] - 1) : (c.x[3] == 0));
        nbr[(size_t)h * g.V + i] = (edge && g.bc_t < 0) ? ~nb : nb;
    }
}

void launch_build_nbr(int* nbr, const Geom& g, cudaStream_t st) {
    k_build_nbr<<<(g.V + 127) / 128, 128, 0, st>>>(nbr, g);
}

// ---------------------------------------------------------------- layouts --
__global__ void k_pack_gauge(const double2* __restrict__ Uc, double2* __restrict__ U64, float4* __restrict__ U12,
                             float2* __restrict__ U18, float4* __restrict__ Udf, Geom g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const Coord c = site_coord(g, i);
    const int s = canon_index(g, c.x);
    for (int nu = 0; nu < 4; ++nu) {
        double2 e[9];
        for (int q = 0; q < 9; ++q) e[q] = Uc[((size_t)s * 4 + nu) * 9 + q];
        for (int q = 0; q < 9; ++q) {
            U64[((size_t)nu * 9 + q) * g.V + i] = e[q];
            U18[((size_t)nu * 9 + q) * g.V + i] = make_float2((float)e[q].x, (float)e[q].y);
            const dfc d = c2dfc(d2df(e[q]));
            Udf[((size_t)nu * 9 + q) * g.V + i] = make_float4(d.rh, d.rl, d.ih, d.il);
        }
        U12[((size_t)nu * 3 + 0) * g.V + i] = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
        U12[((size_t)nu * 3 + 1) * g.V + i] = make_float4(e[2].x, e[2].y, e[3].x, e[3].y);
        U12[((size_t)nu * 3 + 2) * g.V + i] = make_float4(e[4].x, e[4].y, e[5].x, e[5].y);
    }
}

__global__ void k_f64_to_df(void* x, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 v = reinterpret_cast<double2*>(x)[e];
        reinterpret_cast<dfc*>(x)[e] = c2dfc(d2df(v));
    }
}
__global__ void k_df_to_f64(void* x, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const dfc v = reinterpret_cast<dfc*>(x)[e];
        reinterpret_cast<double2*>(x)[e] = df2d(dfc2c(v));
    }
}
void launch_f64_to_df(void* x, size_t n, cudaStream_t st) {
    k_f64_to_df<<<(int)std::min<size_t>((n + 255) / 256, 2048), 256, 0, st>>>(x, n);
}
void launch_df_to_f64(void* x, size_t n, cudaStream_t st) {
    k_df_to_f64<<<(int)std::min<size_t>((n + 255) / 256, 2048), 256, 0, st>>>(x, n);
}

void launch_pack_gauge(const double2* U_canon, double2* U64, float4* U12, float2* U18, float4* Udf, const Geom& g,
                       cudaStream_t st) {
    k_pack_gauge<<<(g.V + 127) / 128, 128, 0, st>>>(U_canon, U64, U12, U18, Udf, g);
}

__global__ void k_pack_spinor(const double2* __restrict__ canon, void* __restrict__ native, int prec, Geom g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const Coord c = site_coord(g, i);
    const int s = canon_index(g, c.x);
    if (prec == 0) {
        double2* o = (double2*)native;
        for (int q = 0; q < 12; ++q) o[(size_t)q * g.V + i] = canon[(size_t)s * 12 + q];
    } else {
        float4* o = (float4*)native;
        for (int q = 0; q < 6; ++q) {
            double2 a = canon[(size_t)s * 12 + 2 * q], b = canon[(size_t)s * 12 + 2 * q + 1];
            o[(size_t)q * g.V + i] = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

void launch_pack_spinor(const double2* canon, void* native, int prec, const Geom& g, cudaStream_t st) {
    k_pack_spinor<<<(g.V + 127) / 128, 128, 0, st>>>(canon, native, prec, g);
}

__global__ void k_unpack_spinor(const void* __restrict__ native, int prec, double2* __restrict__ canon,
                                const double2* __restrict__ b, int g5, Geom g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const Coord c = site_coord(g, i);
    const int s = canon_index(g, c.x);
    for (int q = 0; q < 12; ++q) {
        double2 v;
        if (prec == 0) {
            v = ((const double2*)native)[(size_t)q * g.V + i];
        } else {
            float4 f = ((const float4*)native)[(size_t)(q / 2) * g.V + i];
            v = (q & 1) ? make_double2(f.z, f.w) : make_double2(f.x, f.y);
        }
        if (g5 && q >= 6) v = make_double2(-v.x, -v.y);
        if (b) {
            double2 bb = b[(size_t)s * 12 + q];
            v.x += bb.x;
            v.y += bb.y;
        }
        canon[(size_t)s * 12 + q] = v;
    }
}

void launch_unpack_spinor(const void* native, int prec, double2* canon, const double2* b_canon, int g5,
                          const Geom& g, cudaStream_t st) {
    k_unpack_spinor<<<(g.V + 127) / 128, 128, 0, st>>>(native, prec, canon, b_canon, g5, g);
}

}  // namespace ovl
