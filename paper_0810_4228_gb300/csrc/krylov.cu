// Krylov recurrences and vector kernels:
//  * the two-sided Lanczos update of Sec. 4, Eq. 4.2 with its three inner
//    products (w^^dag v^, |v^|^2, |w^|^2) fused into the same pass and the
//    coefficients beta_i, gamma_i set by the last block;
//  * classical Gram-Schmidt (applied twice) for the Arnoldi relation
//    A V_k = V_k H_k + beta_k v_{k+1} e_k^T of Sec. 2, Eq. 2.2-2.3, as a
//    many-vector dot product and a many-vector update over the stored basis;
//  * the LR-deflation split of the source (Sec. 3, Eq. 3.2-3.4; Sec. 4, Eq. 4.5);
//  * the final combination y = sum_i c_i v_i (Eq. 2.6 / 4.4).
// All reductions accumulate in FP64 and are deterministic (fixed block order).
// Every kernel returns at once (uniformly) when the solve is finished or failed,
// so a whole solve can be captured once as a CUDA graph and replayed.
#include <type_traits>
#include "df32.cuh"
#include "ovl_kernels.h"

namespace ovl {

template <class T> struct Elem;
template <> struct Elem<double2> {
    using R = double;
    static __device__ __forceinline__ cx<double> ld(const double2* p, size_t e) { double2 v = p[e]; return mk(v.x, v.y); }
    static __device__ __forceinline__ void st(double2* p, size_t e, cx<double> z) { p[e] = make_double2(z.r, z.i); }
};
template <> struct Elem<float2> {
    using R = float;
    static __device__ __forceinline__ cx<float> ld(const float2* p, size_t e) { float2 v = p[e]; return mk(v.x, v.y); }
    static __device__ __forceinline__ void st(float2* p, size_t e, cx<float> z) { p[e] = make_float2(z.r, z.i); }
};

static int grid_for(size_t n, int threads, int cap = 4096) {
    size_t b = (n + threads - 1) / threads;
    if (b > (size_t)cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------------- state --
__global__ void k_state_init(KState* ks) {
    KState z = {};
    z.bdstep = -1;
    z.sv = z.sw = z.svp = z.swp = make_double2(1.0, 0.0);
    *ks = z;
}
void launch_state_init(KState* ks, cudaStream_t st) { k_state_init<<<1, 1, 0, st>>>(ks); }

// ------------------------------------------------------------ 2sL update --
// v^ = t - alpha_i v_i - gamma_{i-1} v_{i-1},  w^ = s - conj(alpha_i) w_i - conj(beta_{i-1}) w_{i-1}
// with v_i = sv v~_i etc.; stores v~_{i+1} = v^, w~_{i+1} = w^.
// With m > 0 the deflated directions are projected out in the same pass
// (re-projection): v^ -= R p, w^ -= L q with p = L^dag t, q = R^dag s given in
// pq (R, L in the precision of the vectors).  In exact arithmetic L^dag v_i = 0 and
// R^dag w_i = 0, so this only removes what rounding brought back.
template <class T>
__global__ void __launch_bounds__(256) k_lanczos_step(const T* __restrict__ t, const T* __restrict__ s,
                                                      const T* __restrict__ vi, const T* __restrict__ wi,
                                                      const T* __restrict__ vim1, const T* __restrict__ wim1,
                                                      T* __restrict__ vn, T* __restrict__ wn, KState* ks,
                                                      const double2* alpha, double2* beta, double2* gamma,
                                                      double2* vscale, int step, double* partials,
                                                      unsigned int* counter, size_t n, const T* __restrict__ Rp,
                                                      const T* __restrict__ Lp, const double2* __restrict__ pq,
                                                      int m) {
    using R = typename Elem<T>::R;
    __shared__ double red[128];
    __shared__ cx<R> pqs[2 * 64];
    if (ks->done || ks->status) return;
    for (int j = threadIdx.x; j < 2 * m; j += blockDim.x) pqs[j] = mk(R(pq[j].x), R(pq[j].y));
    __syncthreads();
    const cx<double> a = d2c(alpha[step]);
    const cx<double> ca = a * d2c(ks->sv);
    const cx<double> da = conj(a) * d2c(ks->sw);
    cx<double> cg = mk(0.0, 0.0), db = mk(0.0, 0.0);
    if (step > 0) {
        cg = d2c(gamma[step - 1]) * d2c(ks->svp);
        db = conj(d2c(beta[step - 1])) * d2c(ks->swp);
    }
    const cx<R> ca_ = mk(R(ca.r), R(ca.i)), da_ = mk(R(da.r), R(da.i));
    const cx<R> cg_ = mk(R(cg.r), R(cg.i)), db_ = mk(R(db.r), R(db.i));
    // per-thread sums of Re/Im w^^dag v^, |v^|^2, |w^|^2: FP64 for FP64 vectors; for FP32 vectors exact
    // FP32 products summed as compensated FP32 pairs on the FP32 pipe (GB300's FP64 pipe would bound
    // the kernel), widened to FP64 for the block and grid sums
    using A = typename std::conditional<sizeof(R) == 4, AccF, AccD>::type;
    A pa[4];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        cx<R> v = Elem<T>::ld(t, e) - ca_ * Elem<T>::ld(vi, e);
        cx<R> w = Elem<T>::ld(s, e) - da_ * Elem<T>::ld(wi, e);
        if (step > 0) {
            v = v - cg_ * Elem<T>::ld(vim1, e);
            w = w - db_ * Elem<T>::ld(wim1, e);
        }
        for (int j = 0; j < m; ++j) {
            v = v - pqs[j] * Elem<T>::ld(Rp + (size_t)j * n, e);
            w = w - pqs[m + j] * Elem<T>::ld(Lp + (size_t)j * n, e);
        }
        Elem<T>::st(vn, e, v);
        Elem<T>::st(wn, e, w);
        acc_cdot(pa, w, v);  // w^^dag v^
        acc_norm2(pa[2], v);
        acc_norm2(pa[3], w);
    }
    double part[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if constexpr (sizeof(R) == 4) part[j] = (double)pa[j].hi + (double)pa[j].lo;
        else part[j] = pa[j].v;
    }
    double out[4];
    if (grid_sum_last<4>(part, partials, counter, out, red)) {
        if (threadIdx.x == 0) {
            const double nv = sqrt(out[2]), nw = sqrt(out[3]);
            const cx<double> delta = mk(out[0], out[1]);
            if (nv <= 1e-13 * fmax(ks->anorm, 1e-300)) {
                ks->done = 1;  // lucky breakdown: K_{i+1}(A, v_1) is invariant
            } else if (sqrt(norm2(delta)) <= 1e-14 * nv * nw) {
                ks->bdstep = step + 1;  // serious breakdown: keep the approximation from G_{i+1}
                ks->done = 1;
            } else {
                const cx<double> g = mk(out[0] / nv, out[1] / nv);
                beta[step] = make_double2(nv, 0.0);
                gamma[step] = c2d(g);
                ks->svp = ks->sv;
                ks->swp = ks->sw;
                ks->sv = make_double2(1.0 / nv, 0.0);
                ks->sw = c2d(cdiv(mk(1.0, 0.0), conj(g)));
                if (vscale) vscale[step + 1] = ks->sv;
            }
        }
    }
}

void launch_lanczos_step(int prec, const void* t, const void* s, const void* vi, const void* wi, const void* vim1,
                         const void* wim1, void* vnext, void* wnext, KState* ks, const double2* alpha, double2* beta,
                         double2* gamma, double2* vscale, int step, int kmax, double* partials,
                         unsigned int* counter, size_t n, cudaStream_t st, const void* Rp, const void* Lp,
                         const double2* pq, int m) {
    (void)kmax;
    const int T = 256, B = grid_for(n, T, 1024);
    if (prec == 0)
        k_lanczos_step<double2><<<B, T, 0, st>>>((const double2*)t, (const double2*)s, (const double2*)vi,
                                                 (const double2*)wi, (const double2*)vim1, (const double2*)wim1,
                                                 (double2*)vnext, (double2*)wnext, ks, alpha, beta, gamma, vscale,
                                                 step, partials, counter, n, (const double2*)Rp, (const double2*)Lp,
                                                 pq, m);
    else
        k_lanczos_step<float2><<<B, T, 0, st>>>((const float2*)t, (const float2*)s, (const float2*)vi,
                                                (const float2*)wi, (const float2*)vim1, (const float2*)wim1,
                                                (float2*)vnext, (float2*)wnext, ks, alpha, beta, gamma, vscale,
                                                step, partials, counter, n, (const float2*)Rp, (const float2*)Lp,
                                                pq, m);
}

// ---------------------------------------------------------- many-vector dot --
// stage 1: block b covers elements [b*256, b*256+256); warp w computes the partial
// dots of vectors l = w, w+8, ... over that chunk.
static constexpr int MD_CHUNK = 256;

__global__ void __launch_bounds__(256) k_multidot1(const double2* __restrict__ V, size_t ld, int nvec,
                                                   const double2* __restrict__ x, double2* __restrict__ part,
                                                   size_t n, const KState* ks) {
    __shared__ double2 xs[MD_CHUNK];
    if (ks && (ks->done || ks->status)) return;
    const size_t base = (size_t)blockIdx.x * MD_CHUNK;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < MD_CHUNK; q += blockDim.x) {
        const size_t e = base + q;
        xs[q] = e < n ? x[e] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int l = wid; l < nvec; l += nw) {
        const double2* Vl = V + (size_t)l * ld;
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int q = lane; q < MD_CHUNK; q += 32) {
            const size_t e = base + q;
            if (e < n) {
                const double2 v = __ldg(Vl + e), xx = xs[q];
                re += v.x * xx.x + v.y * xx.y;
                im += v.x * xx.y - v.y * xx.x;
            }
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) part[(size_t)l * gridDim.x + blockIdx.x] = make_double2(re, im);
    }
}

// stage 2: one warp per vector sums the block partials (fixed order)
__global__ void k_multidot2(const double2* __restrict__ part, int nblk, int nvec, double2* h, int acc,
                            const KState* ks) {
    if (ks && (ks->done || ks->status)) return;
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
        if (acc) {
            h[l].x += re;
            h[l].y += im;
        } else {
            h[l] = make_double2(re, im);
        }
    }
}

// FP32 vectors and FP32 basis: products and the per-lane partial sums in FP32, the
// reduction across lanes and blocks in FP64 (used for re-projection in the FP32 pass,
// where FP32 accuracy is all that is needed).
__global__ void __launch_bounds__(256) k_multidot1_f32(const float2* __restrict__ V, size_t ld, int nvec,
                                                       const float2* __restrict__ x, double2* __restrict__ part,
                                                       size_t n, const KState* ks) {
    __shared__ float2 xs[MD_CHUNK];
    if (ks && (ks->done || ks->status)) return;
    const size_t base = (size_t)blockIdx.x * MD_CHUNK;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = threadIdx.x; q < MD_CHUNK; q += blockDim.x) {
        const size_t e = base + q;
        xs[q] = e < n ? x[e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int l = wid; l < nvec; l += nw) {
        const float2* Vl = V + (size_t)l * ld;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int q = lane; q < MD_CHUNK; q += 32) {
            const size_t e = base + q;
            if (e < n) {
                const float2 v = __ldg(Vl + e), xx = xs[q];
                re += v.x * xx.x + v.y * xx.y;
                im += v.x * xx.y - v.y * xx.x;
            }
        }
        double dr = warp_sum((double)re), di = warp_sum((double)im);
        if (lane == 0) part[(size_t)l * gridDim.x + blockIdx.x] = make_double2(dr, di);
    }
}

void launch_multidot_f32(const float2* V, size_t ld, int nvec, const float2* x, double2* h, double* partials,
                         size_t n, cudaStream_t st, const KState* ks) {
    if (nvec <= 0) return;
    const int nb = (int)((n + MD_CHUNK - 1) / MD_CHUNK);
    double2* part = reinterpret_cast<double2*>(partials);
    k_multidot1_f32<<<nb, 256, 0, st>>>(V, ld, nvec, x, part, n, ks);
    k_multidot2<<<(nvec + 7) / 8, 256, 0, st>>>(part, nb, nvec, h, 0, ks);
}

int multidot_blocks(size_t n) { return (int)((n + MD_CHUNK - 1) / MD_CHUNK); }

void launch_multidot(const double2* V, size_t ld, int nvec, const double2* x, double2* h, int acc, double* partials,
                     size_t n, cudaStream_t st, const KState* ks, int step) {
    (void)step;
    if (nvec <= 0) return;
    const int nb = multidot_blocks(n);
    double2* part = reinterpret_cast<double2*>(partials);
    k_multidot1<<<nb, 256, 0, st>>>(V, ld, nvec, x, part, n, ks);
    k_multidot2<<<(nvec + 7) / 8, 256, 0, st>>>(part, nb, nvec, h, acc, ks);
}

// ------------------------------------------------------- many-vector update --
// x -= sum_l h[l] V_l ; mode 1 additionally finishes Arnoldi step j (norm of x,
// column j of H, breakdown check) in the last block.
struct ArnoldiFin {
    double2* H;
    int ldH;
    const double2* h1;
    const double2* h2;
    int j;
    int jlast;
};

__global__ void __launch_bounds__(256) k_multiaxpy(const double2* __restrict__ V, size_t ld, int nvec,
                                                   const double2* __restrict__ h, double2* __restrict__ x,
                                                   size_t n, KState* ks, int mode, ArnoldiFin af,
                                                   double* partials, unsigned int* counter) {
    extern __shared__ double2 hs[];
    __shared__ double red[32];
    if (ks->done || ks->status) return;
    for (int l = threadIdx.x; l < nvec; l += blockDim.x) hs[l] = h[l];
    __syncthreads();
    double part[1] = {0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        cx<double> z = d2c(x[e]);
        for (int l = 0; l < nvec; ++l) {
            const double2 v = __ldg(V + (size_t)l * ld + e);
            const double2 c = hs[l];
            z.r -= c.x * v.x - c.y * v.y;
            z.i -= c.x * v.y + c.y * v.x;
        }
        x[e] = c2d(z);
        part[0] += norm2(z);
    }
    if (mode == 0) return;
    double out[1];
    if (grid_sum_last<1>(part, partials, counter, out, red)) {
        // Arnoldi: H[0..j, j] = h1 + h2, H[j+1, j] = |x|
        const int j = af.j;
        double hh = 0.0;
        for (int r = threadIdx.x; r <= j; r += blockDim.x) {
            const double2 a = af.h1[r], b = af.h2[r];
            const double2 v = make_double2(a.x + b.x, a.y + b.y);
            af.H[r + (size_t)j * af.ldH] = v;
            hh += v.x * v.x + v.y * v.y;
        }
        double hv[1] = {hh};
        block_sum<1>(hv, red);
        if (threadIdx.x == 0) {
            const double hn = sqrt(out[0]);
            af.H[(j + 1) + (size_t)j * af.ldH] = make_double2(hn, 0.0);
            const double colnorm = sqrt(hv[0] + out[0]);
            if (colnorm > ks->anorm) ks->anorm = colnorm;
            ks->kused = j + 1;
            ks->red[0] = make_double2(hn, 0.0);
            if (hn <= 1e-13 * fmax(ks->anorm, 1e-300) || j == af.jlast) ks->done = 1;
        }
    }
}

void launch_multiaxpy(const double2* V, size_t ld, int nvec, const double2* h, double2* x, double* partials,
                      unsigned int* counter, KState* ks, int norm_out, size_t n, cudaStream_t st, int step) {
    (void)step;
    if (nvec <= 0) return;
    ArnoldiFin af = {};
    k_multiaxpy<<<grid_for(n, 256, 1024), 256, sizeof(double2) * nvec, st>>>(V, ld, nvec, h, x, n, ks, 0, af,
                                                                              partials, counter);
    (void)norm_out;
}

void launch_arnoldi_orth2(const double2* V, size_t ld, int nvec, const double2* h2, double2* x, double2* H, int ldH,
                          const double2* h1, int j, int jlast, double* partials, unsigned int* counter, KState* ks,
                          size_t n, cudaStream_t st) {
    ArnoldiFin af = {H, ldH, h1, h2, j, jlast};
    k_multiaxpy<<<grid_for(n, 256, 1024), 256, sizeof(double2) * nvec, st>>>(V, ld, nvec, h2, x, n, ks, 1, af,
                                                                              partials, counter);
}

// v_{j+1} = t / |t| (skipped after the last step or a lucky breakdown)
__global__ void k_arnoldi_normalize(double2* t, const KState* ks, size_t n) {
    if (ks->done || ks->status) return;
    const double inv = 1.0 / ks->red[0].x;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double2 v = t[e];
        t[e] = make_double2(v.x * inv, v.y * inv);
    }
}
void launch_arnoldi_normalize(double2* t, const KState* ks, size_t n, cudaStream_t st) {
    k_arnoldi_normalize<<<grid_for(n, 256, 1024), 256, 0, st>>>(t, ks, n);
}

// ---------------------------------------------------------- deflation split --
// bR = b - R p, bL = b - L q, y = R (sgn(Re lambda) p); |bR|^2 and bL^dag bR reduced.
// Start of the Krylov processes: v_1 = bR/|bR|; for 2sL w_1 = bL / conj(bL^dag v_1).
__global__ void __launch_bounds__(256) k_deflate_split(const double2* __restrict__ b, const double2* __restrict__ R,
                                                       const double2* __restrict__ L,
                                                       const double2* __restrict__ lam, int m,
                                                       const double2* __restrict__ pq, double2* __restrict__ bR,
                                                       double2* __restrict__ bL, double2* __restrict__ y,
                                                       KState* ks, double2* vscale, double* partials,
                                                       unsigned int* counter, size_t n) {
    extern __shared__ double2 cs[];  // p, q, sgn(lambda) p
    __shared__ double red[128];
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double2 p = pq[j], q = pq[m + j];
        cs[j] = p;
        cs[m + j] = q;
        const double sg = lam[j].x > 0.0 ? 1.0 : -1.0;  // sgn z = sgn(Re z), Eq. 1.4
        cs[2 * m + j] = make_double2(sg * p.x, sg * p.y);
    }
    __syncthreads();
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const cx<double> bv = d2c(b[e]);
        part[3] += norm2(bv);
        cx<double> r = bv, l = bv, yy = mk(0.0, 0.0);
        for (int j = 0; j < m; ++j) {
            const cx<double> Rj = d2c(__ldg(R + (size_t)j * n + e));
            const cx<double> Lj = d2c(__ldg(L + (size_t)j * n + e));
            r = r - Rj * d2c(cs[j]);
            l = l - Lj * d2c(cs[m + j]);
            yy = yy + Rj * d2c(cs[2 * m + j]);
        }
        bR[e] = c2d(r);
        if (bL) bL[e] = c2d(l);
        y[e] = c2d(yy);
        part[0] += norm2(r);
        const cx<double> z = cdot(l, r);
        part[1] += z.r;
        part[2] += z.i;
    }
    double out[4];
    if (grid_sum_last<4>(part, partials, counter, out, red)) {
        if (threadIdx.x == 0) {
            const double nR = sqrt(out[0]);
            ks->nR = nR;
            // b_perp^R vanishes up to rounding (b in the deflated space, or b = 0):
            // nothing is left to approximate and sgn(A) b is the exact part
            if (nR <= 1e-13 * sqrt(out[3])) {
                ks->nR = 0.0;
                ks->done = 1;
                ks->kused = 0;
            } else {
                ks->sv = make_double2(1.0 / nR, 0.0);
                if (vscale) vscale[0] = ks->sv;
                const cx<double> d = mk(out[1] / nR, out[2] / nR);  // bL^dag v_1
                if (norm2(d) == 0.0) {
                    if (bL) {
                        ks->bdstep = 0;  // w_1^dag v_1 = 0: 2sL cannot start
                        ks->done = 1;
                        ks->kused = 0;
                    }
                } else {
                    ks->sw = c2d(cdiv(mk(1.0, 0.0), conj(d)));
                }
            }
        }
    }
}

void launch_deflate_split(const double2* b, const double2* R, const double2* L, const double2* lam, int m,
                          const double2* pq, double2* bR, double2* bL, double2* y, KState* ks, double2* vscale,
                          double* partials, unsigned int* counter, size_t n, cudaStream_t st) {
    k_deflate_split<<<grid_for(n, 256, 512), 256, sizeof(double2) * 3 * (m > 0 ? m : 1), st>>>(
        b, R, L, lam, m, pq, bR, bL, y, ks, vscale, partials, counter, n);
}

// -------------------------------------------------------------- conversions --
// v_1 = x / |x| (FP64, |x| = nR from the deflation split), optionally y += c[0] * v_1
__global__ void k_scale_start(const double2* __restrict__ x, double2* __restrict__ v, double2* __restrict__ y,
                              const double2* __restrict__ c, const KState* ks, size_t n) {
    if (ks->status || ks->nR == 0.0) return;
    const cx<double> sv = mk(1.0 / ks->nR, 0.0);
    const cx<double> c0 = c ? d2c(c[0]) : mk(0.0, 0.0);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const cx<double> z = sv * d2c(x[e]);
        v[e] = c2d(z);
        if (y) {
            cx<double> yy = d2c(y[e]);
            cfma(yy, c0, z);
            y[e] = c2d(yy);
        }
    }
}
void launch_scale_start(const double2* x, double2* v, double2* y, const double2* c, const KState* ks, size_t n,
                        cudaStream_t st) {
    k_scale_start<<<grid_for(n, 256, 1024), 256, 0, st>>>(x, v, y, c, ks, n);
}

// y += sum_{l < kused} c_l s_l V_l, s_l = vscale[l] (or 1)
__global__ void __launch_bounds__(256) k_combine(const double2* __restrict__ V, size_t ld,
                                                 const double2* __restrict__ vscale, const double2* __restrict__ c,
                                                 const KState* ks, double2* __restrict__ y, size_t n) {
    extern __shared__ double2 cf[];
    if (ks->status) return;
    const int nv = ks->kused;
    for (int l = threadIdx.x; l < nv; l += blockDim.x) {
        cx<double> z = d2c(c[l]);
        if (vscale) z = z * d2c(vscale[l]);
        cf[l] = c2d(z);
    }
    __syncthreads();
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        cx<double> z = d2c(y[e]);
        for (int l = 0; l < nv; ++l) {
            const double2 v = __ldg(V + (size_t)l * ld + e);
            const double2 q = cf[l];
            z.r += q.x * v.x - q.y * v.y;
            z.i += q.x * v.y + q.y * v.x;
        }
        y[e] = c2d(z);
    }
}
void launch_combine(const double2* V, size_t ld, const double2* vscale, const double2* c, const KState* ks,
                    int kmax, double2* y, size_t n, cudaStream_t st) {
    k_combine<<<grid_for(n, 256, 1024), 256, sizeof(double2) * (kmax > 0 ? kmax : 1), st>>>(V, ld, vscale, c, ks,
                                                                                            y, n);
}

}  // namespace ovl
