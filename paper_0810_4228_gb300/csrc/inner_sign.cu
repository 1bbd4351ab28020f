// The inner sign function c = |b_perp| sgn(G_k) e_1 of the projected k x k
// matrix (Sec. 2, Eq. 2.6 and the remark after it; Sec. 4, Eq. 4.4-4.5).
//
// Two methods, both FP64 and both driven entirely from device memory (the
// matrix size is the number of Krylov steps actually taken, read from the
// solve state), so they can be captured in a CUDA graph.
//
// (1) Resolvent quadrature, for the tridiagonal G_k of two-sided Lanczos.
//     For a matrix with no eigenvalue on the imaginary axis,
//         sgn(G) = (2/pi) int_0^inf G (G^2 + t^2)^-1 dt
//                = (1/pi) int_R e^u [(G + i e^u)^-1 + (G - i e^u)^-1] du,   t = e^u,
//     which reproduces sgn z = z / sqrt(z^2) (Sec. 1, Eq. 1.4) eigenvalue by
//     eigenvalue.  The u-integrand is analytic in a strip whose half-width is
//     the smallest angle between an eigenvalue and the imaginary axis, so the
//     trapezoidal rule converges geometrically.  Each node costs one
//     tridiagonal solve (Gaussian elimination with partial pivoting, O(k)),
//     one thread per node; the step is halved (reusing all earlier nodes)
//     until two successive sums agree.  Cost O(nodes * k) instead of the
//     O(k^3) per iteration of a dense matrix iteration; on this GPU FP64 runs
//     at 1/58 of the FP32 rate, which makes the difference decisive.
// (2) Roberts' iteration S <- (S + S^-1)/2, S^0 = G (Sec. 2), with
//     |det S|^(-1/n) scaling of the first iterates; the inverse by in-place
//     Gauss-Jordan elimination with partial pivoting in one cooperative kernel
//     (rows distributed over all SMs, bounded grid barriers).  Used for the
//     Hessenberg H_k of Arnoldi and on request for G_k.
#include <math.h>

#include "ovl_kernels.h"
#include "df32.cuh"

namespace ovl {

static constexpr double QUAD_H0 = 0.25;       // first trapezoid step in u
static constexpr double QUAD_HALFWIDTH = 40;  // u range: log|G| -+ 40 (tails below e^-40)
static constexpr int QUAD_LEVELS = 6;         // steps 0.25 ... 0.25/32

static int quad_nodes_level0() { return (int)ceil(2 * QUAD_HALFWIDTH / QUAD_H0); }
static int quad_threads(int level) {
    const int m0 = quad_nodes_level0();
    const int nodes = level == 0 ? m0 : m0 << (level - 1);
    return 2 * nodes;  // +- i e^u
}

// Offsets of sequence j in a batch of independent inner problems (zero for a single one): the
// coefficient arrays, output c, the solve state, the scratch and the reduction buffers of
// sequence j start at j times these strides.
struct QStride {
    size_t coef, work, part;
};

size_t inner_work_elems(int kmax, int method) {
    if (method == 0) {
        // per thread and row: 3 complex (b/d, u/d, w/d), plus T and S sums, plus the double-float
        // copies of alpha, beta, gamma
        return (size_t)quad_threads(QUAD_LEVELS - 1) * (size_t)kmax * 3 + 5 * (size_t)kmax + 64;
    }
    if (method == 2) {
        // Hessenberg quadrature: per thread and row x and the two rotation coefficients, T and S
        // sums, the double-float copy of H (kmax x kmax)
        return (size_t)quad_threads(QUAD_LEVELS - 1) * (size_t)kmax * 3 + 2 * (size_t)kmax + 64 +
               (size_t)kmax * kmax;
    }
    // Newton: S, X (kmax^2 each) + pivots, slots, scalars, barrier, partials
    return 2 * (size_t)kmax * kmax + 4 * (size_t)kmax + 8192;
}

// ---------------------------------------------------------- quadrature --
// log of a Gershgorin bound on |lambda_max(G)| -> ks->red[7].x
__global__ void k_quad_prep(const double2* alpha, const double2* beta, const double2* gamma, KState* ks,
                            double2* work, size_t coef_off, QStride qs) {
    __shared__ double red[32];
    {
        const size_t j = blockIdx.x;
        alpha += j * qs.coef;
        beta += j * qs.coef;
        gamma += j * qs.coef;
        ks += j;
        work += j * qs.work;
    }
    const int n = ks->kused;
    // double-float copies of the tridiagonal coefficients for the solves (dfc in the FP64 slots)
    dfc* cd = reinterpret_cast<dfc*>(work + coef_off);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        cd[i] = c2dfc(d2df(alpha[i]));
        cd[n + i] = c2dfc(d2df(beta[i]));
        cd[2 * n + i] = c2dfc(d2df(gamma[i]));
    }
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = hypot(alpha[i].x, alpha[i].y);
        if (i > 0) r += hypot(beta[i - 1].x, beta[i - 1].y);
        if (i + 1 < n) r += hypot(gamma[i].x, gamma[i].y);
        m = fmax(m, r);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
        ks->red[7] = make_double2(log(fmax(mm, 1e-300)), 0.0);
        ks->inner_done = 0;
        ks->inner_iters = 0;
        ks->inner_method = 0;
        ks->inner_err = 0.0;
        if (n == 0) ks->inner_done = 1;
    }
}

// Double-float complex helpers of the solves: conj, 1/z with a power-of-two scaling (the FP32
// exponent range of the hi parts: |z| reaches e^40 |G| at the quadrature's ends), |re| + |im|.
__device__ __forceinline__ cx<df> dconj(const cx<df>& z) { return mk(z.r, -z.i); }
__device__ __forceinline__ df df_scale(df a, float s) { return df(a.hi * s, a.lo * s); }  // exact (power of 2)
__device__ __forceinline__ df df_rcp(df a) {
    const df r0(__frcp_rn(a.hi), 0.f);
    const df e = df(1) - a * r0;  // one Newton step: r = r0 + r0 (1 - a r0)
    return r0 + r0 * e;
}
__device__ __forceinline__ cx<df> crcp(const cx<df>& z) {
    const float mx = fmaxf(fabsf(z.r.hi), fabsf(z.i.hi));
    int e;
    frexpf(mx, &e);
    const float sc = ldexpf(1.f, -e);
    const cx<df> zs = mk(df_scale(z.r, sc), df_scale(z.i, sc));
    const df inv = df_rcp(zs.r * zs.r + zs.i * zs.i);
    return mk(df_scale(zs.r * inv, sc), df_scale(-(zs.i * inv), sc));
}
__device__ __forceinline__ float cabs1f(const cx<df>& z) { return fabsf(z.r.hi) + fabsf(z.i.hi); }

// One thread per (node, sign): solve (G + s i e^u) x = e_1 by Gaussian elimination with partial
// pivoting (interchanging rows i and i+1 when |beta_i| > |d_i|), store e^u x in the scratch column
// of the thread (row-major over rows, thread fastest).  Double-float arithmetic (df32.cuh) on the
// FP32 pipe: a node's elimination is one dependent chain of complex operations per row, and
// GB300's FP64 unit would run each of them 64x slower; 48 significant bits keep the quadrature's
// 1e-14 accuracy.
__global__ void k_quad_solve(KState* ks, double2* __restrict__ work, size_t coef_off, int level, int nthreads,
                             QStride qs) {
    {
        const size_t j = blockIdx.y;
        ks += j;
        work += j * qs.work;
    }
    if (ks->inner_done || ks->status || ks->timeout) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    const int n = ks->kused;
    const dfc* ca = reinterpret_cast<const dfc*>(work + coef_off);
    const dfc* cb = ca + n;
    const dfc* cg = ca + 2 * n;
    const double lo = ks->red[7].x - QUAD_HALFWIDTH;
    const int node = t >> 1;
    const float sgn = (t & 1) ? -1.f : 1.f;
    double u;
    if (level == 0) {
        u = lo + node * QUAD_H0;
    } else {
        const double hl = QUAD_H0 / (double)(1 << level);
        u = lo + (2 * node + 1) * hl;
    }
    const df tau(exp(u));
    const cx<df> sig = mk(df(0), df(tau.hi * sgn, tau.lo * sgn));
    // arrays: bd = b/d, ud = u/d, wd = w/d of the final (upper triangular) rows
    dfc* bd = reinterpret_cast<dfc*>(work);
    dfc* ud = bd + (size_t)n * nthreads;
    dfc* wd = bd + 2 * (size_t)n * nthreads;
    const dfc zero = {0.f, 0.f, 0.f, 0.f};
#define IDX(i) ((size_t)(i) * nthreads + t)
    // current row i: (d, u) at (i, i+1), rhs rb
    cx<df> d = dfc2c(ca[0]) + sig;
    cx<df> uu = n > 1 ? dfc2c(cg[0]) : mk(df(0), df(0));
    cx<df> rb = mk(df(1), df(0));
    for (int i = 0; i + 1 < n; ++i) {
        const cx<df> l = dfc2c(cb[i]);                  // row i+1, column i
        const cx<df> dn = dfc2c(ca[i + 1]) + sig;       // row i+1, column i+1
        const cx<df> un = (i + 2 < n) ? dfc2c(cg[i + 1]) : mk(df(0), df(0));
        if (cabs1f(d) >= cabs1f(l)) {
            // no interchange: final row i = (d, uu, 0)
            const cx<df> id = crcp(d);
            const cx<df> m = l * id;
            bd[IDX(i)] = c2dfc(rb * id);
            ud[IDX(i)] = c2dfc(uu * id);
            wd[IDX(i)] = zero;
            d = dn - m * uu;
            uu = un;
            rb = -(m * rb);  // rhs of row i+1 is 0 for e_1 beyond row 0
        } else {
            // interchange rows i and i+1: final row i = (l, dn, un), rhs 0
            const cx<df> il = crcp(l);
            const cx<df> m = d * il;
            bd[IDX(i)] = zero;
            ud[IDX(i)] = c2dfc(dn * il);
            wd[IDX(i)] = c2dfc(un * il);
            const cx<df> nd = uu - m * dn;
            uu = -(m * un);
            d = nd;
            // new rhs of row i+1: rb (old row i) - m * 0
        }
    }
    if (d.r.hi == 0.f && d.i.hi == 0.f) {
        atomicExch(&ks->status, 5);  // singular shifted matrix
        return;
    }
    // back substitution, x overwrites bd
    cx<df> x1 = rb * crcp(d), x2 = mk(df(0), df(0));
    bd[IDX(n - 1)] = c2dfc(mk(tau * x1.r, tau * x1.i));
    for (int i = n - 2; i >= 0; --i) {
        const cx<df> x = dfc2c(bd[IDX(i)]) - dfc2c(ud[IDX(i)]) * x1 - dfc2c(wd[IDX(i)]) * x2;
        bd[IDX(i)] = c2dfc(mk(tau * x.r, tau * x.i));
        x2 = x1;
        x1 = x;
    }
#undef IDX
}

// T_l = (l == 0 ? 0 : T_{l-1}/2) + (h_l/pi) sum_threads x ; convergence on |T_l - T_{l-1}|.
__global__ void k_quad_sum(const double2* __restrict__ work, double2* __restrict__ T, double2* __restrict__ c,
                           KState* ks, int level, int nthreads, double* partials, unsigned int* counter, QStride qs) {
    __shared__ double red[96];
    {
        const size_t j = blockIdx.y;
        work += j * qs.work;
        T += j * qs.work;
        c += j * qs.coef;
        ks += j;
        partials += j * qs.part;
        counter += j;
    }
    if (ks->inner_done || ks->status || ks->timeout) return;
    const int n = ks->kused;
    const double hl = QUAD_H0 / (double)(1 << level);
    const double wgt = hl / M_PI;
    double part[2] = {0.0, 0.0};  // |T_l - T_{l-1}|^2, |T_l|^2
    // one warp per row i
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = blockIdx.x * nw + wid; i < n; i += gridDim.x * nw) {
        // double-float sums of the solves' double-float outputs (all nodes; even nodes, step 2h)
        df dsr(0), dsi(0), der(0), dei(0);
        const dfc* wk = reinterpret_cast<const dfc*>(work);
        for (int t = lane; t < nthreads; t += 32) {
            const cx<df> v = dfc2c(wk[(size_t)i * nthreads + t]);
            dsr = df_add_lazy(dsr, v.r);
            dsi = df_add_lazy(dsi, v.i);
            if (((t >> 1) & 1) == 0) {
                der = df_add_lazy(der, v.r);
                dei = df_add_lazy(dei, v.i);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            dsr = dsr + df(__shfl_xor_sync(0xffffffffu, dsr.hi, o), __shfl_xor_sync(0xffffffffu, dsr.lo, o));
            dsi = dsi + df(__shfl_xor_sync(0xffffffffu, dsi.hi, o), __shfl_xor_sync(0xffffffffu, dsi.lo, o));
            der = der + df(__shfl_xor_sync(0xffffffffu, der.hi, o), __shfl_xor_sync(0xffffffffu, der.lo, o));
            dei = dei + df(__shfl_xor_sync(0xffffffffu, dei.hi, o), __shfl_xor_sync(0xffffffffu, dei.lo, o));
        }
        const double sr = dsr.to_double(), si = dsi.to_double(), er = der.to_double(), ei = dei.to_double();
        if (lane == 0) {
            // level 0 compares with the trapezoid sum of step 2h over its even nodes
            double2 old = level == 0 ? make_double2(2.0 * wgt * er, 2.0 * wgt * ei) : T[i];
            double2 nt = make_double2((level == 0 ? 0.0 : 0.5 * old.x) + wgt * sr,
                                      (level == 0 ? 0.0 : 0.5 * old.y) + wgt * si);
            // (at level 0 `old` is the 2h estimate, not a previous level)
            T[i] = nt;
            const double nr = ks->nR;
            c[i] = make_double2(nr * nt.x, nr * nt.y);
            part[0] += (nt.x - old.x) * (nt.x - old.x) + (nt.y - old.y) * (nt.y - old.y);
            part[1] += nt.x * nt.x + nt.y * nt.y;
        }
    }
    double out[2];
    if (grid_sum_last<2>(part, partials, counter, out, red)) {
        if (threadIdx.x == 0) {
            const double diff = sqrt(out[0]), nrm = sqrt(out[1]);
            ks->inner_iters += nthreads;
            // geometric convergence: the error of T_l is about (diff/|T|)^2
            const double rel = diff / fmax(nrm, 1e-300);
            ks->inner_err = rel * rel;
            if (rel <= 1e-7) ks->inner_done = 1;
            if (level == QUAD_LEVELS - 1 && !ks->inner_done) ks->status = 6;  // no convergence
        }
    }
}

static void quad_launch(const double2* alpha, const double2* beta, const double2* gamma, KState* ks, double2* c,
                        double2* work, int kmax, double* partials, unsigned int* counter, int nseq, QStride qs,
                        cudaStream_t st) {
    const int tmax = quad_threads(QUAD_LEVELS - 1);
    double2* T = work + (size_t)tmax * kmax * 3;
    const size_t coef_off = (size_t)tmax * kmax * 3 + 2 * (size_t)kmax + 64;
    k_quad_prep<<<nseq, 256, 0, st>>>(alpha, beta, gamma, ks, work, coef_off, qs);
    for (int level = 0; level < QUAD_LEVELS; ++level) {
        const int nt = quad_threads(level);
        k_quad_solve<<<dim3((nt + 31) / 32, nseq), 32, 0, st>>>(ks, work, coef_off, level, nt, qs);
        int blocks = (kmax + 7) / 8;
        if (blocks > 256) blocks = 256;
        k_quad_sum<<<dim3(blocks, nseq), 256, 0, st>>>(work, T, c, ks, level, nt, partials, counter, qs);
    }
}

int launch_inner_quadrature(const double2* alpha, const double2* beta, const double2* gamma, KState* ks,
                            double2* c, double2* work, size_t work_elems, int kmax, double* partials,
                            unsigned int* counter, cudaStream_t st) {
    if (inner_work_elems(kmax, 0) > work_elems) return -1;
    quad_launch(alpha, beta, gamma, ks, c, work, kmax, partials, counter, 1, QStride{0, 0, 0}, st);
    return 0;
}

int launch_inner_quadrature_batched(int nseq, const double2* alpha, const double2* beta, const double2* gamma,
                                    KState* ks, double2* c, size_t coef_stride, double2* work, size_t work_stride,
                                    int kmax, double* partials, size_t part_stride, unsigned int* counters,
                                    cudaStream_t st) {
    if (inner_work_elems(kmax, 0) > work_stride || nseq < 1) return -1;
    quad_launch(alpha, beta, gamma, ks, c, work, kmax, partials, counters, nseq,
                QStride{coef_stride, work_stride, part_stride}, st);
    return 0;
}

// ------------------------------------------------- Hessenberg quadrature --
// The same trapezoidal rule for the upper Hessenberg H_k of Arnoldi (Sec. 2, Eq. 2.6).  Each node
// needs x = M^-1 e_1 for M = H + s i e^u.  Givens rotations applied to pairs of columns from the
// right, (k-2, k-1) first and (0, 1) last, each annihilating one subdiagonal entry, reduce M to
// upper triangular form: M Q = R.  Then M x = e_1 gives R (Q^dag x) = e_1, and since R is upper
// triangular, Q^dag x = e_1 / R_00, i.e.  x = Q e_1 / R_00.  So the sweep needs only the
// rotations and R_00: it carries one column (the one being rotated next) instead of the
// triangular factor, O(k^2) operations and O(k) memory per node.  Rotations are unitary, so the
// solve is backward stable without pivoting.  With the rotation on columns (j, j+1) written as
// G = [[b, conj(a)], [-a, conj(b)]] / rho (a, b the row-(j+1) entries of column j and of the carried
// column, rho = sqrt(|a|^2 + |b|^2)), Q e_1 has components x_j = p_j b_j / rho_j (j < k-1) and
// x_{k-1} = p_{k-1}, with p_0 = 1 and p_{j+1} = -p_j a_j / rho_j.
//
// One warp per (node, sign), its carried column in shared memory, double-float arithmetic.

// log of the Frobenius norm of H (a bound on its spectral radius) -> ks->red[7].x; H -> double-float
__global__ void __launch_bounds__(256) k_hess_prep(const double2* __restrict__ H, int ldH, KState* ks,
                                                   dfc* __restrict__ Hd, int ldd, double* partials,
                                                   unsigned int* counter) {
    __shared__ double red[32];
    if (ks->status || ks->timeout) return;
    const int n = ks->kused;
    double part[1] = {0.0};
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const int rmax = j + 1 < n - 1 ? j + 1 : n - 1;  // column j: rows 0..j+1
        for (int r = threadIdx.x; r <= rmax; r += blockDim.x) {
            const double2 v = H[r + (size_t)j * ldH];
            Hd[r + (size_t)j * ldd] = c2dfc(d2df(v));
            part[0] += v.x * v.x + v.y * v.y;
        }
    }
    double out[1];
    if (grid_sum_last<1>(part, partials, counter, out, red)) {
        if (threadIdx.x == 0) {
            ks->red[7] = make_double2(log(fmax(sqrt(out[0]), 1e-300)), 0.0);
            ks->inner_done = (n == 0);
            ks->inner_iters = 0;
            ks->inner_method = 0;
            ks->inner_err = 0.0;
        }
    }
}

__device__ __forceinline__ cx<df> cscale(const cx<df>& z, float s) { return mk(df_scale(z.r, s), df_scale(z.i, s)); }
// 1 / sqrt(x) for x in [1/4, 8): one Newton step y + y (1 - x y^2) / 2 from the FP32 estimate
__device__ __forceinline__ df df_rsqrt(df x) {
    const df y0(rsqrtf(x.hi), 0.f);
    const df e = df(1) - x * y0 * y0;
    return y0 + df_scale(y0 * e, 0.5f);
}
// (ca, cb) = (a, b) / sqrt(|a|^2 + |b|^2), scaled by a power of two first (FP32 exponent range)
__device__ __forceinline__ void givens_df(const cx<df>& a, const cx<df>& b, cx<df>& ca, cx<df>& cb) {
    const float mx = fmaxf(fmaxf(fabsf(a.r.hi), fabsf(a.i.hi)), fmaxf(fabsf(b.r.hi), fabsf(b.i.hi)));
    if (mx == 0.f) {  // row already zero in both columns: identity
        ca = mk(df(0), df(0));
        cb = mk(df(1), df(0));
        return;
    }
    int e;
    frexpf(mx, &e);
    const float sc = ldexpf(1.f, -e);
    const cx<df> as = cscale(a, sc), bs = cscale(b, sc);
    const df nn = (as.r * as.r + as.i * as.i) + (bs.r * bs.r + bs.i * bs.i);
    const df ri = df_rsqrt(nn);
    ca = mk(as.r * ri, as.i * ri);
    cb = mk(bs.r * ri, bs.i * ri);
}
// cb h - ca c, each component one sum of four double-float products
__device__ __forceinline__ cx<df> rot_combine(const cx<df>& cb, const cx<df>& h, const cx<df>& ca, const cx<df>& c) {
    dfacc re, im;
    dfacc_first(re, cb.r, h.r, false);
    dfacc_add(re, cb.i, h.i, true);
    dfacc_add(re, ca.r, c.r, true);
    dfacc_add(re, ca.i, c.i, false);
    dfacc_first(im, cb.r, h.i, false);
    dfacc_add(im, cb.i, h.r, false);
    dfacc_add(im, ca.r, c.i, true);
    dfacc_add(im, ca.i, c.r, true);
    return mk(dfacc_value(re), dfacc_value(im));
}
__device__ __forceinline__ cx<df> shfl_cdf(const cx<df>& z, int src) {
    return mk(df(__shfl_sync(0xffffffffu, z.r.hi, src), __shfl_sync(0xffffffffu, z.r.lo, src)),
              df(__shfl_sync(0xffffffffu, z.i.hi, src), __shfl_sync(0xffffffffu, z.i.lo, src)));
}

static constexpr int HQ_WPB_MAX = 4;  // warps (nodes) per block

__global__ void k_hess_solve(KState* ks, double2* __restrict__ work, size_t hoff, int ldd, int kmax, int level,
                             int nthreads) {
    extern __shared__ float4 hq_col[];
    if (ks->inner_done || ks->status || ks->timeout) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int t = blockIdx.x * (blockDim.x >> 5) + wid;
    if (t >= nthreads) return;  // whole warps
    const int n = ks->kused;
    const dfc* Hd = reinterpret_cast<const dfc*>(work + hoff);
    float4* col = hq_col + (size_t)wid * kmax;
    const double lo = ks->red[7].x - QUAD_HALFWIDTH;
    const int node = t >> 1;
    const float sgn = (t & 1) ? -1.f : 1.f;
    const double u = level == 0 ? lo + node * QUAD_H0 : lo + (2 * node + 1) * (QUAD_H0 / (double)(1 << level));
    const df tau(exp(u));
    const cx<df> sig = mk(df(0), df(tau.hi * sgn, tau.lo * sgn));
    dfc* X = reinterpret_cast<dfc*>(work);
    dfc* CA = X + (size_t)n * nthreads;
    dfc* CB = X + 2 * (size_t)n * nthreads;
#define IDX(i) ((size_t)(i) * nthreads + t)
    // carried column: column n-1 of M
    for (int r = lane; r < n; r += 32) {
        cx<df> h = dfc2c(Hd[r + (size_t)(n - 1) * ldd]);
        if (r == n - 1) h = h + sig;
        col[r] = make_float4(h.r.hi, h.r.lo, h.i.hi, h.i.lo);
    }
    __syncwarp();
    for (int i = n - 1; i >= 1; --i) {
        // rotate columns (i-1, i): a = M[i, i-1] (subdiagonal, unshifted), b = carried M[i, i]
        const cx<df> a = dfc2c(Hd[i + (size_t)(i - 1) * ldd]);
        const float4 bv = col[i];
        const cx<df> b = mk(df(bv.x, bv.y), df(bv.z, bv.w));
        cx<df> ca, cb;
        givens_df(a, b, ca, cb);
        if (lane == 0) {
            CA[IDX(i - 1)] = c2dfc(ca);
            CB[IDX(i - 1)] = c2dfc(cb);
        }
        // new carried column (column i-1 after the rotation), rows 0..i-1; its row i is zero
        for (int r = lane; r < i; r += 32) {
            cx<df> h = dfc2c(Hd[r + (size_t)(i - 1) * ldd]);
            if (r == i - 1) h = h + sig;
            const float4 cv = col[r];
            const cx<df> z = rot_combine(cb, h, ca, mk(df(cv.x, cv.y), df(cv.z, cv.w)));
            col[r] = make_float4(z.r.hi, z.r.lo, z.i.hi, z.i.lo);
        }
        __syncwarp();
    }
    const float4 r0 = col[0];
    const cx<df> R00 = mk(df(r0.x, r0.y), df(r0.z, r0.w));
    if (R00.r.hi == 0.f && R00.i.hi == 0.f) {
        if (lane == 0) atomicExch(&ks->status, 5);  // singular shifted matrix
        return;
    }
    __syncwarp();  // CA, CB written by lane 0 are read by every lane below
    const cx<df> ir = crcp(R00);
    const cx<df> s0 = mk(tau * ir.r, tau * ir.i);  // e^u / R_00
    // p_j = prod_{l < j} (-a_l / rho_l): segments of the rotation list per lane, then an exclusive
    // scan of the segment products across the warp
    const int nr = n - 1;  // rotations
    const int seg = (nr + 31) / 32;
    const int j0 = lane * seg, j1 = min(nr, j0 + seg);
    cx<df> pr = mk(df(1), df(0));
    for (int j = j0; j < j1; ++j) pr = pr * (-dfc2c(CA[IDX(j)]));
    // inclusive scan (Hillis-Steele): pr becomes the product of the segments of lanes 0..lane
    for (int o = 1; o < 32; o <<= 1) {
        const cx<df> other = shfl_cdf(pr, (lane - o) & 31);
        if (lane >= o) pr = other * pr;
    }
    // exclusive prefix: the inclusive product of the previous lane
    cx<df> p = shfl_cdf(pr, (lane - 1) & 31);
    if (lane == 0) p = mk(df(1), df(0));
    for (int j = j0; j < j1; ++j) {
        const cx<df> x = p * dfc2c(CB[IDX(j)]) * s0;
        X[IDX(j)] = c2dfc(x);
        p = p * (-dfc2c(CA[IDX(j)]));
    }
    // x_{n-1} = p_{n-1} / R_00: p after the last rotation (the lane holding it, or lane 0 if n = 1)
    const int last = nr > 0 ? (nr - 1) / seg : 0;
    if (lane == last) X[IDX(n - 1)] = c2dfc((nr > 0 ? p : mk(df(1), df(0))) * s0);
#undef IDX
}

static void hess_quad_launch(const double2* H, int ldH, KState* ks, double2* c, double2* work, int kmax,
                             double* partials, unsigned int* counter, cudaStream_t st) {
    const int tmax = quad_threads(QUAD_LEVELS - 1);
    double2* T = work + (size_t)tmax * kmax * 3;
    const size_t hoff = (size_t)tmax * kmax * 3 + 2 * (size_t)kmax + 64;
    int pb = (kmax + 7) / 8;
    if (pb > 1024) pb = 1024;
    k_hess_prep<<<pb, 256, 0, st>>>(H, ldH, ks, reinterpret_cast<dfc*>(work + hoff), kmax, partials, counter);
    const size_t per_warp = sizeof(float4) * (size_t)kmax;
    int wpb = (int)((96u * 1024u) / per_warp);
    if (wpb > HQ_WPB_MAX) wpb = HQ_WPB_MAX;
    if (wpb < 1) wpb = 1;
    const size_t smem = per_warp * wpb;
    // the limit needed grows with kmax: kept per device (the attribute is per device)
    static size_t smem_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (smem > 48 * 1024 && smem > smem_set[dev]) {
        if (cudaFuncSetAttribute(k_hess_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
            smem_set[dev] = smem;
    }
    for (int level = 0; level < QUAD_LEVELS; ++level) {
        const int nt = quad_threads(level);
        k_hess_solve<<<(nt + wpb - 1) / wpb, 32 * wpb, smem, st>>>(ks, work, hoff, kmax, kmax, level, nt);
        int blocks = (kmax + 7) / 8;
        if (blocks > 256) blocks = 256;
        k_quad_sum<<<dim3(blocks, 1), 256, 0, st>>>(work, T, c, ks, level, nt, partials, counter, QStride{0, 0, 0});
    }
}

int launch_inner_quadrature_hess(const double2* H, int ldH, KState* ks, double2* c, double2* work,
                                 size_t work_elems, int kmax, double* partials, unsigned int* counter,
                                 cudaStream_t st) {
    if (inner_work_elems(kmax, 2) > work_elems) return -1;
    if ((size_t)kmax * sizeof(float4) > 200u * 1024u) return -1;  // carried column beyond shared memory
    hess_quad_launch(H, ldH, ks, c, work, kmax, partials, counter, st);
    return 0;
}

// --------------------------------------------------------------- Newton --
struct NewtonWork {
    double2* S;            // n x n (ld kmax), current iterate
    double2* X;            // n x n, inverse workspace
    int* pivrow;           // kmax
    int* invr;             // kmax
    unsigned long long* slot;  // kmax + 1
    double* scal;          // [0] logdet, [1] mu, [2] diff2, [3] norm2, [4] final flag
    unsigned int* bar;     // grid barrier (count, generation)
    unsigned int* counter;
    double* partials;
};

static NewtonWork newton_layout(double2* work, int kmax) {
    NewtonWork w;
    w.S = work;
    w.X = work + (size_t)kmax * kmax;
    char* p = reinterpret_cast<char*>(work + 2 * (size_t)kmax * kmax);
    w.pivrow = reinterpret_cast<int*>(p);
    p += sizeof(int) * kmax;
    w.invr = reinterpret_cast<int*>(p);
    p += sizeof(int) * kmax;
    p = reinterpret_cast<char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    w.slot = reinterpret_cast<unsigned long long*>(p);
    p += sizeof(unsigned long long) * (kmax + 1);
    w.scal = reinterpret_cast<double*>(p);
    p += sizeof(double) * 8;
    w.bar = reinterpret_cast<unsigned int*>(p);
    p += 16;
    w.counter = reinterpret_cast<unsigned int*>(p);
    p += 16;
    w.partials = reinterpret_cast<double*>(p);
    return w;
}

__device__ __forceinline__ unsigned long long pivkey(double mag, int row) {
    // non-negative float bits are monotone; ties prefer the smaller row
    const float f = (float)mag;
    return ((unsigned long long)__float_as_uint(f) << 32) | (unsigned long long)(0x7fffffff - row);
}

// Roberts' iteration in one cooperative kernel: every iteration copies S to X,
// inverts X in place by Gauss-Jordan elimination with partial pivoting (rows
// owned cyclically by the blocks, the pivot row chosen at step p is pivrow[p],
// S^-1[a][b] = X[pivrow[a]][invr[b]]), then S <- (mu S + S^-1 / mu) / 2 with
// |det S|^(-1/n) scaling of the first iterates.  All blocks add the per-block
// partial sums in the same order, so they take the same convergence decision.
// With `fallback` the kernel only runs when the quadrature did not converge.
__global__ void __launch_bounds__(256) k_newton_coop(const double2* alpha, const double2* beta,
                                                     const double2* gamma, const double2* H, int ldH, int tri,
                                                     KState* ks, NewtonWork w, double2* c, int kmax, int max_it,
                                                     int fallback) {
    extern __shared__ double2 prow[];
    __shared__ unsigned long long best;
    __shared__ double red[2 * 32];  // block_sum<2>: 32 doubles per value
    const long long max_spins = 20000000;
    int* err = &ks->timeout;
    // uniform entry decision (all blocks read the same state before anyone writes it)
    const int st0 = ks->status;
    const int done0 = ks->inner_done;
    if (ks->timeout) return;
    if (fallback) {
        if (done0 || (st0 != 0 && st0 != 6)) return;
    } else if (st0) {
        return;
    }
    const int n = ks->kused;
    const int G = gridDim.x;
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
    grid_barrier(w.bar, err, 1, max_spins);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ks->status = 0;
        ks->inner_done = (n == 0);
        ks->inner_iters = 0;
        ks->inner_method = 1;
        ks->inner_err = 0.0;
    }
    if (n == 0) return;
    // rows are owned by block (row % G) for S and X alike, so a block only reads rows
    // written by other blocks (the pivot row, the scrambled inverse) through L2
    for (int r = blockIdx.x; r < n; r += G)
        for (int cI = threadIdx.x; cI < n; cI += blockDim.x) {
            double2 v = make_double2(0.0, 0.0);
            if (tri) {
                if (r == cI) v = alpha[r];
                else if (r == cI + 1) v = beta[cI];
                else if (cI == r + 1) v = gamma[r];
            } else if (r <= cI + 1) {
                v = H[r + (size_t)cI * ldH];  // column-major Hessenberg; zero below the subdiagonal
            }
            w.S[(size_t)r * kmax + cI] = v;
        }
    bool fin = false;   // the extra unscaled step after convergence is pending
    bool conv = false;
    int it = 0;
    for (; it < max_it && !conv; ++it) {
        // X = S, clear the pivot bookkeeping (own rows)
        for (int r = blockIdx.x; r < n; r += G) {
            for (int cI = threadIdx.x; cI < n; cI += blockDim.x)
                w.X[(size_t)r * kmax + cI] = w.S[(size_t)r * kmax + cI];
            if (threadIdx.x == 0) w.invr[r] = -1;
        }
        for (size_t e = tid; e <= (size_t)n; e += nth) w.slot[e] = 0ull;
        if (tid == 0) w.scal[0] = 0.0;
        grid_barrier(w.bar, err, 1, max_spins);
        if (*(volatile int*)err) return;
        // candidate pivot of column 0
        if (threadIdx.x == 0) {
            best = 0ull;
            for (int r = blockIdx.x; r < n; r += G) {
                const double2 v = __ldcg(w.X + (size_t)r * kmax);
                const unsigned long long k = pivkey(hypot(v.x, v.y), r);
                if (k > best) best = k;
            }
            if (best) atomicMax(&w.slot[0], best);
        }
        grid_barrier(w.bar, err, 1, max_spins);
        if (*(volatile int*)err) return;
        for (int p = 0; p < n; ++p) {
            const unsigned long long key = __ldcg(&w.slot[p]);
            const int r = key ? 0x7fffffff - (int)(key & 0xffffffffull) : -1;
            if (r < 0 || r >= n) {  // cannot happen for p < n: report, never index
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ks->status, 5);
                return;
            }
            // phase A: the owner scales the pivot row in place
            if (r % G == (int)blockIdx.x) {
                const double2 pv = w.X[(size_t)r * kmax + p];
                const cx<double> ip = cdiv(mk(1.0, 0.0), d2c(pv));
                __syncthreads();
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    if (j == p) w.X[(size_t)r * kmax + j] = c2d(ip);
                    else w.X[(size_t)r * kmax + j] = c2d(ip * d2c(w.X[(size_t)r * kmax + j]));
                }
                if (threadIdx.x == 0) {
                    w.pivrow[p] = r;
                    w.invr[r] = p;
                    const double am = hypot(pv.x, pv.y);
                    if (am == 0.0) atomicExch(&ks->status, 5);
                    atomicAdd(&w.scal[0], log(am));
                }
            }
            grid_barrier(w.bar, err, 1, max_spins);
            if (*(volatile int*)err) return;
            for (int j = threadIdx.x; j < n; j += blockDim.x) prow[j] = __ldcg(w.X + (size_t)r * kmax + j);
            if (threadIdx.x == 0) best = 0ull;
            __syncthreads();
            const cx<double> pp = d2c(prow[p]);
            for (int i = blockIdx.x; i < n; i += G) {
                if (i == r) continue;
                const cx<double> f = d2c(w.X[(size_t)i * kmax + p]);
                const bool cand = (p + 1 < n) && (__ldcg(w.invr + i) < 0);
                __syncthreads();  // every thread has read X[i][p] before it is overwritten
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    cx<double> x;
                    if (j == p) x = mk(0.0, 0.0) - f * pp;
                    else x = d2c(w.X[(size_t)i * kmax + j]) - f * d2c(prow[j]);
                    w.X[(size_t)i * kmax + j] = c2d(x);
                    if (j == p + 1 && cand) atomicMax(&best, pivkey(hypot(x.r, x.i), i));
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && best && p + 1 < n) atomicMax(&w.slot[p + 1], best);
            grid_barrier(w.bar, err, 1, max_spins);
            if (*(volatile int*)err) return;
        }
        // update S and the partial sums of |S_new - S|^2, |S_new|^2
        const bool scale = it < 8 && !fin;
        const double mu = scale ? exp(-__ldcg(&w.scal[0]) / n) : 1.0;
        double d2 = 0.0, n2 = 0.0;
        for (int aa = blockIdx.x; aa < n; aa += G) {
            const int pr = __ldcg(w.pivrow + aa);
            for (int bb = threadIdx.x; bb < n; bb += blockDim.x) {
                const cx<double> sv = d2c(w.S[(size_t)aa * kmax + bb]);
                const cx<double> xi = d2c(__ldcg(w.X + (size_t)pr * kmax + __ldcg(w.invr + bb)));
                const cx<double> ns = mk(0.5 * (mu * sv.r + xi.r / mu), 0.5 * (mu * sv.i + xi.i / mu));
                w.S[(size_t)aa * kmax + bb] = c2d(ns);
                d2 += norm2(ns - sv);
                n2 += norm2(ns);
            }
        }
        double v2[2] = {d2, n2};
        block_sum<2>(v2, red);
        if (threadIdx.x == 0) {
            w.partials[2 * blockIdx.x] = v2[0];
            w.partials[2 * blockIdx.x + 1] = v2[1];
        }
        grid_barrier(w.bar, err, 1, max_spins);
        if (*(volatile int*)err) return;
        __shared__ double sdn[2];
        {
            const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
            if (wq < 2) {
                double acc = 0.0;
                for (int bk = lane; bk < G; bk += 32) acc += __ldcg(w.partials + 2 * bk + wq);
                acc = warp_sum(acc);
                if (lane == 0) sdn[wq] = acc;
            }
            __syncthreads();
        }
        const double sd = sdn[0], sn = sdn[1];
        const double diff = sqrt(sd), nrm = sqrt(sn);
        if (fin) conv = true;                  // the extra unscaled step after convergence
        else if (diff <= 1e-7 * nrm) fin = true;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ks->inner_iters = it + 1;
            ks->inner_err = diff / fmax(nrm, 1e-300);
        }
        grid_barrier(w.bar, err, 1, max_spins);  // nobody rewrites X or the partials before all read them
        if (*(volatile int*)err) return;
    }
    for (size_t i = tid; i < (size_t)n; i += nth) {
        const double2 sv = __ldcg(w.S + i * kmax);
        c[i] = make_double2(ks->nR * sv.x, ks->nR * sv.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (conv) ks->inner_done = 1;
        else ks->status = 6;
    }
}

__global__ void k_newton_bar_reset(NewtonWork w) {
    w.bar[0] = 0u;
    w.bar[1] = 0u;
}

int launch_inner_newton(const double2* alpha, const double2* beta, const double2* gamma, const double2* H, int ldH,
                        int tri, KState* ks, double2* c, double2* work, size_t work_elems, int kmax, int num_sms,
                        cudaStream_t st, int fallback) {
    if (inner_work_elems(kmax, 1) > work_elems) return -1;
    NewtonWork w = newton_layout(work, kmax);
    const int max_it = 40;
    const size_t smem = sizeof(double2) * kmax;
    static unsigned long long attr_dev = 0;
    if (first_use_on_device(attr_dev))
        cudaFuncSetAttribute(k_newton_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k_newton_bar_reset<<<1, 1, 0, st>>>(w);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(num_sms);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_newton_coop, alpha, beta, gamma, H, ldH, tri, ks, w, c, kmax, max_it,
                                       fallback);
    return (int)e;
}

}  // namespace ovl
