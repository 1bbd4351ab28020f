// Derivatives of l = Re <g, y>, y = sgn(A) b, A = gamma5 D_w(mu; U) (Sec. 1, Eq. 1.2 and Eq. 1.3),
// with respect to the links U, the chemical potential mu and the source b, for any upstream
// gradient g = g_y.  Gradients follow PyTorch's convention for complex tensors: for real l and
// complex z, g_z = dl/dRe z + i dl/dIm z, so dl = Re <g_z, dz>, <a, b> = a^dag b.
//
// The derivative of the exact function is used.  With the resolvent form of sgn that the inner
// solve also uses, sgn(A) = (1/pi) int e^u sum_+- (A +- i e^u)^-1 du, its Frechet derivative is
//   L(A, E) = -(1/pi) int e^u sum_+- R_+- E R_+- du,  R_+- = (A +- i e^u)^-1,
// so for a parameter theta of A (E = dA/dtheta)
//   dl/dtheta = Re <g, L(A, E) b> = -(1/pi) int e^u sum_+- Re <R_+-^dag g, E R_+- b> du.
// One two-sided Lanczos process (Sec. 4, Eq. 4.2) started from v_1 = b / |b| and
// w_1 = g / conj(g^dag v_1) spans K_k(A, b) and K_k(A^dag, g), with W^dag V = 1 and
// A V = V G + ..., A^dag W = W G^dag + ..., so
//   R_s b ~ |b| V a_s,  a_s = (G + s i e^u)^-1 e_1,   R_s^dag g ~ zeta W d_s,  d_s = (G^dag - s i e^u)^-1 e_1,
// zeta = v_1^dag g, and
//   dl/dtheta = Re sum_pq M_pq <w_p, E v_q>,  M_pq = -(|b| conj(zeta)/pi) int e^u sum_s conj(d_s,p) a_s,q du.
// With Z_q = sum_p conj(M_pq) w_p this is sum_q Re <Z_q, E v_q>: the link force of the pairs
// (v_q, Z_q) (the adjoint of y = A x, as in grad.cu) and their mu derivative.  The same process
// gives y ~ |b| V sgn(G) e_1 and g_b = sgn(A)^dag g ~ zeta W sgn(G^dag) e_1,
// sgn(G^dag) e_1 = (1/pi) int e^u sum_s d_s du.  The u integrals use the trapezoid rule with the
// step halved until M settles; every node costs two tridiagonal solves of size k.
//
// The approximations converge like those of two-sided Lanczos for bilinear forms
// w^dag f(A) b.  The bases V, W (k + 1 vectors each) stay resident in device memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "df32.cuh"
#include "stencil_impl.cuh"

namespace ovl {
namespace {

constexpr int GT = 128;  // threads per block of the site kernels
constexpr int TADJ_LEVELS = 7;
constexpr double TADJ_H0 = 0.25;
constexpr double TADJ_HALFWIDTH = 40.0;

__device__ __forceinline__ cx<double> ld(const double2* p, size_t e) { return d2c(p[e]); }

// Start: v~_1 = b, w~_1 = g, y = 0; scales sv = 1/|b|, sw = 1/conj(g^dag v_1); zeta = v_1^dag g.
// A vanishing b ends the process (kused = 0); g^dag v_1 = 0 is a breakdown at step 0.
__global__ void __launch_bounds__(256) k_bilinear_start(const double2* __restrict__ b, const double2* __restrict__ g,
                                                        double2* __restrict__ v0, double2* __restrict__ w0,
                                                        double2* __restrict__ y, KState* ks, double2* vscale,
                                                        double2* wscale, double2* zeta, double* partials,
                                                        unsigned int* counter, size_t n) {
    __shared__ double red[128];
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const cx<double> bv = ld(b, e), gv = ld(g, e);
        v0[e] = b[e];
        w0[e] = g[e];
        y[e] = make_double2(0.0, 0.0);
        part[0] += norm2(bv);
        part[1] += norm2(gv);
        const cx<double> z = cdot(bv, gv);  // b^dag g
        part[2] += z.r;
        part[3] += z.i;
    }
    double out[4];
    if (grid_sum_last<4>(part, partials, counter, out, red) && threadIdx.x == 0) {
        const double nb = sqrt(out[0]), ng = sqrt(out[1]);
        ks->nR = nb;
        if (nb == 0.0) {
            ks->done = 1;
            ks->kused = 0;
            *zeta = make_double2(0.0, 0.0);
            return;
        }
        const cx<double> zt = mk(out[2] / nb, out[3] / nb);  // v_1^dag g
        *zeta = c2d(zt);
        ks->sv = make_double2(1.0 / nb, 0.0);
        vscale[0] = ks->sv;
        if (sqrt(norm2(zt)) <= 1e-10 * ng || ng == 0.0) {
            ks->bdstep = 0;  // w_1^dag v_1 = 0: the process cannot start
            ks->done = 1;
            ks->kused = 0;
        } else {
            ks->sw = c2d(cdiv(mk(1.0, 0.0), zt));  // 1 / conj(g^dag v_1)
            wscale[0] = ks->sw;
        }
    }
}

// scales of the stored w~: w_{i+1} = w~_{i+1} / conj(gamma_i)
__global__ void k_wscale(const double2* gamma, const KState* ks, double2* wscale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= ks->kused) return;
    wscale[i + 1] = c2d(cdiv(mk(1.0, 0.0), conj(d2c(gamma[i]))));
}

// Gershgorin bound of G -> scal[0] = log bound
__global__ void k_tadj_prep(const double2* alpha, const double2* beta, const double2* gamma, int n, double* scal) {
    __shared__ double red[32];
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
        scal[0] = log(fmax(mm, 1e-300));
    }
}

// Solve M x = rhs for the tridiagonal M (diag d_j + shift, below l_j, above u_j), Gaussian elimination
// with partial pivoting; rows of the eliminated system in the thread's scratch columns (stride nt).
// adj = true solves with M = G^dag (diag conj(alpha), below conj(gamma), above conj(beta)).
// rhs: e_1 if null.  Returns false if singular.  x overwrites bd.
__device__ bool tri_solve(const double2* alpha, const double2* beta, const double2* gamma, bool adj, cx<double> shift,
                          const double2* rhs, int n, double2* bd, double2* ud, double2* wd, int nt, int t) {
#define IDX(i) ((size_t)(i) * nt + t)
    auto D = [&](int j) { const cx<double> a = d2c(alpha[j]); return (adj ? conj(a) : a) + shift; };
    auto Lw = [&](int j) { return adj ? conj(d2c(gamma[j])) : d2c(beta[j]); };   // row j+1, col j
    auto Up = [&](int j) { return adj ? conj(d2c(beta[j])) : d2c(gamma[j]); };   // row j, col j+1
    auto R = [&](int j) { return rhs ? d2c(rhs[j]) : (j == 0 ? mk(1.0, 0.0) : mk(0.0, 0.0)); };
    cx<double> d = D(0);
    cx<double> uu = n > 1 ? Up(0) : mk(0.0, 0.0);
    cx<double> rb = R(0);
    for (int i = 0; i + 1 < n; ++i) {
        const cx<double> l = Lw(i), dn = D(i + 1);
        const cx<double> un = (i + 2 < n) ? Up(i + 1) : mk(0.0, 0.0);
        const cx<double> rn = R(i + 1);
        if (norm2(d) >= norm2(l)) {
            if (norm2(d) == 0.0) return false;
            const double inv = 1.0 / norm2(d);
            const cx<double> id = mk(d.r * inv, -d.i * inv);
            const cx<double> m = l * id;
            bd[IDX(i)] = c2d(rb * id);
            ud[IDX(i)] = c2d(uu * id);
            wd[IDX(i)] = make_double2(0.0, 0.0);
            d = dn - m * uu;
            uu = un;
            rb = rn - m * rb;
        } else {
            const double inv = 1.0 / norm2(l);
            const cx<double> il = mk(l.r * inv, -l.i * inv);
            const cx<double> m = d * il;
            bd[IDX(i)] = c2d(rn * il);
            ud[IDX(i)] = c2d(dn * il);
            wd[IDX(i)] = c2d(un * il);
            const cx<double> nd = uu - m * dn;
            const cx<double> nu = mk(0.0, 0.0) - m * un;
            rb = rb - m * rn;
            d = nd;
            uu = nu;
        }
    }
    if (norm2(d) == 0.0) return false;
    cx<double> x1 = cdiv(rb, d), x2 = mk(0.0, 0.0);
    bd[IDX(n - 1)] = c2d(x1);
    for (int i = n - 2; i >= 0; --i) {
        const cx<double> x = d2c(bd[IDX(i)]) - d2c(ud[IDX(i)]) * x1 - d2c(wd[IDX(i)]) * x2;
        bd[IDX(i)] = c2d(x);
        x2 = x1;
        x1 = x;
    }
#undef IDX
    return true;
}


// one thread per (node, sign s): a = (G + s i e^u)^-1 e_1 and d = (G^dag - s i e^u)^-1 e_1 into the
// scratch (region 0: a, region 3: d; thread columns)
__global__ void k_gq_solve(const double2* alpha, const double2* beta, const double2* gamma, int n,
                           const double* scal, double2* work, int level, int nt, int* status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double lo = scal[0] - TADJ_HALFWIDTH;
    const int node = t >> 1;
    const double sg = (t & 1) ? -1.0 : 1.0;
    const double u = level == 0 ? lo + node * TADJ_H0 : lo + (2 * node + 1) * (TADJ_H0 / (double)(1 << level));
    const double tau = exp(u);
    double2* r = work;
    double2* d = work + 3 * (size_t)n * nt;
    if (!tri_solve(alpha, beta, gamma, false, mk(0.0, sg * tau), nullptr, n, r, r + (size_t)n * nt,
                   r + 2 * (size_t)n * nt, nt, t) ||
        !tri_solve(alpha, beta, gamma, true, mk(0.0, -sg * tau), nullptr, n, d, d + (size_t)n * nt,
                   d + 2 * (size_t)n * nt, nt, t)) {
        atomicExch(status, 5);
        return;
    }
    // weight e^u folded into a; e^u kept for the d sum (region 1 is free after the solves)
    for (int j = 0; j < n; ++j) r[(size_t)j * nt + t] = c2d(tau * d2c(r[(size_t)j * nt + t]));
    work[(size_t)n * nt + t] = make_double2(tau, 0.0);
}

// M_l = M_{l-1}/2 + h_l sum_threads conj(d_p) (e^u a_q), a 16 x 16 tile of (p, q) per block, the
// thread sum in chunks of 32 through shared memory (fixed order); partial sums of |M_l - M_{l-1}|^2
// and |M_l|^2
constexpr int GQ_T = 16, GQ_C = 32;
__global__ void __launch_bounds__(256) k_gq_accum(const double2* __restrict__ work, int n, int nt, int level,
                                                  double2* __restrict__ M, double* partials, unsigned int* counter,
                                                  double* dn) {
    __shared__ double2 ds[GQ_T][GQ_C + 1];
    __shared__ double2 as[GQ_T][GQ_C + 1];
    __shared__ double red[64];
    const double hl = TADJ_H0 / (double)(1 << level);
    const double2* a = work;
    const double2* d = work + 3 * (size_t)n * nt;
    // one-dimensional grid (the grid reduction below counts blocks along x): tile (p, q) of M
    const int ntq = (n + GQ_T - 1) / GQ_T;
    const int p0 = (blockIdx.x / ntq) * GQ_T, q0 = (blockIdx.x % ntq) * GQ_T;
    const int tp = threadIdx.x >> 4, tq = threadIdx.x & 15;
    cx<double> acc = mk(0.0, 0.0);
    for (int t0 = 0; t0 < nt; t0 += GQ_C) {
        for (int x = threadIdx.x; x < GQ_T * GQ_C; x += blockDim.x) {
            const int rr = x / GQ_C, tt = x % GQ_C;
            const bool okt = t0 + tt < nt;
            ds[rr][tt] = (okt && p0 + rr < n) ? d[(size_t)(p0 + rr) * nt + t0 + tt] : make_double2(0.0, 0.0);
            as[rr][tt] = (okt && q0 + rr < n) ? a[(size_t)(q0 + rr) * nt + t0 + tt] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 8
        for (int tt = 0; tt < GQ_C; ++tt) cfma(acc, conj(d2c(ds[tp][tt])), d2c(as[tq][tt]));
        __syncthreads();
    }
    double part[2] = {0.0, 0.0};
    const int p = p0 + tp, q = q0 + tq;
    if (p < n && q < n) {
        const size_t e = (size_t)p * n + q;
        const double2 old = M[e];
        const double2 nv = make_double2((level == 0 ? 0.0 : 0.5 * old.x) + hl * acc.r,
                                        (level == 0 ? 0.0 : 0.5 * old.y) + hl * acc.i);
        M[e] = nv;
        part[0] = (nv.x - old.x) * (nv.x - old.x) + (nv.y - old.y) * (nv.y - old.y);
        part[1] = nv.x * nv.x + nv.y * nv.y;
    }
    double o[2];
    if (grid_sum_last<2>(part, partials, counter, o, red) && threadIdx.x == 0) {
        dn[0] = o[0];
        dn[1] = o[1];
    }
}

// sd_l = sd_{l-1}/2 + h_l sum_threads e^u d (one warp per row p)
__global__ void k_gq_dsum(const double2* __restrict__ work, int n, int nt, int level, double2* __restrict__ sd) {
    const double hl = TADJ_H0 / (double)(1 << level);
    const double2* d = work + 3 * (size_t)n * nt;
    const double2* tau = work + (size_t)n * nt;
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= n) return;
    double sr = 0.0, si = 0.0;
    for (int t = lane; t < nt; t += 32) {
        const double w = tau[t].x;
        sr += w * d[(size_t)p * nt + t].x;
        si += w * d[(size_t)p * nt + t].y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
        const double2 old = sd[p];
        sd[p] = make_double2((level == 0 ? 0.0 : 0.5 * old.x) + hl * sr, (level == 0 ? 0.0 : 0.5 * old.y) + hl * si);
    }
}

// M~_pq = -(|b| conj(zeta)/pi) M_pq conj(ws_p) vs_q (for the stored, unnormalised v~, w~), in place;
// sd_p <- (zeta/pi) ws_p sd_p (the coefficients of g_b in w~)
__global__ void k_gq_finish(double2* M, double2* sd, int n, const KState* ks, const double2* zeta,
                            const double2* vscale, const double2* wscale) {
    const size_t nn = (size_t)n * n;
    const cx<double> zt = d2c(*zeta);
    const cx<double> f = (-ks->nR / M_PI) * conj(zt);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn + n; e += (size_t)gridDim.x * blockDim.x) {
        if (e < nn) {
            const int p = (int)(e / n), q = (int)(e % n);
            M[e] = c2d(f * d2c(M[e]) * conj(d2c(wscale[p])) * d2c(vscale[q]));
        } else {
            const int p = (int)(e - nn);
            sd[p] = c2d((1.0 / M_PI) * zt * d2c(wscale[p]) * d2c(sd[p]));
        }
    }
}

// Z_q = sum_p conj(M~_pq) w~_p for q < k (vectors of n complex, ld n): tiles of 64 elements x 16
// columns, the p sum in chunks of 16 through shared memory
constexpr int ZT_E = 64, ZT_Q = 16, ZT_P = 16;
__global__ void __launch_bounds__(256) k_gq_combine(const double2* __restrict__ W, const double2* __restrict__ M,
                                                    double2* __restrict__ Z, int k, size_t n) {
    __shared__ double2 ws[ZT_P][ZT_E];
    __shared__ double2 ms[ZT_P][ZT_Q];
    const size_t e0 = (size_t)blockIdx.x * ZT_E;
    const int q0 = blockIdx.y * ZT_Q;
    const int te = threadIdx.x & 63, tq = threadIdx.x >> 6;  // 4 groups of 4 columns
    cx<double> acc[4] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
    for (int p0 = 0; p0 < k; p0 += ZT_P) {
        for (int x = threadIdx.x; x < ZT_P * ZT_E; x += blockDim.x) {
            const int pp = x / ZT_E, ee = x % ZT_E;
            const size_t e = e0 + ee;
            ws[pp][ee] = (p0 + pp < k && e < n) ? W[(size_t)(p0 + pp) * n + e] : make_double2(0.0, 0.0);
        }
        for (int x = threadIdx.x; x < ZT_P * ZT_Q; x += blockDim.x) {
            const int pp = x / ZT_Q, qq = x % ZT_Q;
            const double2 m = (p0 + pp < k && q0 + qq < k) ? M[(size_t)(p0 + pp) * k + q0 + qq] : make_double2(0.0, 0.0);
            ms[pp][qq] = make_double2(m.x, -m.y);
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < ZT_P; ++pp) {
            const cx<double> w = d2c(ws[pp][te]);
#pragma unroll
            for (int j = 0; j < 4; ++j) cfma(acc[j], d2c(ms[pp][tq * 4 + j]), w);
        }
        __syncthreads();
    }
    const size_t e = e0 + te;
    if (e < n)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = q0 + tq * 4 + j;
            if (q < k) Z[(size_t)q * n + e] = c2d(acc[j]);
        }
}

// (1 + S gamma_nu) gamma5 x as a full spinor
template <int NU, int S>
__device__ __forceinline__ void proj_g5_full(const Spinor<double>& x, Spinor<double>& o) {
    Spinor<double> g5 = x;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g5.s[2][a] = -x.s[2][a];
        g5.s[3][a] = -x.s[3][a];
    }
    Half<double> h;
    project<NU, S>(g5, h);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) o.s[sp][a] = mk(0.0, 0.0);
    recon_acc<NU, S>(o, h, 1.0);
}

template <int NU, int S, class R>
__device__ __forceinline__ void proj_g5_full_r(const Spinor<R>& x, Spinor<R>& o) {
    Spinor<R> g5 = x;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g5.s[2][a] = -x.s[2][a];
        g5.s[3][a] = -x.s[3][a];
    }
    Half<R> h;
    project<NU, S>(g5, h);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) o.s[sp][a] = mk(R(0), R(0));
    recon_acc<NU, S>(o, h, R(1));
}

// link force of y = gamma5 D_w(m) x for the adjoint gr of y, added into gU (device link layout):
// gU[x, nu] += -kappa ph (cf g~ (x) conj(x(x+nu)) + cb x(x) (x) conj(g^)),
// g~ = (1 + gamma_nu) gamma5 gr(x), g^ = (1 - gamma_nu) gamma5 gr(x + nu)
template <int NU>
__device__ __forceinline__ void link_force(const Geom& g, const Coord& c, int s, const double2* x,
                                           const double2* gr, double cf, double cb, cx<double> (&z)[9]) {
    const int f = neighbour(g, c, NU, +1);
    const double ph = (NU == 3 && c.x[3] == g.L[3] - 1) ? (double)g.bc_t : 1.0;
    Spinor<double> gx, gy, px, py, gt, gh;
    load_spinor(gr, g.V, s, gx);
    load_spinor(gr, g.V, f, gy);
    load_spinor(x, g.V, s, px);
    load_spinor(x, g.V, f, py);
    proj_g5_full<NU, +1>(gx, gt);
    proj_g5_full<NU, -1>(gy, gh);
    const double af = -cf * ph, ab = -cb * ph;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> w = z[3 * i + j];
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
                w = w + af * cdot(py.s[sp][j], gt.s[sp][i]);
                w = w + ab * cdot(gh.s[sp][j], px.s[sp][i]);
            }
            z[3 * i + j] = w;
        }
}


// Re <gr, dA/dmu x> at site s, dA/dmu = -kappa gamma5 (e^mu T_4^+ - e^-mu T_4^-)
__device__ __forceinline__ double dmu_site(const Geom& g, const Coord& c, int s, const double2* U,
                                           const double2* x, const double2* gr, double kappa, double m) {
    Spinor<double> acc, p, gs;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc.s[sp][a] = mk(0.0, 0.0);
    Link<double> L;
    Half<double> h, uh;
    const int f = neighbour(g, c, 3, +1), b = neighbour(g, c, 3, -1);
    const double phf = (c.x[3] == g.L[3] - 1) ? (double)g.bc_t : 1.0;
    const double phb = (c.x[3] == 0) ? (double)g.bc_t : 1.0;
    load_spinor(x, g.V, f, p);
    load_link(U, g.V, 3, s, L);
    project<3, +1>(p, h);
    mul_link(L, h, uh);
    recon_acc<3, +1>(acc, uh, -kappa * exp(m) * phf);
    load_spinor(x, g.V, b, p);
    load_link(U, g.V, 3, b, L);
    project<3, -1>(p, h);
    mul_link_dag(L, h, uh);
    recon_acc<3, -1>(acc, uh, kappa * exp(-m) * phb);
    load_spinor(gr, g.V, s, gs);
    double r = 0.0;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const cx<double> e = sp >= 2 ? -acc.s[sp][a] : acc.s[sp][a];
            r += cdot(gs.s[sp][a], e).r;
        }
    return r;
}

// gU = sum_q force(v~_q, Z_q) (the link adjoint of Re <Z_q, A v~_q>), gmu = sum_q Re <Z_q, dA/dmu v~_q>;
// one thread per site and direction block, the q sum inside (fixed order)
// The same product in double-float arithmetic (products exact through the FMA split, sums
// compensated; about 48 significant bits, on the FP32 pipe), FP64 in and out.
__global__ void __launch_bounds__(256) k_gq_combine_df(const double2* __restrict__ W, const double2* __restrict__ M,
                                                       double2* __restrict__ Z, int k, size_t n) {
    __shared__ float4 ws[ZT_P][ZT_E];
    __shared__ float4 ms[ZT_P][ZT_Q];
    const size_t e0 = (size_t)blockIdx.x * ZT_E;
    const int q0 = blockIdx.y * ZT_Q;
    const int te = threadIdx.x & 63, tq = threadIdx.x >> 6;  // 4 groups of 4 columns
    dfacc ar[4], ai[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) ar[j] = ai[j] = {0.f, 0.f};
    for (int p0 = 0; p0 < k; p0 += ZT_P) {
        for (int x = threadIdx.x; x < ZT_P * ZT_E; x += blockDim.x) {
            const int pp = x / ZT_E, ee = x % ZT_E;
            const size_t e = e0 + ee;
            const double2 w = (p0 + pp < k && e < n) ? W[(size_t)(p0 + pp) * n + e] : make_double2(0.0, 0.0);
            const dfc d = c2dfc(d2df(w));
            ws[pp][ee] = make_float4(d.rh, d.rl, d.ih, d.il);
        }
        for (int x = threadIdx.x; x < ZT_P * ZT_Q; x += blockDim.x) {
            const int pp = x / ZT_Q, qq = x % ZT_Q;
            const double2 m = (p0 + pp < k && q0 + qq < k) ? M[(size_t)(p0 + pp) * k + q0 + qq] : make_double2(0.0, 0.0);
            const dfc d = c2dfc(d2df(make_double2(m.x, -m.y)));
            ms[pp][qq] = make_float4(d.rh, d.rl, d.ih, d.il);
        }
        __syncthreads();
#pragma unroll 2
        for (int pp = 0; pp < ZT_P; ++pp) {
            const float4 wv = ws[pp][te];
            const df wr(wv.x, wv.y), wi(wv.z, wv.w);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 mv = ms[pp][tq * 4 + j];
                const df mr(mv.x, mv.y), mi(mv.z, mv.w);
                dfacc_add(ar[j], mr, wr, false);
                dfacc_add(ar[j], mi, wi, true);
                dfacc_add(ai[j], mr, wi, false);
                dfacc_add(ai[j], mi, wr, false);
            }
        }
        __syncthreads();
    }
    const size_t e = e0 + te;
    if (e < n)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = q0 + tq * 4 + j;
            if (q < k) Z[(size_t)q * n + e] = df2d(mk(dfacc_value(ar[j]), dfacc_value(ai[j])));
        }
}

// The same product in FP32 (the mixed-precision gradient), FP64 in and out.
__global__ void __launch_bounds__(256) k_gq_combine_f32(const double2* __restrict__ W, const double2* __restrict__ M,
                                                        double2* __restrict__ Z, int k, size_t n) {
    __shared__ float2 ws[ZT_P][ZT_E];
    __shared__ float2 ms[ZT_P][ZT_Q];
    const size_t e0 = (size_t)blockIdx.x * ZT_E;
    const int q0 = blockIdx.y * ZT_Q;
    const int te = threadIdx.x & 63, tq = threadIdx.x >> 6;
    cx<float> acc[4] = {mk(0.f, 0.f), mk(0.f, 0.f), mk(0.f, 0.f), mk(0.f, 0.f)};
    for (int p0 = 0; p0 < k; p0 += ZT_P) {
        for (int x = threadIdx.x; x < ZT_P * ZT_E; x += blockDim.x) {
            const int pp = x / ZT_E, ee = x % ZT_E;
            const size_t e = e0 + ee;
            const double2 w = (p0 + pp < k && e < n) ? W[(size_t)(p0 + pp) * n + e] : make_double2(0.0, 0.0);
            ws[pp][ee] = make_float2((float)w.x, (float)w.y);
        }
        for (int x = threadIdx.x; x < ZT_P * ZT_Q; x += blockDim.x) {
            const int pp = x / ZT_Q, qq = x % ZT_Q;
            const double2 m = (p0 + pp < k && q0 + qq < k) ? M[(size_t)(p0 + pp) * k + q0 + qq] : make_double2(0.0, 0.0);
            ms[pp][qq] = make_float2((float)m.x, (float)-m.y);
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < ZT_P; ++pp) {
            const float2 wv = ws[pp][te];
            const cx<float> w = mk(wv.x, wv.y);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 mv = ms[pp][tq * 4 + j];
                cfma(acc[j], mk(mv.x, mv.y), w);
            }
        }
        __syncthreads();
    }
    const size_t e = e0 + te;
    if (e < n)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = q0 + tq * 4 + j;
            if (q < k) Z[(size_t)q * n + e] = make_double2((double)acc[j].r, (double)acc[j].i);
        }
}

// FP32 form of the link force and mu derivative over the pairs (v_q, Z_q) for the mixed-precision
// gradient: every pair's contribution in FP32 from the FP64 vectors, the sum over pairs compensated
// (Kahan) in FP32 for the links and in FP64 for d/dmu.
template <int NU>
__device__ __forceinline__ void link_force_f32(const Geom& g, const Coord& c, int s, const double2* x,
                                               const double2* gr, float cf, float cb, cx<float> (&z)[9],
                                               cx<float> (&zc)[9]) {
    const int f = neighbour(g, c, NU, +1);
    const float ph = (NU == 3 && c.x[3] == g.L[3] - 1) ? (float)g.bc_t : 1.f;
    Spinor<double> dgx, dgy, dpx, dpy;
    load_spinor(gr, g.V, s, dgx);
    load_spinor(gr, g.V, f, dgy);
    load_spinor(x, g.V, s, dpx);
    load_spinor(x, g.V, f, dpy);
    Spinor<float> gx, gy, px, py, gt, gh;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gx.s[sp][a] = mk((float)dgx.s[sp][a].r, (float)dgx.s[sp][a].i);
            gy.s[sp][a] = mk((float)dgy.s[sp][a].r, (float)dgy.s[sp][a].i);
            px.s[sp][a] = mk((float)dpx.s[sp][a].r, (float)dpx.s[sp][a].i);
            py.s[sp][a] = mk((float)dpy.s[sp][a].r, (float)dpy.s[sp][a].i);
        }
    proj_g5_full_r<NU, +1, float>(gx, gt);
    proj_g5_full_r<NU, -1, float>(gy, gh);
    const float af = -cf * ph, ab = -cb * ph;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<float> w = mk(0.f, 0.f);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
                w = w + af * cdot(py.s[sp][j], gt.s[sp][i]);
                w = w + ab * cdot(gh.s[sp][j], px.s[sp][i]);
            }
            // Kahan: z + w with the lost low part carried in zc
            const cx<float> yv = w - zc[3 * i + j];
            const cx<float> t = z[3 * i + j] + yv;
            zc[3 * i + j] = (t - z[3 * i + j]) - yv;
            z[3 * i + j] = t;
        }
}

__global__ void __launch_bounds__(GT) k_force_sum_f32(const double2* __restrict__ U, const double2* __restrict__ V,
                                                      const double2* __restrict__ Z, int k, double2* __restrict__ gU,
                                                      double kappa, double mu, Geom g, double* partials,
                                                      unsigned int* counter, double* gmu) {
    __shared__ double red[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int nu = blockIdx.y;  // 0..3 links, 4: the mu derivative
    const size_t n = (size_t)12 * g.V;
    double part[1] = {0.0};
    if (s < g.V) {
        const Coord c = site_coord(g, s);
        if (nu < 4) {
            cx<float> z[9], zc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) z[q] = zc[q] = mk(0.f, 0.f);
            const float cf = nu == 3 ? (float)(kappa * exp(mu)) : (float)kappa;
            const float cb = nu == 3 ? (float)(kappa * exp(-mu)) : (float)kappa;
            for (int q = 0; q < k; ++q) {
                const double2* x = V + (size_t)q * n;
                const double2* gr = Z + (size_t)q * n;
                switch (nu) {
                    case 0: link_force_f32<0>(g, c, s, x, gr, cf, cb, z, zc); break;
                    case 1: link_force_f32<1>(g, c, s, x, gr, cf, cb, z, zc); break;
                    case 2: link_force_f32<2>(g, c, s, x, gr, cf, cb, z, zc); break;
                    default: link_force_f32<3>(g, c, s, x, gr, cf, cb, z, zc); break;
                }
            }
#pragma unroll
            for (int q = 0; q < 9; ++q)
                gU[((size_t)nu * 9 + q) * g.V + s] = make_double2((double)z[q].r - (double)zc[q].r,
                                                                  (double)z[q].i - (double)zc[q].i);
        } else {
            for (int q = 0; q < k; ++q) part[0] += dmu_site(g, c, s, U, V + (size_t)q * n, Z + (size_t)q * n, kappa, mu);
        }
    }
    if (nu == 4) {
        double out[1];
        if (grid_sum_last<1>(part, partials, counter, out, red) && threadIdx.x == 0) *gmu = out[0];
    }
}

__global__ void __launch_bounds__(GT) k_force_sum(const double2* __restrict__ U, const double2* __restrict__ V,
                                                  const double2* __restrict__ Z, int k, double2* __restrict__ gU,
                                                  double kappa, double mu, Geom g, double* partials,
                                                  unsigned int* counter, double* gmu) {
    __shared__ double red[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int nu = blockIdx.y;  // 0..3 links, 4: the mu derivative
    const size_t n = (size_t)12 * g.V;
    double part[1] = {0.0};
    if (s < g.V) {
        const Coord c = site_coord(g, s);
        if (nu < 4) {
            cx<double> z[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) z[q] = mk(0.0, 0.0);
            const double cf = nu == 3 ? kappa * exp(mu) : kappa, cb = nu == 3 ? kappa * exp(-mu) : kappa;
            for (int q = 0; q < k; ++q) {
                const double2* x = V + (size_t)q * n;
                const double2* gr = Z + (size_t)q * n;
                switch (nu) {
                    case 0: link_force<0>(g, c, s, x, gr, cf, cb, z); break;
                    case 1: link_force<1>(g, c, s, x, gr, cf, cb, z); break;
                    case 2: link_force<2>(g, c, s, x, gr, cf, cb, z); break;
                    default: link_force<3>(g, c, s, x, gr, cf, cb, z); break;
                }
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) gU[((size_t)nu * 9 + q) * g.V + s] = c2d(z[q]);
        } else {
            for (int q = 0; q < k; ++q) part[0] += dmu_site(g, c, s, U, V + (size_t)q * n, Z + (size_t)q * n, kappa, mu);
        }
    }
    if (nu == 4) {
        double out[1];
        if (grid_sum_last<1>(part, partials, counter, out, red) && threadIdx.x == 0) *gmu = out[0];
    }
}

// device link layout -> canonical [site][nu][3][3]
__global__ void k_links_to_canon(const double2* __restrict__ gU, double2* __restrict__ out, Geom g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const Coord c = site_coord(g, s);
    const int cs = canon_index(g, c.x);
    for (int nu = 0; nu < 4; ++nu)
        for (int q = 0; q < 9; ++q) out[((size_t)cs * 4 + nu) * 9 + q] = gU[((size_t)nu * 9 + q) * g.V + s];
}


int grid_n(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 1024); }

}  // namespace
}  // namespace ovl

using namespace ovl_priv;
using ovl::make_coef;

extern "C" int ovl_sign_grad(ovl_ctx* c, int k, double mu, double kappa, const void* b, const void* gy, void* y,
                             void* grad_U, double* grad_mu, void* grad_b, int flags, ovl_info* info) {
    if (!c || !b || !gy) return fail(c, OVL_EINVAL, "null argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    if (k < 1) return fail(c, OVL_EINVAL, "k must be positive");
    if (flags & OVL_HOST) return fail(c, OVL_EINVAL, "device pointers only");
    if (flags & ~OVL_MIXED) return fail(c, OVL_EINVAL, "flags: 0 or OVL_MIXED");
    const bool mixed = (flags & OVL_MIXED) != 0;
    int r = ensure_solve(c, k);
    if (r) return r;
    cudaStream_t st = c->st;
    const size_t n = c->n;
    const ovl::Geom& g = c->g;
    const size_t vb = n * sizeof(double2);
    ovl::KState* ks = c->ks;
    double* part = c->partials;
    unsigned int* cnt = c->counter;
    // ---- workspace: W (k + 1 vectors), Z (k vectors), g_y packed, link gradient, scalars
    const size_t kk1 = (size_t)k + 1;
    // (mixed: the FP32 bases, (k + 1) vectors of n complex64 each, after the FP64 ones)
    const size_t need = ((2 * kk1 + 1 + 3 + 1) * n + 4 * kk1 + (size_t)k * k + 64) * sizeof(double2) +
                        (mixed ? 2 * kk1 * n * sizeof(float2) : 0);
    if (c->gwork_bytes < need) {
        if (c->gwork) cudaFree(c->gwork);
        c->gwork = nullptr;
        c->gwork_bytes = 0;
        if (cudaMalloc(&c->gwork, need) != cudaSuccess) return fail(c, OVL_ENOMEM, "gradient workspace");
        c->gwork_bytes = need;
    }
    double2* W = (double2*)c->gwork;
    double2* Z = W + kk1 * n;
    double2* gyd = Z + kk1 * n;
    double2* gUd = gyd + n;  // 36 V = 3 n
    double2* tmp = gUd + 3 * n;
    double2* wscale = tmp + n;
    double2* sd = wscale + kk1;
    double2* M = sd + kk1;
    double2* misc = M + (size_t)k * k + 2 * kk1;
    double2* zeta = misc;
    double* gmu_acc = reinterpret_cast<double*>(misc + 2);
    double* dn = gmu_acc + 2;
    double* tscal = gmu_acc + 8;
    int* tstatus = reinterpret_cast<int*>(gmu_acc + 16);
    OVL_CUDA_TRY(c, cudaMemsetAsync(misc, 0, 32 * sizeof(double2), st));
    ovl::launch_pack_spinor((const double2*)b, c->b64, 0, g, st);
    ovl::launch_pack_spinor((const double2*)gy, gyd, 0, g, st);
    // ---- two-sided Lanczos from (b, g), bases kept (Sec. 4, Eq. 4.2); mixed: in FP32 with 12-real
    // links and FP64 reductions and coefficients, the FP32 bases then widened to FP64
    double2* V = c->V64;
    ovl::launch_state_init(ks, st);
    ovl::k_bilinear_start<<<ovl::grid_n(n), 256, 0, st>>>(c->b64, gyd, V, W, c->y64, ks, c->vscale, wscale, zeta,
                                                          part, cnt, n);
    if (mixed) {
        float2* V32 = reinterpret_cast<float2*>(misc + 32);
        float2* W32 = V32 + kk1 * n;
        ovl::launch_native_f64_to_f32(V, V32, g, 1, st);
        ovl::launch_native_f64_to_f32(W, W32, g, 1, st);
        for (int i = 0; i < k; ++i) {
            const float2* vi = V32 + (size_t)i * n;
            const float2* wi = W32 + (size_t)i * n;
            ovl::launch_dslash_pair(c->U12, 1, vi, wi, c->t32, c->s32, mu, kappa, ks, c->alpha, i, k - 1, part, cnt, g,
                                    st);
            if (i + 1 < k)
                ovl::launch_lanczos_step(1, c->t32, c->s32, vi, wi, i > 0 ? vi - n : vi, i > 0 ? wi - n : wi,
                                         V32 + (size_t)(i + 1) * n, W32 + (size_t)(i + 1) * n, ks, c->alpha, c->beta,
                                         c->gamma, c->vscale, i, k, part, cnt, n, st);
        }
        ovl::launch_native_f32_to_f64(V32, V, g, k, st);
        ovl::launch_native_f32_to_f64(W32, W, g, k, st);
    } else {
        for (int i = 0; i < k; ++i) {
            const double2* vi = V + (size_t)i * n;
            const double2* wi = W + (size_t)i * n;
            ovl::launch_dslash_pair(c->U64, 0, vi, wi, c->t64, c->s64, mu, kappa, ks, c->alpha, i, k - 1, part, cnt, g,
                                    st);
            if (i + 1 < k)
                ovl::launch_lanczos_step(0, c->t64, c->s64, vi, wi, i > 0 ? vi - n : vi, i > 0 ? wi - n : wi,
                                         V + (size_t)(i + 1) * n, W + (size_t)(i + 1) * n, ks, c->alpha, c->beta,
                                         c->gamma, c->vscale, i, k, part, cnt, n, st);
        }
    }
    ovl::k_wscale<<<(k + 127) / 128, 128, 0, st>>>(c->gamma, ks, wscale);
    // ---- y = |b| V sgn(G) e_1 (inner sign as in the solve)
    r = ovl::launch_inner_quadrature(c->alpha, c->beta, c->gamma, ks, c->cvec, c->inner, c->inner_elems, c->kcap, part,
                                     cnt, st);
    if (!r)
        r = ovl::launch_inner_newton(c->alpha, c->beta, c->gamma, nullptr, 0, 1, ks, c->cvec, c->inner, c->inner_elems,
                                     c->kcap, c->num_sms, st, 1);
    if (r) return fail(c, OVL_ECUDA, "inner sign launch failed");
    ovl::launch_combine(V, n, c->vscale, c->cvec, ks, c->kcap, c->y64, n, st);
    ovl::KState hk;
    OVL_CUDA_TRY(c, cudaMemcpyAsync(&hk, ks, sizeof(hk), cudaMemcpyDeviceToHost, st));
    OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (info) {
        info->k_used = hk.kused;
        info->breakdown_step = hk.bdstep;
        info->inner_iters = hk.inner_iters;
        info->inner_method = hk.inner_method;
        info->bperp_norm = hk.nR;
        info->inner_err = hk.inner_err;
    }
    if (hk.timeout) return fail(c, OVL_ETIMEOUT, "a bounded device wait gave up");
    if (hk.status == OVL_ESINGULAR) return fail(c, OVL_ESINGULAR, "singular projected matrix");
    if (hk.status == OVL_ENOCONV) return fail(c, OVL_ENOCONV, "inner sign did not converge");
    if (hk.status) return fail(c, hk.status, "two-sided Lanczos failed");
    if (hk.bdstep >= 0)
        return fail(c, OVL_EBREAKDOWN, hk.bdstep == 0 ? "g^dag b = 0: the two-sided process from (b, g) cannot start"
                                                      : "two-sided Lanczos serious breakdown");
    if (y) ovl::launch_unpack_spinor(c->y64, 0, (double2*)y, nullptr, 0, g, st);
    const int kk = hk.kused;
    if (kk == 0) {  // b = 0: y and every gradient vanish
        if (grad_U) OVL_CUDA_TRY(c, cudaMemsetAsync(grad_U, 0, (size_t)g.V * 36 * sizeof(double2), st));
        if (grad_b) OVL_CUDA_TRY(c, cudaMemsetAsync(grad_b, 0, vb, st));
        if (grad_mu) *grad_mu = 0.0;
        OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
        return OVL_OK;
    }
    // ---- the k x k matrix M and sgn(G^dag) e_1 by the trapezoid rule in u, step halved until M settles
    {
        const int m0 = (int)std::ceil(2 * ovl::TADJ_HALFWIDTH / ovl::TADJ_H0);
        const int tmax = 2 * (m0 << (ovl::TADJ_LEVELS - 2));
        const size_t tw = 6 * (size_t)kk * tmax + 16;
        if (c->tadj_elems < tw) {
            if (c->tadj) cudaFree(c->tadj);
            c->tadj = nullptr;
            c->tadj_elems = 0;
            if (cudaMalloc(&c->tadj, tw * sizeof(double2)) != cudaSuccess)
                return fail(c, OVL_ENOMEM, "quadrature workspace of the gradient");
            c->tadj_elems = tw;
        }
        ovl::k_tadj_prep<<<1, 256, 0, st>>>(c->alpha, c->beta, c->gamma, kk, tscal);
        bool conv = false;
        for (int level = 0; level < ovl::TADJ_LEVELS && !conv; ++level) {
            const int nt = level == 0 ? 2 * m0 : 2 * (m0 << (level - 1));
            ovl::k_gq_solve<<<(nt + 31) / 32, 32, 0, st>>>(c->alpha, c->beta, c->gamma, kk, tscal, c->tadj, level, nt,
                                                           tstatus);
            const int ntile = (kk + ovl::GQ_T - 1) / ovl::GQ_T;
            ovl::k_gq_accum<<<ntile * ntile, 256, 0, st>>>(c->tadj, kk, nt, level, M, part, cnt, dn);
            ovl::k_gq_dsum<<<(kk + 7) / 8, 256, 0, st>>>(c->tadj, kk, nt, level, sd);
            double hd[2];
            int hst = 0;
            OVL_CUDA_TRY(c, cudaMemcpyAsync(hd, dn, sizeof(hd), cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(c, cudaMemcpyAsync(&hst, tstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
            if (hst) return fail(c, OVL_ESINGULAR, "shifted projected matrix is singular");
            // geometric convergence: the error of level l is about rel^2
            const double rel = std::sqrt(hd[0]) / std::max(std::sqrt(hd[1]), 1e-300);
            if (level > 0 && rel <= 1e-6) conv = true;
        }
        if (!conv) return fail(c, OVL_ENOCONV, "quadrature of the gradient did not converge");
        const size_t ne = (size_t)kk * kk + kk;
        ovl::k_gq_finish<<<ovl::grid_n(ne), 256, 0, st>>>(M, sd, kk, ks, zeta, c->vscale, wscale);
    }
    // ---- Z = W~ conj(M~), then the link force and mu derivative of the pairs (v~_q, Z_q)
    const int B = (g.V + ovl::GT - 1) / ovl::GT;
    if (grad_U || grad_mu) {
        dim3 gz((unsigned)((n + ovl::ZT_E - 1) / ovl::ZT_E), (unsigned)((kk + ovl::ZT_Q - 1) / ovl::ZT_Q));
        if (mixed) {
            ovl::k_gq_combine_f32<<<gz, 256, 0, st>>>(W, M, Z, kk, n);
            ovl::k_force_sum_f32<<<dim3(B, 5), ovl::GT, 0, st>>>(c->U64, V, Z, kk, gUd, kappa, mu, g, part, cnt,
                                                                 gmu_acc);
        } else {
            ovl::k_gq_combine_df<<<gz, 256, 0, st>>>(W, M, Z, kk, n);
            ovl::k_force_sum<<<dim3(B, 5), ovl::GT, 0, st>>>(c->U64, V, Z, kk, gUd, kappa, mu, g, part, cnt, gmu_acc);
        }
        if (grad_U) ovl::k_links_to_canon<<<B, ovl::GT, 0, st>>>(gUd, (double2*)grad_U, g);
    }
    if (grad_b) {
        OVL_CUDA_TRY(c, cudaMemsetAsync(tmp, 0, vb, st));
        ovl::launch_combine(W, n, nullptr, sd, ks, c->kcap, tmp, n, st);
        ovl::launch_unpack_spinor(tmp, 0, (double2*)grad_b, nullptr, 0, g, st);
    }
    double hmu = 0.0;
    OVL_CUDA_TRY(c, cudaMemcpyAsync(&hmu, gmu_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
    OVL_CUDA_TRY(c, cudaGetLastError());
    if (grad_mu) *grad_mu = hmu;
    return OVL_OK;
}
