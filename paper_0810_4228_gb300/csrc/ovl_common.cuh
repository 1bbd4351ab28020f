// Shared device-side definitions of the overlap library: complex arithmetic,
// the even/odd lattice geometry, the Wilson hop (spin projection + SU(3)
// multiply + reconstruction, Sec. 1 Eq. 1.2), block/grid reductions and a
// bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef OVL_HD
#define OVL_HD __host__ __device__ __forceinline__
#endif

namespace ovl {

// True the first time it is called on the current device with this `seen` mask (one bit per device
// ordinal below 64; always true beyond): kernel attributes such as the dynamic shared-memory limit
// belong to the device they are set on, so a launcher sets them once per device.
inline bool first_use_on_device(unsigned long long& seen) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
    const unsigned long long bit = 1ull << dev;
    if (seen & bit) return false;
    seen |= bit;
    return true;
}

// ---------------------------------------------------------------- complex --
template <class R> struct cx {
    R r, i;
};
template <class R> OVL_HD cx<R> mk(R r, R i) { cx<R> z; z.r = r; z.i = i; return z; }
template <class R> OVL_HD cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.r + b.r, a.i + b.i); }
template <class R> OVL_HD cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.r - b.r, a.i - b.i); }
template <class R> OVL_HD cx<R> operator-(cx<R> a) { return mk(-a.r, -a.i); }
template <class R> OVL_HD cx<R> operator*(cx<R> a, cx<R> b) {
    return mk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <class R> OVL_HD cx<R> operator*(R s, cx<R> a) { return mk(s * a.r, s * a.i); }
template <class R> OVL_HD cx<R> conj(cx<R> a) { return mk(a.r, -a.i); }
template <class R> OVL_HD cx<R> times_i(cx<R> a) { return mk(-a.i, a.r); }   // i*a
template <class R> OVL_HD R norm2(cx<R> a) { return a.r * a.r + a.i * a.i; }
// conj(a) * b
template <class R> OVL_HD cx<R> cdot(cx<R> a, cx<R> b) {
    return mk(a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r);
}
// a += b * c
template <class R> OVL_HD void cfma(cx<R>& a, cx<R> b, cx<R> c) {
    a.r += b.r * c.r - b.i * c.i;
    a.i += b.r * c.i + b.i * c.r;
}
// a += conj(b) * c
template <class R> OVL_HD void cfmac(cx<R>& a, cx<R> b, cx<R> c) {
    a.r += b.r * c.r + b.i * c.i;
    a.i += b.r * c.i - b.i * c.r;
}
OVL_HD cx<double> up(cx<float> a) { return mk<double>(a.r, a.i); }
OVL_HD cx<double> up(cx<double> a) { return a; }
OVL_HD cx<double> d2c(double2 a) { return mk(a.x, a.y); }
OVL_HD double2 c2d(cx<double> a) { return make_double2(a.r, a.i); }
OVL_HD cx<double> cdiv(cx<double> a, cx<double> b) {
    // Smith's algorithm
    if (fabs(b.r) >= fabs(b.i)) {
        double q = b.i / b.r, d = b.r + b.i * q;
        return mk((a.r + a.i * q) / d, (a.i - a.r * q) / d);
    } else {
        double q = b.r / b.i, d = b.r * q + b.i;
        return mk((a.r * q + a.i) / d, (a.i * q - a.r) / d);
    }
}

// ---------------------------------------------------------------- geometry --
// Device layout: internal site index i = parity * Vh + (s >> 1), with s the
// canonical index ((x1*L2 + x2)*L3 + x3)*L4 + x4 and parity = (x1+x2+x3+x4) & 1.
// L4 must be even so that s>>1 enumerates the sites of one parity.
struct Geom {
    int L[4];
    int L4h;       // L4 / 2
    int V, Vh;
    int bc_t;      // +1 periodic, -1 antiperiodic in time
};

struct Coord {
    int x[4];
    int par;
};

OVL_HD Coord site_coord(const Geom& g, int i) {
    Coord c;
    c.par = i >= g.Vh;
    int cb = i - c.par * g.Vh;
    int x4h = cb % g.L4h;
    int rest = cb / g.L4h;
    c.x[2] = rest % g.L[2];
    rest /= g.L[2];
    c.x[1] = rest % g.L[1];
    c.x[0] = rest / g.L[1];
    c.x[3] = 2 * x4h + ((c.par + c.x[0] + c.x[1] + c.x[2]) & 1);
    return c;
}

OVL_HD int canon_index(const Geom& g, const int x[4]) {
    return ((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

OVL_HD int internal_index(const Geom& g, const int x[4]) {
    int s = canon_index(g, x);
    int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    return par * g.Vh + (s >> 1);
}

// neighbour x + dir*nu (dir = +1 / -1), internal index
OVL_HD int neighbour(const Geom& g, const Coord& c, int nu, int dir) {
    int y[4] = {c.x[0], c.x[1], c.x[2], c.x[3]};
    int v = y[nu] + dir;
    if (v == g.L[nu]) v = 0;
    if (v < 0) v = g.L[nu] - 1;
    y[nu] = v;
    return internal_index(g, y);
}

// ---------------------------------------------------------------- spinors --
// A 4-spinor as 4 spins x 3 colours; a half spinor as 2 x 3.
template <class R> struct Spinor { cx<R> s[4][3]; };
template <class R> struct Half { cx<R> h[2][3]; };

// S x for S = +1 or -1 (no multiplication)
template <int S, class T> OVL_HD T sgn_mul(T x) {
    if constexpr (S > 0) return x;
    else return -x;
}

// Spin projection (1 + S gamma_nu) psi -> half spinor h (upper two spins of the
// result), chiral basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
// gamma_4 = [[0, 1], [1, 0]].  The lower two spins of (1 + S gamma_nu) psi are
// recovered from h by `recon`.
template <int NU, int S, class R>
OVL_HD void project(const Spinor<R>& p, Half<R>& h) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (NU == 0) {          // sigma_1
            h.h[0][a] = p.s[0][a] - sgn_mul<S>(times_i(p.s[3][a]));
            h.h[1][a] = p.s[1][a] - sgn_mul<S>(times_i(p.s[2][a]));
        } else if (NU == 1) {   // sigma_2
            h.h[0][a] = p.s[0][a] - sgn_mul<S>(p.s[3][a]);
            h.h[1][a] = p.s[1][a] + sgn_mul<S>(p.s[2][a]);
        } else if (NU == 2) {   // sigma_3
            h.h[0][a] = p.s[0][a] - sgn_mul<S>(times_i(p.s[2][a]));
            h.h[1][a] = p.s[1][a] + sgn_mul<S>(times_i(p.s[3][a]));
        } else {                // gamma_4
            h.h[0][a] = p.s[0][a] + sgn_mul<S>(p.s[2][a]);
            h.h[1][a] = p.s[1][a] + sgn_mul<S>(p.s[3][a]);
        }
    }
}

// acc += coef * (full spinor reconstructed from the half spinor h)
template <int NU, int S, class R>
OVL_HD void recon_acc(Spinor<R>& acc, const Half<R>& h, R coef) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<R> h0 = coef * h.h[0][a], h1 = coef * h.h[1][a];
        acc.s[0][a] = acc.s[0][a] + h0;
        acc.s[1][a] = acc.s[1][a] + h1;
        if (NU == 0) {
            acc.s[2][a] = acc.s[2][a] + sgn_mul<S>(times_i(h1));
            acc.s[3][a] = acc.s[3][a] + sgn_mul<S>(times_i(h0));
        } else if (NU == 1) {
            acc.s[2][a] = acc.s[2][a] + sgn_mul<S>(h1);
            acc.s[3][a] = acc.s[3][a] - sgn_mul<S>(h0);
        } else if (NU == 2) {
            acc.s[2][a] = acc.s[2][a] + sgn_mul<S>(times_i(h0));
            acc.s[3][a] = acc.s[3][a] - sgn_mul<S>(times_i(h1));
        } else {
            acc.s[2][a] = acc.s[2][a] + sgn_mul<S>(h0);
            acc.s[3][a] = acc.s[3][a] + sgn_mul<S>(h1);
        }
    }
}

// SU(3) link as a full 3x3 matrix
template <class R> struct Link { cx<R> u[3][3]; };

// out = U h  (both half-spinor spins)
template <class R>
OVL_HD void mul_link(const Link<R>& U, const Half<R>& h, Half<R>& o) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> z = U.u[a][0] * h.h[s][0];
            cfma(z, U.u[a][1], h.h[s][1]);
            cfma(z, U.u[a][2], h.h[s][2]);
            o.h[s][a] = z;
        }
}
// out = U^dag h
template <class R>
OVL_HD void mul_link_dag(const Link<R>& U, const Half<R>& h, Half<R>& o) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> z = cdot(U.u[0][a], h.h[s][0]);
            cfmac(z, U.u[1][a], h.h[s][1]);
            cfmac(z, U.u[2][a], h.h[s][2]);
            o.h[s][a] = z;
        }
}

// third row of an SU(3) matrix from its first two rows: u2 = conj(u0 x u1)
template <class R>
OVL_HD void reconstruct_row2(Link<R>& U) {
    U.u[2][0] = conj(U.u[0][1] * U.u[1][2] - U.u[0][2] * U.u[1][1]);
    U.u[2][1] = conj(U.u[0][2] * U.u[1][0] - U.u[0][0] * U.u[1][2]);
    U.u[2][2] = conj(U.u[0][0] * U.u[1][1] - U.u[0][1] * U.u[1][0]);
}

// ------------------------------------------------------------ field access --
// FP64 spinor: double2 x[c][V], c = 3*spin + colour.
// FP32 spinor: float4 x[c2][V] holding components (2*c2, 2*c2+1).
// FP64 links: double2 U[nu][e][V], e = 3*row + col.
// FP32 12-real links: float4 U[nu][q][V], rows 0,1 = (u00,u01),(u02,u10),(u11,u12).
// FP32 18-real links: float2 U[nu][e][V].
// Double-float links (df32.cuh): float4 U[nu][e][V] = {re.hi, re.lo, im.hi, im.lo}.
enum LinkFmt { LINK_F64 = 0, LINK_F32_12 = 1, LINK_F32_18 = 2, LINK_DF = 3 };

__device__ __forceinline__ void load_spinor(const double2* __restrict__ x, int V, int i, Spinor<double>& p) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 v = __ldg(x + (size_t)c * V + i);
        p.s[c / 3][c % 3] = mk(v.x, v.y);
    }
}
__device__ __forceinline__ void load_spinor(const float4* __restrict__ x, int V, int i, Spinor<float>& p) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float4 v = __ldg(x + (size_t)c * V + i);
        p.s[(2 * c) / 3][(2 * c) % 3] = mk(v.x, v.y);
        p.s[(2 * c + 1) / 3][(2 * c + 1) % 3] = mk(v.z, v.w);
    }
}
__device__ __forceinline__ void store_spinor(double2* __restrict__ x, int V, int i, const Spinor<double>& p) {
#pragma unroll
    for (int c = 0; c < 12; ++c) x[(size_t)c * V + i] = make_double2(p.s[c / 3][c % 3].r, p.s[c / 3][c % 3].i);
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ x, int V, int i, const Spinor<float>& p) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        cx<float> a = p.s[(2 * c) / 3][(2 * c) % 3], b = p.s[(2 * c + 1) / 3][(2 * c + 1) % 3];
        x[(size_t)c * V + i] = make_float4(a.r, a.i, b.r, b.i);
    }
}

// L2-coherent variants (ld.global.cg) for vectors that other blocks of the same
// kernel write (persistent kernels): the read-only and L1 paths may hold stale lines.
__device__ __forceinline__ void load_spinor_cg(const double2* x, int V, int i, Spinor<double>& p) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 v = __ldcg(x + (size_t)c * V + i);
        p.s[c / 3][c % 3] = mk(v.x, v.y);
    }
}
__device__ __forceinline__ void load_spinor_cg(const float4* x, int V, int i, Spinor<float>& p) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float4 v = __ldcg(x + (size_t)c * V + i);
        p.s[(2 * c) / 3][(2 * c) % 3] = mk(v.x, v.y);
        p.s[(2 * c + 1) / 3][(2 * c + 1) % 3] = mk(v.z, v.w);
    }
}

__device__ __forceinline__ void load_link(const double2* __restrict__ U, int V, int nu, int i, Link<double>& L) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        double2 v = __ldg(U + ((size_t)nu * 9 + e) * V + i);
        L.u[e / 3][e % 3] = mk(v.x, v.y);
    }
}
__device__ __forceinline__ void load_link12(const float4* __restrict__ U, int V, int nu, int i, Link<float>& L) {
    float4 a = __ldg(U + ((size_t)nu * 3 + 0) * V + i);
    float4 b = __ldg(U + ((size_t)nu * 3 + 1) * V + i);
    float4 c = __ldg(U + ((size_t)nu * 3 + 2) * V + i);
    L.u[0][0] = mk(a.x, a.y); L.u[0][1] = mk(a.z, a.w);
    L.u[0][2] = mk(b.x, b.y); L.u[1][0] = mk(b.z, b.w);
    L.u[1][1] = mk(c.x, c.y); L.u[1][2] = mk(c.z, c.w);
    reconstruct_row2(L);
}
__device__ __forceinline__ void load_link18(const float2* __restrict__ U, int V, int nu, int i, Link<float>& L) {
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        float2 v = __ldg(U + ((size_t)nu * 9 + e) * V + i);
        L.u[e / 3][e % 3] = mk(v.x, v.y);
    }
}

// ------------------------------------------------------------- reductions --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV doubles over the block; result valid in thread 0.  smem: 32*NV doubles (value j of warp w
// goes to smem[j * 32 + w]), whatever the block size.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) smem[j * 32 + wid] = v[j];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = lane < nw ? smem[j * 32 + lane] : 0.0;
            v[j] = warp_sum(t);
        }
    }
}

// Deterministic grid reduction: every block writes its NV partial sums to
// partials[j * gridDim.x + blockIdx.x]; the last block to finish (ticket
// counter) sums them in block order into out[0..NV) (thread 0) and resets the
// counter.  Returns true in the last block (all threads), where the caller
// may then run a finalisation step.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* partials, unsigned int* counter,
                                              double* out, double* smem, unsigned int blk, unsigned int nblk) {
    block_sum<NV>(v, smem);
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[(size_t)j * nblk + blk] = v[j];
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        last = (t == nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // sum partials in a fixed order: thread-strided then tree within block; the loads of UB
    // strides are issued together (NV x UB in flight per thread) and then added in the same order
    constexpr int UB = NV <= 2 ? 8 : 4;
    double acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.0;
    const unsigned int bs = blockDim.x;
    unsigned int b = threadIdx.x;
    for (; b + (UB - 1) * bs < nblk; b += UB * bs) {
        double x[NV][UB];
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int u = 0; u < UB; ++u) x[j][u] = __ldcg(partials + (size_t)j * nblk + b + u * bs);
#pragma unroll
        for (int j = 0; j < NV; ++j)
#pragma unroll
            for (int u = 0; u < UB; ++u) acc[j] += x[j][u];
    }
    for (; b < nblk; b += bs)
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] += __ldcg(partials + (size_t)j * nblk + b);
    block_sum<NV>(acc, smem);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] = acc[j];
        *counter = 0u;
    }
    __syncthreads();
    return true;
}
// the same over a one-dimensional grid (block blockIdx.x of gridDim.x)
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* partials, unsigned int* counter,
                                              double* out, double* smem) {
    return grid_sum_last<NV>(v, partials, counter, out, smem, blockIdx.x, gridDim.x);
}

// Bounded grid barrier for cooperative launches.  `bar` points to two
// unsigned ints (count, generation).  A wait that exceeds `max_spins` polls
// sets *err = code and continues, so the kernel always terminates.
__device__ __forceinline__ void grid_barrier(unsigned int* bar, int* err, int code, long long max_spins) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = bar + 1;
        unsigned int gen = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (++spins > max_spins) { atomicExch(err, code); break; }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Bounded grid barrier with a monotonic arrival counter (zeroed before the launch): the n-th
// barrier of a launch waits for G n arrivals, so no reset and no second atomic are needed.
// The arrival is a GPU-scope release and the poll a GPU-scope acquire: the block's writes
// before the barrier (ordered to thread 0 by __syncthreads) are visible to every block after it.
__device__ __forceinline__ void grid_barrier_mono(unsigned int* ctr, unsigned int target, int* err, int code,
                                                  long long max_spins) {
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
        long long spins = 0;
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if ((int)(v - target) >= 0) break;
            if (++spins > max_spins) {
                atomicExch(err, code);
                break;
            }
        }
    }
    __syncthreads();
}

}  // namespace ovl
