// Persistent forms of the two passes of the mixed-precision two-sided Lanczos
// solve (Sec. 4, Eq. 4.2; two-pass procedure of Sec. 5).
//
// On lattices that hold a few thousand sites per SM the per-step kernels are
// bound by launch gaps and dependent-load latency, not by work.  Here one
// cooperative launch runs all k steps: every block owns fixed 32-site tiles,
// computes the pair stencil for them (four warps = four directions), keeps
// t = A v_i and s = A^dag w_i in shared memory, and meets the other blocks at
// two bounded grid barriers per step -- after the partial sums of alpha (and
// of the re-projection coefficients L^dag t, R^dag s), and after those of
// w^^dag v^, |v^|^2, |w^|^2.  Every block then adds the per-block partial sums
// in the same fixed order, so all blocks hold identical coefficients without a
// further exchange.  Pass 2 regenerates the basis in FP64 with one barrier per
// step.  Vectors written by other blocks are read through L2 (ld.global.cg).
#include <algorithm>

#include "stencil_impl.cuh"

namespace ovl {

static constexpr int PT = 32;        // sites per tile
static constexpr int PW = 8;         // warps per block: one hop (4 directions x forward/backward) each
static constexpr int PMAX_M = 64;    // deflated vectors handled by re-projection
static constexpr long long PSPIN = 20000000;

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
    double* partA;       // [G][4 + 4m]
    double* partC;       // [G][4]
    unsigned int* bar;
    HopCoef<float> hv, hw;
    Geom g;
    int k;
    int ntiles;
};

// coef[q] = sum over blocks b of part[b * stride + q] for q < nq: warp w takes q = w, w + 4, ...,
// its lanes load blocks lane, lane + 32, ... in parallel, and the warp tree adds them in a fixed
// order, so every block obtains bit-identical sums.
__device__ __forceinline__ void sum_partials(const double* part, int stride, int nq, int G, double* coef) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = wid; q < nq; q += nw) {
        double acc = 0.0;
        for (int b = lane; b < G; b += 32) acc += __ldcg(part + (size_t)b * stride + q);
        acc = warp_sum(acc);
        if (lane == 0) coef[q] = acc;
    }
    __syncthreads();
}

// block-wide sum of a double held by every thread (result in every thread)
__device__ __forceinline__ double block_all_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q];
    return s;
}

__global__ void __launch_bounds__(256) k_pass1_persistent(P1Args a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<float>* dirpart = reinterpret_cast<cx<float>*>(smraw);                        // 8 x 2 x 32 x 12
    cx<float>* ts = dirpart + PW * 2 * PT * 12;                                        // tiles x 32 x 12 x 2
    __shared__ double red[PW];
    __shared__ double coef[4 + 4 * PMAX_M];
    KState* ks = a.ks;
    int* err = &ks->timeout;
    if (ks->done || ks->status) return;
    const Geom g = a.g;
    const int G = gridDim.x;
    const int tid = threadIdx.x, site = tid >> 2, sp = tid & 3;
    const int lane = tid & 31, wid = tid >> 5;
    const int m = a.m;
    const int NA = 4 + 4 * m;
    cx<double> sv = d2c(ks->sv), sw = d2c(ks->sw), svp = d2c(ks->svp), swp = d2c(ks->swp);
    double anorm = ks->anorm;
    cx<double> beta_prev = mk(0.0, 0.0), gamma_prev = mk(0.0, 0.0);
    int kused = 0, done = 0, bd = -1;
    for (int i = 0; i < a.k && !done; ++i) {
        const float4* vi = a.v[i % 3];
        const float4* wi = a.w[i % 3];
        // ---- phase A: t = sv A v~_i, s = sw A^dag w~_i on the own tiles (kept in smem)
        double pa[3] = {0.0, 0.0, 0.0};
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
            if (tid < 128 && ii < g.V) {
                const cx<float> csv = mk((float)sv.r, (float)sv.i), csw = mk((float)sw.r, (float)sw.i);
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    const int q = 3 * sp + c3;
                    cx<float> tv = ld_comp_cg<float>(vi, g.V, ii, q), sq = ld_comp_cg<float>(wi, g.V, ii, q);
                    const cx<float> wq = sq;
#pragma unroll
                    for (int w4 = 0; w4 < PW; ++w4) {
                        tv = tv + dirpart[((w4 * 2 + 0) * PT + site) * 12 + q];
                        sq = sq + dirpart[((w4 * 2 + 1) * PT + site) * 12 + q];
                    }
                    if (sp >= 2) {
                        tv = -tv;
                        sq = -sq;
                    }
                    tv = csv * tv;
                    sq = csw * sq;
                    ts[((jt * PT + site) * 12 + q) * 2 + 0] = tv;
                    ts[((jt * PT + site) * 12 + q) * 2 + 1] = sq;
                    const cx<double> z = cdot(up(wq), up(tv));
                    pa[0] += z.r;
                    pa[1] += z.i;
                    pa[2] += norm2(up(tv));
                }
            }
            __syncthreads();
        }
        // per-block partials of alpha, |t|^2 and the re-projection coefficients
        {
            double s0 = block_all_sum(pa[0], red), s1 = block_all_sum(pa[1], red), s2 = block_all_sum(pa[2], red);
            if (tid == 0) {
                a.partA[(size_t)blockIdx.x * NA + 0] = s0;
                a.partA[(size_t)blockIdx.x * NA + 1] = s1;
                a.partA[(size_t)blockIdx.x * NA + 2] = s2;
                a.partA[(size_t)blockIdx.x * NA + 3] = 0.0;
            }
            for (int j = 0; j < m; ++j) {
                // p_j = l_j^dag t, q_j = r_j^dag s over the own sites (FP32 products)
                float pr = 0.f, pi = 0.f, qr = 0.f, qi = 0.f;
                int jt2 = 0;
                for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt2) {
                    const int ii = tile * PT + site;
                    if (tid >= 128 || ii >= g.V) continue;
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        const int q = 3 * sp + c3;
                        const cx<float> tv = ts[((jt2 * PT + site) * 12 + q) * 2 + 0];
                        const cx<float> sq = ts[((jt2 * PT + site) * 12 + q) * 2 + 1];
                        const cx<float> lj = ld_comp<float>(reinterpret_cast<const float4*>(a.L32 + (size_t)j * 12 * g.V), g.V, ii, q);
                        const cx<float> rj = ld_comp<float>(reinterpret_cast<const float4*>(a.R32 + (size_t)j * 12 * g.V), g.V, ii, q);
                        const cx<float> z1 = cdot(lj, tv), z2 = cdot(rj, sq);
                        pr += z1.r;
                        pi += z1.i;
                        qr += z2.r;
                        qi += z2.i;
                    }
                }
                const double d0 = block_all_sum(pr, red), d1 = block_all_sum(pi, red);
                const double d2 = block_all_sum(qr, red), d3 = block_all_sum(qi, red);
                if (tid == 0) {
                    double* pb = a.partA + (size_t)blockIdx.x * NA + 4;
                    pb[2 * j] = d0;
                    pb[2 * j + 1] = d1;
                    pb[2 * m + 2 * j] = d2;
                    pb[2 * m + 2 * j + 1] = d3;
                }
            }
        }
        grid_barrier(a.bar, err, 1, PSPIN);
        if (*(volatile int*)err) return;
        sum_partials(a.partA, NA, NA, G, coef);
        const cx<double> alpha = cdot(sw, mk(coef[0], coef[1]));
        anorm = fmax(anorm, sqrt(coef[2]));
        kused = i + 1;
        if (blockIdx.x == 0 && tid == 0) a.alpha[i] = c2d(alpha);
        if (i == a.k - 1) break;
        // ---- phase C: the recurrence on the own sites, reductions for beta, gamma
        const cx<double> ca = alpha * sv, da = conj(alpha) * sw;
        const cx<double> cg = i > 0 ? gamma_prev * svp : mk(0.0, 0.0);
        const cx<double> db = i > 0 ? conj(beta_prev) * swp : mk(0.0, 0.0);
        const cx<float> ca_ = mk((float)ca.r, (float)ca.i), da_ = mk((float)da.r, (float)da.i);
        const cx<float> cg_ = mk((float)cg.r, (float)cg.i), db_ = mk((float)db.r, (float)db.i);
        const float4* vim1 = a.v[(i + 2) % 3];
        const float4* wim1 = a.w[(i + 2) % 3];
        float4* vn = a.v[(i + 1) % 3];
        float4* wn = a.w[(i + 1) % 3];
        double pc[4] = {0.0, 0.0, 0.0, 0.0};
        jt = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G, ++jt) {
            const int ii = tile * PT + site;
            if (tid >= 128 || ii >= g.V) continue;
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                const int q = 3 * sp + c3;
                cx<float> v = ts[((jt * PT + site) * 12 + q) * 2 + 0] - ca_ * ld_comp_cg<float>(vi, g.V, ii, q);
                cx<float> w = ts[((jt * PT + site) * 12 + q) * 2 + 1] - da_ * ld_comp_cg<float>(wi, g.V, ii, q);
                if (i > 0) {
                    v = v - cg_ * ld_comp_cg<float>(vim1, g.V, ii, q);
                    w = w - db_ * ld_comp_cg<float>(wim1, g.V, ii, q);
                }
                for (int j = 0; j < m; ++j) {
                    const cx<float> pj = mk((float)coef[4 + 2 * j], (float)coef[4 + 2 * j + 1]);
                    const cx<float> qj = mk((float)coef[4 + 2 * m + 2 * j], (float)coef[4 + 2 * m + 2 * j + 1]);
                    v = v - pj * ld_comp<float>(reinterpret_cast<const float4*>(a.R32 + (size_t)j * 12 * g.V), g.V, ii, q);
                    w = w - qj * ld_comp<float>(reinterpret_cast<const float4*>(a.L32 + (size_t)j * 12 * g.V), g.V, ii, q);
                }
                st_comp<float>(vn, g.V, ii, q, v);
                st_comp<float>(wn, g.V, ii, q, w);
                const cx<double> vd = up(v), wd = up(w);
                const cx<double> z = cdot(wd, vd);
                pc[0] += z.r;
                pc[1] += z.i;
                pc[2] += norm2(vd);
                pc[3] += norm2(wd);
            }
        }
        {
            double s0 = block_all_sum(pc[0], red), s1 = block_all_sum(pc[1], red);
            double s2 = block_all_sum(pc[2], red), s3 = block_all_sum(pc[3], red);
            if (tid == 0) {
                a.partC[(size_t)blockIdx.x * 4 + 0] = s0;
                a.partC[(size_t)blockIdx.x * 4 + 1] = s1;
                a.partC[(size_t)blockIdx.x * 4 + 2] = s2;
                a.partC[(size_t)blockIdx.x * 4 + 3] = s3;
            }
        }
        grid_barrier(a.bar, err, 1, PSPIN);
        if (*(volatile int*)err) return;
        __shared__ double oc[4];
        sum_partials(a.partC, 4, 4, G, oc);
        const double o[4] = {oc[0], oc[1], oc[2], oc[3]};
        const double nv = sqrt(o[2]), nw = sqrt(o[3]);
        const cx<double> delta = mk(o[0], o[1]);
        if (nv <= 1e-13 * fmax(anorm, 1e-300)) {
            done = 1;  // lucky breakdown
        } else if (sqrt(norm2(delta)) <= 1e-14 * nv * nw) {
            done = 1;  // serious breakdown
            bd = i + 1;
        } else {
            const cx<double> gm = mk(o[0] / nv, o[1] / nv);
            beta_prev = mk(nv, 0.0);
            gamma_prev = gm;
            if (blockIdx.x == 0 && tid == 0) {
                a.beta[i] = c2d(beta_prev);
                a.gamma[i] = c2d(gm);
            }
            svp = sv;
            swp = sw;
            sv = mk(1.0 / nv, 0.0);
            sw = cdiv(mk(1.0, 0.0), conj(gm));
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        ks->kused = kused;
        ks->done = 1;
        ks->anorm = anorm;
        if (bd >= 0) ks->bdstep = bd;
        ks->sv = c2d(sv);
        ks->sw = c2d(sw);
        ks->svp = c2d(svp);
        ks->swp = c2d(swp);
    }
}

struct P2Args {
    const double2* U;
    double2* v[3];
    double2* y;
    const KState* ks;
    const double2* alpha;
    const double2* beta;
    const double2* gamma;
    const double2* c;
    unsigned int* bar;
    int* err;
    HopCoef<double> hc;
    Geom g;
    int ntiles;
};

// FP64 regeneration v_{i+1} = ((A - alpha_i) v_i - gamma_{i-1} v_{i-1}) / beta_i, y += c_{i+1} v_{i+1}
__global__ void __launch_bounds__(256) k_pass2_persistent(P2Args a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<double>* dirpart = reinterpret_cast<cx<double>*>(smraw);  // 8 x 32 x 12
    if (a.ks->status) return;
    const int kused = a.ks->kused;
    const Geom g = a.g;
    const int G = gridDim.x;
    const int tid = threadIdx.x, site = tid >> 2, sp = tid & 3;
    const int lane = tid & 31, wid = tid >> 5;
    for (int i = 0; i + 1 < kused; ++i) {
        const double2* vi = a.v[i % 3];
        const double2* vim1 = a.v[(i + 2) % 3];
        double2* vn = a.v[(i + 1) % 3];
        const cx<double> al = d2c(a.alpha[i]);
        const cx<double> ib = cdiv(mk(1.0, 0.0), d2c(a.beta[i]));
        const cx<double> gm = i > 0 ? d2c(a.gamma[i - 1]) : mk(0.0, 0.0);
        const cx<double> cc = d2c(a.c[i + 1]);
        for (int tile = blockIdx.x; tile < a.ntiles; tile += G) {
            {
                const int i0 = tile * PT + lane;
                Spinor<double> acc[1];
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[0].s[s][c] = mk(0.0, 0.0);
                if (i0 < g.V) {
                    const Coord c = site_coord(g, i0);
                    const double2* const xs[1] = {vi};
                    const HopCoef<double> hcs[1] = {a.hc};
                    one_hop<LINK_F64, double, 1, true>(wid, g, c, i0, a.U, xs, acc, hcs);
                }
#pragma unroll
                for (int q = 0; q < 12; ++q) dirpart[(wid * PT + lane) * 12 + q] = acc[0].s[q / 3][q % 3];
            }
            __syncthreads();
            const int ii = tile * PT + site;
            if (tid < 128 && ii < g.V) {
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    const int q = 3 * sp + c3;
                    const size_t e = (size_t)q * g.V + ii;
                    const cx<double> self = d2c(__ldcg(vi + e));
                    cx<double> z = self;
#pragma unroll
                    for (int w4 = 0; w4 < PW; ++w4) z = z + dirpart[(w4 * PT + site) * 12 + q];
                    if (sp >= 2) z = -z;
                    z = z - al * self;
                    if (i > 0) z = z - gm * d2c(__ldcg(vim1 + e));
                    z = ib * z;
                    vn[e] = c2d(z);
                    cx<double> yy = d2c(a.y[e]);
                    cfma(yy, cc, z);
                    a.y[e] = c2d(yy);
                }
            }
            __syncthreads();
        }
        grid_barrier(a.bar, a.err, 1, PSPIN);
        if (*(volatile int*)a.err) return;
    }
}

static int persistent_grid(int ntiles, int num_sms) { return std::max(1, std::min(ntiles, num_sms)); }

size_t pass1_partials_doubles(int num_sms, int m) { return (size_t)num_sms * (8 + 4 * m) + 16; }

bool persistent_ok(const Geom& g, int num_sms) {
    // tiles per block small enough for the shared-memory copy of t and s
    const int ntiles = (g.V + PT - 1) / PT;
    const int tpb = (ntiles + num_sms - 1) / num_sms;
    return tpb <= 16;
}

int launch_pass1_persistent(const float4* U12, float4* const v[3], float4* const w[3], KState* ks, double2* alpha,
                            double2* beta, double2* gamma, const float2* R32, const float2* L32, int m, double mu,
                            double kappa, int k, double* partials, unsigned int* bar, const Geom& g, int num_sms,
                            cudaStream_t st) {
    if (m > PMAX_M) return -1;
    P1Args a;
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
    a.partA = partials;
    a.partC = partials + (size_t)G * (4 + 4 * m);
    a.bar = bar;
    a.hv = make_coef<float>(mu, kappa);
    a.hw = make_coef<float>(-mu, kappa);
    a.g = g;
    a.k = k;
    const int tpb = (a.ntiles + G - 1) / G;
    const size_t smem = sizeof(cx<float>) * (PW * 2 * PT * 12 + (size_t)tpb * PT * 12 * 2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pass1_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(32 * PW);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_pass1_persistent, a);
}

int launch_pass2_persistent(const double2* U64, double2* const v[3], double2* y, const KState* ks,
                            const double2* alpha, const double2* beta, const double2* gamma, const double2* c,
                            double mu, double kappa, unsigned int* bar, int* err, const Geom& g, int num_sms,
                            cudaStream_t st) {
    P2Args a;
    a.U = U64;
    for (int q = 0; q < 3; ++q) a.v[q] = v[q];
    a.y = y;
    a.ks = ks;
    a.alpha = alpha;
    a.beta = beta;
    a.gamma = gamma;
    a.c = c;
    a.bar = bar;
    a.err = err;
    a.hc = make_coef<double>(mu, kappa);
    a.g = g;
    a.ntiles = (g.V + PT - 1) / PT;
    const int G = persistent_grid(a.ntiles, num_sms);
    const size_t smem = sizeof(cx<double>) * PW * PT * 12;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pass2_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(32 * PW);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_pass2_persistent, a);
}

}  // namespace ovl
