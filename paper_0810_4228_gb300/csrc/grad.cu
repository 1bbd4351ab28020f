// Adjoint of y = A x, A = gamma5 D_w(mu; U) (Sec. 1, Eq. 1.2), for gradients of a
// real function l of y, in PyTorch's convention for complex tensors: the gradient
// of a complex z is g_z = dl/dRe z + i dl/dIm z (= 2 dl/dz*), so dl = Re <g_z, dz>
// with <a, b> = a^dag b.  With g = g_y:
//   grad_x        = A^dag g = gamma5 D_w(-mu) g                  (the stencil itself)
//   grad_U[x,nu]  = g_U
//                 = -kappa ( c+ ph sum_s g~_s (x) conj(psi(x+nu)_s)
//                          + c- ph sum_s psi(x)_s (x) conj(g^_s) ),
//        g~ = (1 + gamma_nu) gamma5 g(x),  g^ = (1 - gamma_nu) gamma5 g(x+nu),
//        (a (x) conj(b))_ij = a_i conj(b_j) in colour, c+- = e^{+-mu} for nu = 4
//        (1 otherwise), ph the antiperiodic phase of a hop across the time edge;
//   dl/dmu        = Re <g, (dA/dmu) x>,  dA/dmu = -kappa gamma5 (e^mu T_4^+ - e^-mu T_4^-).
// Every link receives the forward hop of its own site and the backward hop of
// the site it points to.  One thread per site, canonical layouts in and out.
#include "ctx.h"
#include "stencil_impl.cuh"

namespace ovl {
namespace {

// canonical spinor access: psi[s][12]
__device__ __forceinline__ void load_canon(const double2* __restrict__ p, int s, Spinor<double>& o) {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const double2 v = p[(size_t)s * 12 + q];
        o.s[q / 3][q % 3] = mk(v.x, v.y);
    }
}

// (1 + S gamma_nu) gamma5 g as a full spinor
template <int NU, int S, class R>
__device__ __forceinline__ void proj_g5(const Spinor<R>& g, Spinor<R>& o) {
    Spinor<R> g5 = g;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g5.s[2][a] = -g.s[2][a];
        g5.s[3][a] = -g.s[3][a];
    }
    Half<R> h;
    project<NU, S>(g5, h);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) o.s[sp][a] = mk(R(0), R(0));
    recon_acc<NU, S>(o, h, R(1));
}

// canonical spinor in precision R
template <class R>
__device__ __forceinline__ void load_canon_r(const double2* __restrict__ p, int s, Spinor<R>& o) {
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const double2 v = p[(size_t)s * 12 + q];
        o.s[q / 3][q % 3] = mk((R)v.x, (R)v.y);
    }
}

// (R = float: the FP32 form of OVL_F32, every product and sum in FP32)
template <int NU, class R>
__device__ __forceinline__ void link_grad(const Geom& g, const Coord& c, int s, const double2* __restrict__ x,
                                          const double2* __restrict__ gr, double2* __restrict__ gU, double cf,
                                          double cb) {
    int y[4] = {c.x[0], c.x[1], c.x[2], c.x[3]};
    y[NU] = (y[NU] + 1) % g.L[NU];
    const int sf = canon_index(g, y);
    const R ph = (NU == 3 && c.x[3] == g.L[3] - 1) ? (R)g.bc_t : R(1);
    Spinor<R> gx, gy, px, py, gt, gh;
    load_canon_r(gr, s, gx);
    load_canon_r(gr, sf, gy);
    load_canon_r(x, s, px);
    load_canon_r(x, sf, py);
    proj_g5<NU, +1>(gx, gt);
    proj_g5<NU, -1>(gy, gh);
    const R af = -(R)cf * ph, ab = -(R)cb * ph;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<R> z = mk(R(0), R(0));
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
                z = z + af * cdot(py.s[sp][j], gt.s[sp][i]);  // g~_i conj(psi(x+nu)_j)
                z = z + ab * cdot(gh.s[sp][j], px.s[sp][i]);  // psi(x)_i conj(g^_j)
            }
            gU[((size_t)s * 4 + NU) * 9 + 3 * i + j] = make_double2((double)z.r, (double)z.i);
        }
}

template <class R>
__global__ void __launch_bounds__(128) k_dw_grad(const double2* __restrict__ U, const double2* __restrict__ x,
                                                 const double2* __restrict__ gr, double2* __restrict__ gU,
                                                 double kappa, double mu, Geom g, double* partials,
                                                 unsigned int* counter, double* gmu) {
    __shared__ double red[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double part[1] = {0.0};
    if (s < g.V) {
        Coord c;
        {
            int r = s;
            c.x[3] = r % g.L[3];
            r /= g.L[3];
            c.x[2] = r % g.L[2];
            r /= g.L[2];
            c.x[1] = r % g.L[1];
            c.x[0] = r / g.L[1];
            c.par = (c.x[0] + c.x[1] + c.x[2] + c.x[3]) & 1;
        }
        if (gU) {
            link_grad<0, R>(g, c, s, x, gr, gU, kappa, kappa);
            link_grad<1, R>(g, c, s, x, gr, gU, kappa, kappa);
            link_grad<2, R>(g, c, s, x, gr, gU, kappa, kappa);
            link_grad<3, R>(g, c, s, x, gr, gU, kappa * exp(mu), kappa * exp(-mu));
        }
        // Re <g, dA/dmu x> at this site: the temporal hops with e^mu and -e^-mu
        const int i = internal_index(g, c.x);
        Spinor<double> acc, xs;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc.s[sp][a] = mk(0.0, 0.0);
        Link<double> L;
        Spinor<double> p;
        Half<double> h, uh;
        int y[4] = {c.x[0], c.x[1], c.x[2], c.x[3]};
        y[3] = (c.x[3] + 1) % g.L[3];
        load_canon(x, canon_index(g, y), p);
        const double phf = (c.x[3] == g.L[3] - 1) ? (double)g.bc_t : 1.0;
        load_link(U, g.V, 3, i, L);
        project<3, +1>(p, h);
        mul_link(L, h, uh);
        recon_acc<3, +1>(acc, uh, -kappa * exp(mu) * phf);
        y[3] = (c.x[3] - 1 + g.L[3]) % g.L[3];
        load_canon(x, canon_index(g, y), p);
        const double phb = (c.x[3] == 0) ? (double)g.bc_t : 1.0;
        load_link(U, g.V, 3, internal_index(g, y), L);
        project<3, -1>(p, h);
        mul_link_dag(L, h, uh);
        recon_acc<3, -1>(acc, uh, kappa * exp(-mu) * phb);
        load_canon(gr, s, xs);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const cx<double> e = sp >= 2 ? -acc.s[sp][a] : acc.s[sp][a];
                part[0] += cdot(xs.s[sp][a], e).r;
            }
    }
    double out[1];
    if (grid_sum_last<1>(part, partials, counter, out, red))
        if (threadIdx.x == 0) *gmu = out[0];
}

}  // namespace
}  // namespace ovl

using namespace ovl_priv;

extern "C" int ovl_dw_grad(ovl_ctx* c, double mu, double kappa, const void* x, const void* g, void* grad_U,
                           double* grad_mu, int flags) {
    if (!c || !x || !g) return fail(c, OVL_EINVAL, "null argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    if (flags & OVL_HOST) return fail(c, OVL_EINVAL, "device pointers only");
    if (flags & ~OVL_F32) return fail(c, OVL_EINVAL, "flags: 0 or OVL_F32");
    int r = ensure_solve(c, std::max(c->kcap, 1));
    if (r) return r;
    double* gmu = reinterpret_cast<double*>(c->h2);
    const int T = 128, B = (c->g.V + T - 1) / T;
    if (flags & OVL_F32)
        ovl::k_dw_grad<float><<<B, T, 0, c->st>>>(c->U64, (const double2*)x, (const double2*)g, (double2*)grad_U,
                                                  kappa, mu, c->g, c->partials, c->counter, gmu);
    else
        ovl::k_dw_grad<double><<<B, T, 0, c->st>>>(c->U64, (const double2*)x, (const double2*)g, (double2*)grad_U,
                                                   kappa, mu, c->g, c->partials, c->counter, gmu);
    OVL_CUDA_TRY(c, cudaGetLastError());
    if (grad_mu) {
        OVL_CUDA_TRY(c, cudaMemcpyAsync(grad_mu, gmu, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        OVL_CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
    return OVL_OK;
}
