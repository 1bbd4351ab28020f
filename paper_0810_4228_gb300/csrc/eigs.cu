// Deflation phase on the GPU: the critical left and right eigenpairs of
// A = gamma5 D_w(mu) needed by LR deflation (Sec. 3, Eq. 3.1), computed once
// per gauge field and mu for all sources (Sec. 3, last paragraph; Sec. 5 uses
// ARPACK on the CPU for this step).
//
// Method: Chebyshev-filtered subspace iteration on T = A^2.  The eigenvalues of
// A nearest 0 are the smallest of T = A^2, which for gamma5 D_w(mu) at moderate
// mu lie close to the positive real axis; a degree-d Chebyshev polynomial of T
// on [a, b] (a = the largest Ritz value of T in the current block, b an upper
// bound of |T|) damps everything above a and amplifies the wanted end.  Each
// iteration filters the block, orthonormalises it (classical Gram-Schmidt
// twice) and performs a Rayleigh-Ritz projection with A itself, whose small
// dense eigenproblem is solved on the host (host_eig.cpp).  Ritz vectors of
// A^dag = gamma5 D_w(-mu) give the left eigenvectors; pairs are matched by
// lambda_left = conj(lambda_right), the m of smallest |Re lambda| are kept and
// bi-orthonormalised (L <- L (L^dag R)^-H) when installed.
// All vector work runs in the library's kernels; only nb x nb matrices visit
// the host.  Not on the timed path (the paper excludes the deflation phase
// from its timings, Sec. 5).
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace ovl {
int host_eig(int n, std::vector<std::complex<double>>& A, std::vector<std::complex<double>>& w,
             std::vector<std::complex<double>>& X);
}

using namespace ovl_priv;
using ovl::cx;
using ovl::KState;

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// deterministic pseudo-random start block, entries uniform in [-1, 1) + i [-1, 1)
__global__ void k_rand_fill(double2* x, size_t n, unsigned long long seed) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long a = mix64(seed ^ (2 * e)), b = mix64(seed ^ (2 * e + 1));
        x[e] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
    }
}

// Chebyshev step: ynext = s1 * (u - c y) - s0 * yprev   (s0 = 0 on the first step)
// (u and yn may be the same buffer: every element is read before it is written)
__global__ void k_cheb(const double2* u, const double2* y, const double2* yp, double2* yn, double c, double s1,
                       double s0, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 uu = u[e], yy = y[e];
        double2 r = make_double2(s1 * (uu.x - c * yy.x), s1 * (uu.y - c * yy.y));
        if (s0 != 0.0) {
            const double2 pp = yp[e];
            r.x -= s0 * pp.x;
            r.y -= s0 * pp.y;
        }
        yn[e] = r;
    }
}

// y <- y / sqrt(h.x)   (h = y^dag y from a preceding dot product)
__global__ void k_normalize(double2* y, const double2* h, size_t n) {
    const double inv = 1.0 / sqrt(fmax(h->x, 1e-300));
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 v = y[e];
        y[e] = make_double2(v.x * inv, v.y * inv);
    }
}

// |t - theta x|^2 -> ks->red[0].x
__global__ void __launch_bounds__(256) k_resid(const double2* __restrict__ t, const double2* __restrict__ x,
                                               double2 theta, KState* ks, double* partials, unsigned int* counter,
                                               size_t n) {
    __shared__ double red[32];
    double part[1] = {0.0};
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 a = t[e], b = x[e];
        const double rr = a.x - (theta.x * b.x - theta.y * b.y), ri = a.y - (theta.x * b.y + theta.y * b.x);
        part[0] += rr * rr + ri * ri;
    }
    double out[1];
    if (ovl::grid_sum_last<1>(part, partials, counter, out, red))
        if (threadIdx.x == 0) ks->red[0] = make_double2(out[0], 0.0);
}

int grid_n(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 1024); }

struct EigRun {
    std::vector<std::complex<double>> theta;  // Ritz values (all nb)
    std::vector<double> resid;
    int iterations = 0;
    long long matvecs = 0;
    double acut = 0;
};

// One side (dagger = 0: A, 1: A^dag): Ritz pairs of the nb-block, the first
// `want` (smallest |theta|) converged to tol; vectors left in X (nb x n).
int subspace_iteration(ovl_ctx* c, double mu, double kappa, int dagger, int want, int nb, double tol, int degree,
                       int maxit, double2* X, double2* Y, double2* tmp3, EigRun& run) {
    const size_t n = c->n;
    cudaStream_t st = c->st;
    const double m_eff = dagger ? -mu : mu;
    double2* t0 = tmp3;
    double2* t1 = tmp3 + n;
    double2* t2 = tmp3 + 2 * n;
    auto applyA = [&](const double2* x, double2* y) {
        ovl::launch_dslash(c->U64, 0, x, y, m_eff, kappa, 1, c->g, st);
        ++run.matvecs;
    };
    // upper bound of |A|^2 by power iteration on A^dag A
    k_rand_fill<<<grid_n(n), 256, 0, st>>>(t0, n, 0x5eedull + dagger);
    double2* h = c->h1;
    double sig2 = 0.0;
    for (int it = 0; it < 30; ++it) {
        ovl::launch_multidot(t0, n, 1, t0, h, 0, c->partials, n, st);
        k_normalize<<<grid_n(n), 256, 0, st>>>(t0, h, n);
        applyA(t0, t1);
        ovl::launch_dslash(c->U64, 0, t1, t2, -m_eff, kappa, 1, c->g, st);  // A^dag
        ++run.matvecs;
        ovl::launch_multidot(t0, n, 1, t2, h, 0, c->partials, n, st);
        double2 hv;
        OVL_CUDA_TRY(c, cudaMemcpyAsync(&hv, h, sizeof(double2), cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
        sig2 = std::max(sig2, hv.x);
        std::swap(t0, t2);
    }
    t0 = tmp3, t1 = tmp3 + n, t2 = tmp3 + 2 * n;
    const double bup = 1.15 * sig2;
    double acut = bup / 20.0;
    // random start block
    for (int j = 0; j < nb; ++j)
        k_rand_fill<<<grid_n(n), 256, 0, st>>>(X + (size_t)j * n, n, 0x1234ull * (j + 1) + 77 * dagger);
    std::vector<std::complex<double>> H((size_t)nb * nb), Hr((size_t)nb * nb), w, Z;
    double2* Hd = c->inner;  // nb*nb + nb*nb scratch
    double2* Zd = c->inner + (size_t)nb * nb;
    KState zero;
    std::memset(&zero, 0, sizeof(zero));
    OVL_CUDA_TRY(c, cudaMemcpyAsync(c->ks, &zero, sizeof(KState), cudaMemcpyHostToDevice, st));
    for (int iter = 0; iter < maxit; ++iter) {
        run.iterations = iter + 1;
        // filter every block vector: Y_j = p_d(A^2) X_j on [acut, bup]
        const double cc = 0.5 * (bup + acut), ee = 0.5 * (bup - acut);
        for (int j = 0; j < nb; ++j) {
            const double2* x = X + (size_t)j * n;
            double2 *yp = t0, *y = t1, *yn = t2;
            OVL_CUDA_TRY(c, cudaMemcpyAsync(yp, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            applyA(yp, Y + (size_t)j * n);
            applyA(Y + (size_t)j * n, y);  // y = A^2 x
            k_cheb<<<grid_n(n), 256, 0, st>>>(y, yp, nullptr, y, cc, 1.0 / ee, 0.0, n);
            for (int d = 1; d < degree; ++d) {
                applyA(y, Y + (size_t)j * n);
                applyA(Y + (size_t)j * n, yn);
                k_cheb<<<grid_n(n), 256, 0, st>>>(yn, y, yp, yn, cc, 2.0 / ee, 1.0, n);
                double2* tswap = yp;
                yp = y;
                y = yn;
                yn = tswap;
            }
            OVL_CUDA_TRY(c, cudaMemcpyAsync(Y + (size_t)j * n, y, n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            // classical Gram-Schmidt twice against Y_0..Y_{j-1}, then normalise
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                ovl::launch_multidot(Y, n, j, Y + (size_t)j * n, c->h2, 0, c->partials, n, st);
                ovl::launch_multiaxpy(Y, n, j, c->h2, Y + (size_t)j * n, c->partials, c->counter, c->ks, 0, n, st);
            }
            ovl::launch_multidot(Y + (size_t)j * n, n, 1, Y + (size_t)j * n, h, 0, c->partials, n, st);
            k_normalize<<<grid_n(n), 256, 0, st>>>(Y + (size_t)j * n, h, n);
        }
        // Rayleigh-Ritz with A: H = Y^dag A Y (column j = Y^dag (A y_j))
        for (int j = 0; j < nb; ++j) {
            applyA(Y + (size_t)j * n, t0);
            ovl::launch_multidot(Y, n, nb, t0, Hd + (size_t)j * nb, 0, c->partials, n, st);
        }
        OVL_CUDA_TRY(c, cudaMemcpyAsync(H.data(), Hd, sizeof(double2) * nb * nb, cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
        for (int i = 0; i < nb; ++i)
            for (int j = 0; j < nb; ++j) Hr[(size_t)i * nb + j] = H[i + (size_t)j * nb];
        if (ovl::host_eig(nb, Hr, w, Z) != 0) return fail(c, OVL_ENOCONV, "Rayleigh-Ritz eigensolver failed");
        // order Ritz pairs by |theta|
        std::vector<int> ord(nb);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return std::abs(w[a]) < std::abs(w[b]); });
        // X_j = sum_i Z[i][ord j] y_i
        std::vector<std::complex<double>> neg((size_t)nb * nb);
        for (int j = 0; j < nb; ++j)
            for (int i = 0; i < nb; ++i) neg[(size_t)j * nb + i] = -Z[(size_t)i * nb + ord[j]];
        OVL_CUDA_TRY(c, cudaMemcpyAsync(Zd, neg.data(), sizeof(double2) * nb * nb, cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(c, cudaMemsetAsync(X, 0, sizeof(double2) * n * nb, st));
        for (int j = 0; j < nb; ++j)
            ovl::launch_multiaxpy(Y, n, nb, Zd + (size_t)j * nb, X + (size_t)j * n, c->partials, c->counter, c->ks, 0,
                                  n, st);
        run.theta.assign(nb, 0.0);
        run.resid.assign(nb, 0.0);
        for (int j = 0; j < nb; ++j) run.theta[j] = w[ord[j]];
        // residuals of the wanted pairs
        double worst = 0.0;
        for (int j = 0; j < want; ++j) {
            applyA(X + (size_t)j * n, t0);
            const double2 th = make_double2(run.theta[j].real(), run.theta[j].imag());
            k_resid<<<grid_n(n), 256, 0, st>>>(t0, X + (size_t)j * n, th, c->ks, c->partials, c->counter, n);
            double2 rv;
            OVL_CUDA_TRY(c, cudaMemcpyAsync(&rv, &c->ks->red[0], sizeof(double2), cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
            run.resid[j] = std::sqrt(rv.x);
            worst = std::max(worst, run.resid[j]);
        }
        // next filter: damp everything above the largest Ritz value of A^2 in the block
        double amax = 0.0;
        for (int j = 0; j < nb; ++j) amax = std::max(amax, std::norm(run.theta[j]));
        acut = std::min(amax, bup / 4.0);
        run.acut = acut;
        if (worst <= tol * std::sqrt(sig2)) return OVL_OK;
    }
    return fail(c, OVL_ENOCONV, "deflation eigensolver did not converge");
}

}  // namespace

extern "C" int ovl_deflation_eigs(ovl_ctx* c, double mu, double kappa, int m, int nextra, double tol, int degree,
                                  int maxit, ovl_eiginfo* info) {
    if (!c || m < 1 || nextra < 0 || m + nextra > 512 || degree < 1 || maxit < 1 || !(tol > 0))
        return fail(c, OVL_EINVAL, "bad argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    const int want = m + nextra;
    const int nb = want + std::max(8, want / 2);
    int r = ensure_solve(c, std::max(c->kcap, 2 * nb + 2));
    if (r) return r;
    if (c->inner_elems < (size_t)2 * nb * nb) return fail(c, OVL_ENOMEM, "workspace too small");
    const size_t n = c->n;
    double2 *X = nullptr, *Y = nullptr, *T = nullptr, *XL = nullptr;
    auto cleanup = [&]() {
        if (X) cudaFree(X);
        if (Y) cudaFree(Y);
        if (T) cudaFree(T);
        if (XL) cudaFree(XL);
    };
    if (cudaMalloc(&X, sizeof(double2) * n * nb) != cudaSuccess || cudaMalloc(&Y, sizeof(double2) * n * nb) != cudaSuccess ||
        cudaMalloc(&T, sizeof(double2) * n * 3) != cudaSuccess || cudaMalloc(&XL, sizeof(double2) * n * nb) != cudaSuccess) {
        cleanup();
        return fail(c, OVL_ENOMEM, "eigensolver workspace");
    }
    EigRun right, left;
    r = subspace_iteration(c, mu, kappa, 0, want, nb, tol, degree, maxit, X, Y, T, right);
    if (!r) r = subspace_iteration(c, mu, kappa, 1, want, nb, tol, degree, maxit, XL, Y, T, left);
    if (r) {
        cleanup();
        return r;
    }
    // select the m right pairs of smallest |Re lambda| among the converged ones, pair with left
    std::vector<int> ord(want);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(),
              [&](int a, int b) { return std::fabs(right.theta[a].real()) < std::fabs(right.theta[b].real()); });
    std::vector<double> lam(2 * m);
    double2* Rsel = Y;  // reuse: m selected right vectors
    double2* Lsel = T;  // needs m vectors: reallocate if 3 < m
    if (m > 3) {
        cudaFree(T);
        T = nullptr;
        if (cudaMalloc(&T, sizeof(double2) * n * m) != cudaSuccess) {
            cleanup();
            return fail(c, OVL_ENOMEM, "eigensolver workspace");
        }
        Lsel = T;
    }
    double worst_pair = 0.0;
    for (int q = 0; q < m; ++q) {
        const int j = ord[q];
        const std::complex<double> l = right.theta[j];
        int best = -1;
        double bd = 1e300;
        for (int i = 0; i < want; ++i) {
            const double d = std::abs(std::conj(left.theta[i]) - l);
            if (d < bd) bd = d, best = i;
        }
        worst_pair = std::max(worst_pair, bd / std::max(std::abs(l), 1e-300));
        lam[2 * q] = l.real();
        lam[2 * q + 1] = l.imag();
        cudaMemcpyAsync(Rsel + (size_t)q * n, X + (size_t)j * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(Lsel + (size_t)q * n, XL + (size_t)best * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice,
                        c->st);
    }
    if (worst_pair > 1e-6) {
        cleanup();
        return fail(c, OVL_ENOCONV, "left and right eigenvalues do not pair up");
    }
    r = install_deflation(c, mu, kappa, m, lam.data(), Rsel, Lsel);
    cudaStreamSynchronize(c->st);
    if (info) {
        info->m = m;
        info->iterations = right.iterations + left.iterations;
        info->matvecs = right.matvecs + left.matvecs;
        double wr = 0.0;
        for (int q = 0; q < m; ++q) wr = std::max(wr, std::max(right.resid[ord[q]], 0.0));
        info->max_residual = wr;
        info->lambda_cut = std::sqrt(right.acut);
    }
    cleanup();
    return r;
}
