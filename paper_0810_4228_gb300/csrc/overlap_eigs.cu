// Eigenvalues of the overlap operator D_ov(mu) = 1 + gamma5 sgn(gamma5 D_w(mu)) (Sec. 1,
// Eq. 1.1) nearest 0: the application of the sign-function machinery that Sec. 5 names as the
// work to follow.  The paper gives no method for it; this is thick-restart Arnoldi with D_ov
// applied through the library's own sign solves (ovl_sign_krylov with OVL_OVERLAP: two-sided
// Lanczos or Arnoldi with the installed LR deflation, in the precision the caller chooses).
//
// Each cycle extends an orthonormal basis V to nkrylov vectors (one D_ov application per new
// vector, then classical Gram-Schmidt applied twice with the library's FP64 kernels), computes the
// Ritz pairs of the projected matrix H on the host (host_eig.cpp, nkrylov x nkrylov), and restarts
// from the orthonormalised Ritz vectors of the nev + keep Ritz values of smallest modulus and the
// last basis vector: with Q their coordinates, D_ov (V Q) = (V Q)(Q^dag H Q) + h v_next e^T Q
// keeps the Arnoldi relation with a full last row.  A Ritz pair (theta, V z) has the residual
// |h| |e^T z| (up to the sign solves' own error), the convergence test.  The converged
// eigenvectors are then formed, normalised, and checked with one more D_ov application each.
//
// The sign solves dominate: every D_ov application is a full Krylov solve of k steps.  Only
// nkrylov x nkrylov matrices visit the host.
#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "ctx.h"

namespace ovl {
int host_eig(int n, std::vector<std::complex<double>>& A, std::vector<std::complex<double>>& w,
             std::vector<std::complex<double>>& X);
}

using namespace ovl_priv;
using ovl::KState;

namespace {

using cd = std::complex<double>;

int grid_of(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 1024); }

// splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014): a counter-based hash for the start vector
__device__ __forceinline__ unsigned long long sm64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// x[e] = u1 + i u2, u1, u2 uniform in [-1, 1) from the hash of (seed, e)
__global__ void k_ov_fill(double2* x, size_t n, unsigned long long seed) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long a = sm64(seed ^ (2 * e)), b = sm64(seed ^ (2 * e + 1));
        x[e] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
    }
}

// x <- x / sqrt(h.x)   (h = x^dag x from a preceding dot product)
__global__ void k_ov_normalize(double2* x, const double2* h, size_t n) {
    const double inv = 1.0 / sqrt(fmax(h->x, 1e-300));
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 v = x[e];
        x[e] = make_double2(v.x * inv, v.y * inv);
    }
}

// r = y - theta x (for the residual check)
__global__ void k_ov_resid(const double2* __restrict__ y, const double2* __restrict__ x, double2 th,
                           double2* __restrict__ r, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 a = y[e], b = x[e];
        r[e] = make_double2(a.x - (th.x * b.x - th.y * b.y), a.y - (th.x * b.y + th.y * b.x));
    }
}

struct OvWork {
    double2* V;   // (nk + 1) basis vectors
    double2* W;   // nk vectors: rotation target
    double2* t0;  // one vector
    double2* Hd;  // (nk + 1) x nk, column-major
    double2* h1;  // nk + 2
    double2* h2;  // nk + 2
    double2* Qd;  // nk x nk coefficients
    double* part;
    KState* ks;
    unsigned int* counter;
};

// out_j = sum_l coef[l + j ld] V_l for j < nout (coefficients on the host, column-major)
int rotate(ovl_ctx* c, const OvWork& w, const double2* V, int nv, const std::vector<cd>& coef, int ld, int nout,
           double2* out) {
    const size_t n = c->n;
    cudaStream_t st = c->st;
    std::vector<cd> neg((size_t)nv * nout);
    for (int j = 0; j < nout; ++j)
        for (int l = 0; l < nv; ++l) neg[(size_t)j * nv + l] = -coef[(size_t)j * ld + l];
    OVL_CUDA_TRY(c, cudaMemcpyAsync(w.Qd, neg.data(), sizeof(double2) * nv * nout, cudaMemcpyHostToDevice, st));
    OVL_CUDA_TRY(c, cudaMemsetAsync(out, 0, sizeof(double2) * n * nout, st));
    for (int j = 0; j < nout; ++j)
        ovl::launch_multiaxpy(V, n, nv, w.Qd + (size_t)j * nv, out + (size_t)j * n, w.part, w.counter, w.ks, 0, n, st);
    OVL_CUDA_TRY(c, cudaStreamSynchronize(st));  // the coefficients are read before the next upload
    return OVL_OK;
}

// Columns of Q (ne x kk, column-major) made orthonormal: modified Gram-Schmidt, twice.
bool orthonormalise(std::vector<cd>& Q, int ne, int kk) {
    for (int i = 0; i < kk; ++i) {
        cd* qi = &Q[(size_t)i * ne];
        for (int pass = 0; pass < 2; ++pass)
            for (int l = 0; l < i; ++l) {
                const cd* ql = &Q[(size_t)l * ne];
                cd s = 0.0;
                for (int r = 0; r < ne; ++r) s += std::conj(ql[r]) * qi[r];
                for (int r = 0; r < ne; ++r) qi[r] -= s * ql[r];
            }
        double nn = 0.0;
        for (int r = 0; r < ne; ++r) nn += std::norm(qi[r]);
        nn = std::sqrt(nn);
        if (!(nn > 1e-300)) return false;
        for (int r = 0; r < ne; ++r) qi[r] /= nn;
    }
    return true;
}

}  // namespace

extern "C" int ovl_overlap_eigs(ovl_ctx* c, int method, int k, double mu, double kappa, int flags, int nev,
                                int nkrylov, double tol, int maxit, double* lambda, void* vecs,
                                ovl_ovinfo* info) {
    if (!c || !lambda || nev < 1 || k < 1 || maxit < 1 || !(tol > 0) || nkrylov < 0)
        return fail(c, OVL_EINVAL, "bad argument");
    if (method != OVL_ARNOLDI && method != OVL_LANCZOS2) return fail(c, OVL_EINVAL, "unknown method");
    if (flags & (OVL_HOST | OVL_PROFILE)) return fail(c, OVL_EINVAL, "flags: OVL_HOST and OVL_PROFILE do not apply");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    const size_t n = c->n;
    int nk = nkrylov > 0 ? nkrylov : std::max(2 * nev + 20, 40);
    nk = (int)std::min<size_t>((size_t)nk, n - 1);
    if (nk < nev + 2) return fail(c, OVL_EINVAL, "basis too small for the wanted eigenvalues");
    const int keep = std::max(4, (nk - nev) / 3);
    const int sflags = (flags | OVL_OVERLAP) & ~OVL_NO_GRAPH;
    cudaStream_t st = c->st;
    const int mdb = ovl::multidot_blocks(n);
    const size_t part_bytes = std::max<size_t>((size_t)mdb * (nk + 2) * sizeof(double2), (size_t)1 << 16);
    void* ptrs[10] = {};
    const size_t sizes[10] = {sizeof(double2) * n * (nk + 1), sizeof(double2) * n * nk, sizeof(double2) * n,
                              sizeof(double2) * (size_t)(nk + 1) * nk, sizeof(double2) * (nk + 2),
                              sizeof(double2) * (nk + 2), sizeof(double2) * (size_t)nk * nk, part_bytes,
                              sizeof(KState), 64};
    auto cleanup = [&]() {
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
    for (int i = 0; i < 10; ++i)
        if (cudaMalloc(&ptrs[i], sizes[i]) != cudaSuccess) {
            ptrs[i] = nullptr;
            cleanup();
            return fail(c, OVL_ENOMEM, "overlap eigensolver workspace");
        }
    OvWork w;
    w.V = (double2*)ptrs[0], w.W = (double2*)ptrs[1], w.t0 = (double2*)ptrs[2], w.Hd = (double2*)ptrs[3];
    w.h1 = (double2*)ptrs[4], w.h2 = (double2*)ptrs[5], w.Qd = (double2*)ptrs[6], w.part = (double*)ptrs[7];
    w.ks = (KState*)ptrs[8], w.counter = (unsigned int*)ptrs[9];
    long long nsolve = 0;
    int cycles = 0;
    // y = D_ov x through the sign solve; a failed solve ends the run with its status
    auto apply = [&](const double2* x, double2* y) -> int {
        ovl_info si;
        const int r = ovl_sign_krylov(c, method, k, mu, kappa, x, y, sflags, &si);
        ++nsolve;
        return r;
    };
    auto done = [&](int r) {
        if (info) {
            info->restarts = cycles;
            info->sign_solves = nsolve;
        }
        cleanup();
        return r;
    };
    if (cudaMemsetAsync(w.counter, 0, 64, st) != cudaSuccess || cudaMemsetAsync(w.ks, 0, sizeof(KState), st))
        return done(fail(c, OVL_ECUDA, "overlap eigensolver set-up"));
    k_ov_fill<<<grid_of(n), 256, 0, st>>>(w.V, n, 0x0e16ull);
    ovl::launch_multidot(w.V, n, 1, w.V, w.h1, 0, w.part, n, st);
    k_ov_normalize<<<grid_of(n), 256, 0, st>>>(w.V, w.h1, n);
    const int ldH = nk + 1;
    std::vector<cd> Hh((size_t)ldH * nk, 0.0), Ar, th, Z;
    int kk = 0;
    for (cycles = 1; cycles <= maxit; ++cycles) {
        // ---- extend the basis from kk to nk vectors
        if (cudaMemsetAsync(w.ks, 0, sizeof(KState), st) != cudaSuccess)
            return done(fail(c, OVL_ECUDA, "overlap eigensolver state"));
        for (int j = kk; j < nk; ++j) {
            const double2* vj = w.V + (size_t)j * n;
            double2* x = w.V + (size_t)(j + 1) * n;
            const int r = apply(vj, x);
            if (r) return done(r);
            ovl::launch_multidot(w.V, n, j + 1, x, w.h1, 0, w.part, n, st, w.ks);
            ovl::launch_multiaxpy(w.V, n, j + 1, w.h1, x, w.part, w.counter, w.ks, 0, n, st);
            ovl::launch_multidot(w.V, n, j + 1, x, w.h2, 0, w.part, n, st, w.ks);
            ovl::launch_arnoldi_orth2(w.V, n, j + 1, w.h2, x, w.Hd, ldH, w.h1, j, INT_MAX, w.part, w.counter, w.ks,
                                      n, st);
            ovl::launch_arnoldi_normalize(x, w.ks, n, st);
        }
        KState ks;
        if (cudaMemcpyAsync(&ks, w.ks, sizeof(KState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess || ks.status)
            return done(fail(c, OVL_ECUDA, "overlap eigensolver Arnoldi step"));
        const int ne = ks.done ? ks.kused : nk;  // a lucky breakdown leaves an invariant subspace
        if (ne > kk &&
            cudaMemcpyAsync(&Hh[(size_t)kk * ldH], w.Hd + (size_t)kk * ldH, sizeof(double2) * ldH * (ne - kk),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return done(fail(c, OVL_ECUDA, "overlap eigensolver H"));
        if (cudaStreamSynchronize(st) != cudaSuccess) return done(fail(c, OVL_ECUDA, "overlap eigensolver H"));
        for (int j = kk; j < ne; ++j)  // the Arnoldi step writes rows 0 .. j + 1 of column j only
            for (int r2 = j + 2; r2 < ldH; ++r2) Hh[r2 + (size_t)j * ldH] = 0.0;
        if (ne < nev) return done(fail(c, OVL_ENOCONV, "Krylov space smaller than the wanted eigenspace"));
        // ---- Ritz pairs, smallest |theta| first
        Ar.assign((size_t)ne * ne, 0.0);
        for (int i = 0; i < ne; ++i)
            for (int jj = 0; jj < ne; ++jj) Ar[(size_t)i * ne + jj] = Hh[i + (size_t)jj * ldH];
        const std::vector<cd> Hsq = Ar;
        if (ovl::host_eig(ne, Ar, th, Z) != 0) return done(fail(c, OVL_ENOCONV, "Ritz eigensolver failed"));
        std::vector<int> ord(ne);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return std::abs(th[a]) < std::abs(th[b]); });
        const cd hlast = ks.done ? cd(0.0) : Hh[ne + (size_t)(ne - 1) * ldH];
        auto resid = [&](int i) { return std::abs(hlast) * std::abs(Z[(size_t)(ne - 1) * ne + ord[i]]); };
        double worst = 0.0;
        for (int i = 0; i < nev; ++i) worst = std::max(worst, resid(i));
        if (worst <= tol || ks.done) {
            for (int i = 0; i < nev; ++i) {
                lambda[2 * i] = th[ord[i]].real();
                lambda[2 * i + 1] = th[ord[i]].imag();
            }
            // eigenvectors V z (unit norm) and their residuals with one more D_ov application each
            std::vector<cd> Zw((size_t)ne * nev);
            for (int i = 0; i < nev; ++i)
                for (int r = 0; r < ne; ++r) Zw[(size_t)i * ne + r] = Z[(size_t)r * ne + ord[i]];
            int r = rotate(c, w, w.V, ne, Zw, ne, nev, w.W);
            if (r) return done(r);
            double wr = 0.0;
            for (int i = 0; i < nev; ++i) {
                double2* xi = w.W + (size_t)i * n;
                ovl::launch_multidot(xi, n, 1, xi, w.h1, 0, w.part, n, st);
                k_ov_normalize<<<grid_of(n), 256, 0, st>>>(xi, w.h1, n);
                if ((r = apply(xi, w.t0))) return done(r);
                k_ov_resid<<<grid_of(n), 256, 0, st>>>(w.t0, xi, make_double2(lambda[2 * i], lambda[2 * i + 1]),
                                                       w.t0, n);
                ovl::launch_multidot(w.t0, n, 1, w.t0, w.h1, 0, w.part, n, st);
                double2 rr;
                if (cudaMemcpyAsync(&rr, w.h1, sizeof(double2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return done(fail(c, OVL_ECUDA, "overlap eigensolver residual"));
                wr = std::max(wr, std::sqrt(rr.x));
            }
            if (vecs &&
                cudaMemcpyAsync(vecs, w.W, sizeof(double2) * n * nev, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return done(fail(c, OVL_ECUDA, "overlap eigenvectors"));
            if (cudaStreamSynchronize(st) != cudaSuccess) return done(fail(c, OVL_ECUDA, "overlap eigenvectors"));
            if (info) {
                info->nconv = nev;
                info->max_residual = wr;
                info->ritz_residual = worst;
            }
            return done(OVL_OK);
        }
        // ---- thick restart: the nev + keep Ritz vectors nearest 0 and the last basis vector
        const int kk2 = std::min(nev + keep, ne - 1);
        std::vector<cd> Q((size_t)ne * kk2);
        for (int i = 0; i < kk2; ++i)
            for (int r = 0; r < ne; ++r) Q[(size_t)i * ne + r] = Z[(size_t)r * ne + ord[i]];
        if (!orthonormalise(Q, ne, kk2)) return done(fail(c, OVL_ENOCONV, "Ritz vectors are dependent"));
        int r = rotate(c, w, w.V, ne, Q, ne, kk2, w.W);
        if (r) return done(r);
        if (cudaMemcpyAsync(w.V, w.W, sizeof(double2) * n * kk2, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(w.V + (size_t)kk2 * n, w.V + (size_t)ne * n, sizeof(double2) * n,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return done(fail(c, OVL_ECUDA, "overlap eigensolver restart"));
        // H <- [Q^dag H Q ; h e_ne^T Q]
        std::vector<cd> HQ((size_t)ne * kk2, 0.0);
        for (int i = 0; i < kk2; ++i)
            for (int l = 0; l < ne; ++l) {
                const cd q = Q[(size_t)i * ne + l];
                for (int rr = 0; rr < ne; ++rr) HQ[(size_t)i * ne + rr] += Hsq[(size_t)rr * ne + l] * q;
            }
        std::fill(Hh.begin(), Hh.end(), cd(0.0));
        for (int i = 0; i < kk2; ++i) {
            for (int l = 0; l < kk2; ++l) {
                cd s = 0.0;
                for (int rr = 0; rr < ne; ++rr) s += std::conj(Q[(size_t)l * ne + rr]) * HQ[(size_t)i * ne + rr];
                Hh[l + (size_t)i * ldH] = s;
            }
            Hh[kk2 + (size_t)i * ldH] = hlast * Q[(size_t)i * ne + (ne - 1)];
        }
        // the kept block lives in the host copy; the next cycle's Gram-Schmidt fills columns kk2.. on the device
        kk = kk2;
    }
    cycles = maxit;
    return done(fail(c, OVL_ENOCONV, "overlap eigensolver did not converge"));
}
