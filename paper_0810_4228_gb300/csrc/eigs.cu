// Deflation phase on the GPU: the critical left and right eigenpairs of
// A = gamma5 D_w(mu) needed by LR deflation (Sec. 3, Eq. 3.1), computed once
// per gauge field and mu for all sources (Sec. 3, last paragraph; Sec. 5 uses
// ARPACK on the CPU for this step).
//
// Method: thick-restart Arnoldi (Krylov-Schur form) on a Chebyshev polynomial
// of T = A^2.  The eigenvalues of A nearest 0 are those of T of smallest
// modulus.  For gamma5 D_w(mu) at moderate mu the spectrum of A lies close to
// the real axis, so T's lies in a thin region along the positive real axis,
// and the wanted ones crowd at its bottom end: on 16^3 x 8 the 40 smallest
// eigenvalues of T lie within 15 % of each other against a spread of 5, which
// makes Arnoldi on T itself converge slowly.  One Arnoldi cycle on T locates
// (from above) the end acut of the wanted cluster; then P = T_d((c - T) / e),
// the Chebyshev polynomial of degree d on [acut, |A|^2], maps the eigenvalues
// below acut to the largest of P in modulus and spreads them out, and those
// above acut into [-1, 1].  Each cycle extends an orthonormal basis V to
// nkrylov vectors (classical Gram-Schmidt twice, the library's Arnoldi
// kernels), computes the Ritz pairs of the projected matrix H on the host
// (host_eig.cpp) and restarts from the orthonormalised Ritz vectors of the
// want + keep largest |theta(P)| and the last basis vector: with Q those Ritz
// vectors' coordinates, P (V Q) = (V Q)(Q^dag H Q) + h v_next e^T Q keeps the
// Arnoldi relation with a full last row.  Once the wanted pairs have
// converged, a Rayleigh-Ritz step with A itself on their span gives the
// eigenpairs of A (right vectors from A, left ones from A^dag = gamma5
// D_w(-mu)).  Pairs are matched by lambda_left = conj(lambda_right), the m of
// smallest |Re lambda| kept and bi-orthonormalised (L <- L (L^dag R)^-H) when
// installed.  All vector work runs in the library's kernels; only nkrylov x
// nkrylov matrices visit the host.  Not on the timed path (the paper excludes
// the deflation phase from its timings, Sec. 5).
#include <algorithm>
#include <climits>
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

// y <- y / sqrt(h.x)   (h = y^dag y from a preceding dot product)
__global__ void k_normalize(double2* y, const double2* h, size_t n) {
    const double inv = 1.0 / sqrt(fmax(h->x, 1e-300));
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 v = y[e];
        y[e] = make_double2(v.x * inv, v.y * inv);
    }
}

// Chebyshev step of the filter: yn = s1 (c y - u) - s0 yp, with u = T y already in yn
__global__ void k_cheb_step(const double2* __restrict__ y, const double2* __restrict__ yp, double2* yn, double c,
                            double s1, double s0, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 yy = y[e], u = yn[e];
        double2 r = make_double2(s1 * (c * yy.x - u.x), s1 * (c * yy.y - u.y));
        if (s0 != 0.0) {
            const double2 pp = yp[e];
            r.x -= s0 * pp.x;
            r.y -= s0 * pp.y;
        }
        yn[e] = r;
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

using cd = std::complex<double>;

struct EigRun {
    std::vector<cd> theta;      // eigenvalues of A (want)
    std::vector<double> resid;  // |A x - theta x| of the unit vectors
    int cycles = 0;
    long long matvecs = 0;
    double anorm = 0;           // estimate of |A| (power iteration on A^dag A)
    double tcut = 0;            // |lambda|^2 of the want-th pair
};

// Columns of Q (ne x kk, column-major) made orthonormal: modified Gram-Schmidt, twice.
bool host_orthonormalise(std::vector<cd>& Q, int ne, int kk) {
    for (int i = 0; i < kk; ++i) {
        cd* qi = &Q[(size_t)i * ne];
        for (int pass = 0; pass < 2; ++pass)
            for (int l = 0; l < i; ++l) {
                const cd* ql = &Q[(size_t)l * ne];
                cd sdot = 0.0;
                for (int r = 0; r < ne; ++r) sdot += std::conj(ql[r]) * qi[r];
                for (int r = 0; r < ne; ++r) qi[r] -= sdot * ql[r];
            }
        double nn = 0.0;
        for (int r = 0; r < ne; ++r) nn += std::norm(qi[r]);
        nn = std::sqrt(nn);
        if (!(nn > 1e-300)) return false;
        for (int r = 0; r < ne; ++r) qi[r] /= nn;
    }
    return true;
}

// Device scratch of one run.
struct ArnWork {
    double2* V;      // (nk + 1) basis vectors
    double2* W;      // nk vectors: rotated basis, then the output eigenvectors
    double2* t0;     // one vector
    double2* cb[3];  // Chebyshev recurrence
    double2* Hd;     // (nk + 1) x nk, column-major
    double2* h1;     // nk + 2
    double2* h2;     // nk + 2
    double2* Qd;     // nk x nk
    double* part;    // multidot partials for nk + 2 vectors
    KState* ks;
};

// out_j = sum_l coef[l + j ld] V_l for j < nout (coef on the host, column-major with leading dimension ld).
int rotate(ovl_ctx* c, const ArnWork& w, const double2* V, int nv, const std::vector<cd>& coef, int ld, int nout,
           double2* out) {
    const size_t n = c->n;
    cudaStream_t st = c->st;
    std::vector<cd> neg((size_t)nv * nout);
    for (int j = 0; j < nout; ++j)
        for (int l = 0; l < nv; ++l) neg[(size_t)j * nv + l] = -coef[(size_t)j * ld + l];
    OVL_CUDA_TRY(c, cudaMemcpyAsync(w.Qd, neg.data(), sizeof(double2) * nv * nout, cudaMemcpyHostToDevice, st));
    OVL_CUDA_TRY(c, cudaMemsetAsync(out, 0, sizeof(double2) * n * nout, st));
    for (int j = 0; j < nout; ++j)
        ovl::launch_multiaxpy(V, n, nv, w.Qd + (size_t)j * nv, out + (size_t)j * n, w.part, c->counter, w.ks, 0, n,
                              st);
    // the coefficients are read by the kernels above before the next upload
    OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
    return OVL_OK;
}

// One side (dagger = 0: A, 1: A^dag): the want eigenpairs of A of smallest |lambda| with
// |A x - lambda x| <= tol |A|; unit eigenvectors in out (want x n), eigenvalues in run.theta.
//
// 1. |A|^2 from a power iteration on A^dag A (upper end of the spectrum of T = A^2).
// 2. One Arnoldi cycle on T: its smallest Ritz values locate (from above) the end of the wanted
//    cluster, acut = |theta| of the (want + keep)-th.
// 3. Thick-restart Arnoldi on P = T_d((c - T) / e), the Chebyshev polynomial of degree d on
//    [acut, |A|^2]: the eigenvalues of T below acut become the largest of P in modulus, spread
//    out (the crowded bottom of T's spectrum is what slows Arnoldi on T itself); those above
//    acut map into [-1, 1].  The want + keep Ritz vectors of largest |theta(P)| are kept.
// 4. Rayleigh-Ritz with A on the converged ones; if a wanted |lambda|^2 lies above acut the
//    filter interval is widened and step 3 continues.
int krylov_schur(ovl_ctx* c, double mu, double kappa, int dagger, int want, int nk, int keep, double tol,
                 int maxcycles, const ArnWork& w, double2* out, EigRun& run) {
    const size_t n = c->n;
    cudaStream_t st = c->st;
    const double m_eff = dagger ? -mu : mu;
    const int ldH = nk + 1;
    auto applyA = [&](const double2* x, double2* y) {
        ovl::launch_dslash(c->U64, 0, x, y, m_eff, kappa, 1, c->g, st, w.ks);
        ++run.matvecs;
    };
    auto applyAdag = [&](const double2* x, double2* y) {
        ovl::launch_dslash(c->U64, 0, x, y, -m_eff, kappa, 1, c->g, st, w.ks);
        ++run.matvecs;
    };
    auto reset_state = [&]() { return cudaMemsetAsync(w.ks, 0, sizeof(KState), st); };
    // filter state: mode 0 = T, 1 = P
    int mode = 0, deg = 1;
    double cc = 0.0, ee = 1.0, acut = 0.0;
    auto applyT = [&](const double2* x, double2* y) {
        applyA(x, w.t0);
        applyA(w.t0, y);
    };
    auto applyOp = [&](const double2* x, double2* y) -> int {
        if (mode == 0) {
            applyT(x, y);
            return OVL_OK;
        }
        // y = T_deg((cc - T)/ee) x by the three-term recurrence in the scratch vectors cb[]
        const double2* yp = x;
        double2* yc = w.cb[0];
        applyT(x, yc);
        k_cheb_step<<<grid_n(n), 256, 0, st>>>(x, nullptr, yc, cc, 1.0 / ee, 0.0, n);
        int free_i = 1;
        for (int k = 2; k <= deg; ++k) {
            double2* yn = w.cb[free_i];
            applyT(yc, yn);
            k_cheb_step<<<grid_n(n), 256, 0, st>>>(yc, yp, yn, cc, 2.0 / ee, 1.0, n);
            // rotate: the buffer that held yp (if a scratch one) becomes free
            int next_free = 0;
            for (int q = 0; q < 3; ++q)
                if (w.cb[q] != yc && w.cb[q] != yn) next_free = q;
            yp = yc;
            yc = yn;
            free_i = next_free;
        }
        OVL_CUDA_TRY(c, cudaMemcpyAsync(y, yc, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
        return OVL_OK;
    };
    // ---- 1. |A|^2 by power iteration on A^dag A
    OVL_CUDA_TRY(c, reset_state());
    k_rand_fill<<<grid_n(n), 256, 0, st>>>(w.t0, n, 0x5eedull + dagger);
    double sig2 = 0.0;
    {
        double2* x = w.cb[0];
        double2* ax = w.cb[1];
        double2* aax = w.cb[2];
        OVL_CUDA_TRY(c, cudaMemcpyAsync(x, w.t0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
        for (int it = 0; it < 30; ++it) {
            ovl::launch_multidot(x, n, 1, x, w.h1, 0, w.part, n, st);
            k_normalize<<<grid_n(n), 256, 0, st>>>(x, w.h1, n);
            applyA(x, ax);
            applyAdag(ax, aax);
            ovl::launch_multidot(x, n, 1, aax, w.h1, 0, w.part, n, st);
            double2 hv;
            OVL_CUDA_TRY(c, cudaMemcpyAsync(&hv, w.h1, sizeof(double2), cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
            sig2 = std::max(sig2, hv.x);
            std::swap(x, aax);
        }
    }
    const double bup = 1.15 * sig2;
    run.anorm = std::sqrt(bup);
    // random unit start vector
    k_rand_fill<<<grid_n(n), 256, 0, st>>>(w.V, n, 0x1234ull + 77 * dagger);
    ovl::launch_multidot(w.V, n, 1, w.V, w.h1, 0, w.part, n, st);
    k_normalize<<<grid_n(n), 256, 0, st>>>(w.V, w.h1, n);
    std::vector<cd> Hh((size_t)ldH * nk, 0.0);
    std::vector<cd> Ar, th, Z;
    int kk = 0;
    double ttol = tol;
    auto set_filter = [&](double a) {
        acut = std::min(a, 0.5 * bup);
        cc = 0.5 * (bup + acut);
        ee = 0.5 * (bup - acut);
        // about 8 e-folds of amplification across [0, acut]
        const double rate = std::sqrt(2.0 * 2.0 * acut / (bup - acut));
        deg = (int)std::min(400.0, std::max(16.0, std::ceil(8.0 / std::max(rate, 1e-12))));
        mode = 1;
    };
    for (int cyc = 0; cyc < maxcycles; ++cyc) {
        run.cycles = cyc + 1;
        // ---- extend the basis from kk to nk vectors (CGS2 against V_0..V_j)
        OVL_CUDA_TRY(c, reset_state());
        for (int j = kk; j < nk; ++j) {
            const double2* vj = w.V + (size_t)j * n;
            double2* x = w.V + (size_t)(j + 1) * n;
            int r0 = 0;
            if (mode == 0) applyT(vj, x);
            else if ((r0 = applyOp(vj, x))) return r0;
            ovl::launch_multidot(w.V, n, j + 1, x, w.h1, 0, w.part, n, st, w.ks);
            ovl::launch_multiaxpy(w.V, n, j + 1, w.h1, x, w.part, c->counter, w.ks, 0, n, st);
            ovl::launch_multidot(w.V, n, j + 1, x, w.h2, 0, w.part, n, st, w.ks);
            ovl::launch_arnoldi_orth2(w.V, n, j + 1, w.h2, x, w.Hd, ldH, w.h1, j, INT_MAX, w.part, c->counter, w.ks,
                                      n, st);
            ovl::launch_arnoldi_normalize(x, w.ks, n, st);
        }
        KState ks;
        OVL_CUDA_TRY(c, cudaMemcpyAsync(&ks, w.ks, sizeof(KState), cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
        if (ks.status) return fail(c, OVL_ECUDA, "eigensolver Arnoldi step");
        const int ne = ks.done ? ks.kused : nk;  // a lucky breakdown leaves an invariant subspace
        if (ne > kk)
            OVL_CUDA_TRY(c, cudaMemcpyAsync(&Hh[(size_t)kk * ldH], w.Hd + (size_t)kk * ldH,
                                            sizeof(double2) * ldH * (ne - kk), cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
        // the Arnoldi step writes rows 0 .. j + 1 of column j only: below that H is zero (the device
        // buffer holds older contents there)
        for (int j = kk; j < ne; ++j)
            for (int r2 = j + 2; r2 < ldH; ++r2) Hh[r2 + (size_t)j * ldH] = 0.0;
        OVL_CUDA_TRY(c, reset_state());
        // ---- Ritz pairs of H (ne x ne), wanted first: smallest |theta| of T, largest of P
        Ar.assign((size_t)ne * ne, 0.0);
        for (int i = 0; i < ne; ++i)
            for (int jj = 0; jj < ne; ++jj) Ar[(size_t)i * ne + jj] = Hh[i + (size_t)jj * ldH];
        std::vector<cd> Hsq = Ar;
        if (ovl::host_eig(ne, Ar, th, Z) != 0) return fail(c, OVL_ENOCONV, "Ritz eigensolver failed");
        std::vector<int> ord(ne);
        std::iota(ord.begin(), ord.end(), 0);
        if (mode == 0)
            std::sort(ord.begin(), ord.end(), [&](int a, int b) { return std::abs(th[a]) < std::abs(th[b]); });
        else
            std::sort(ord.begin(), ord.end(), [&](int a, int b) { return std::abs(th[a]) > std::abs(th[b]); });
        const cd hlast = ks.done ? cd(0.0) : Hh[ne + (size_t)(ne - 1) * ldH];
        if (ne < want) return fail(c, OVL_ENOCONV, "Krylov space smaller than the wanted eigenspace");
        const int kk2 = std::min(want + keep, ne - 1);
        if (mode == 0 && !ks.done) {
            // ---- 2. the filter from the first cycle's smallest Ritz values, then restart from the
            // sum of the kept Ritz vectors
            set_filter(std::abs(th[ord[kk2]]));
            std::vector<cd> sumv((size_t)ne, 0.0);
            for (int i = 0; i < kk2; ++i)
                for (int r = 0; r < ne; ++r) sumv[r] += Z[(size_t)r * ne + ord[i]];
            if (!host_orthonormalise(sumv, ne, 1)) return fail(c, OVL_ENOCONV, "start vector");
            int r = rotate(c, w, w.V, ne, sumv, ne, 1, w.W);
            if (r) return r;
            OVL_CUDA_TRY(c, cudaMemcpyAsync(w.V, w.W, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
            std::fill(Hh.begin(), Hh.end(), cd(0.0));
            kk = 0;
            continue;
        }
        // relative residual of each Ritz pair (P spans many orders of magnitude)
        auto rres = [&](int i) {
            const double sc = mode == 0 ? bup : std::max(std::abs(th[ord[i]]), 1e-300);
            return std::abs(hlast) * std::abs(Z[(size_t)(ne - 1) * ne + ord[i]]) / sc;
        };
        double worst = 0.0;
        for (int i = 0; i < want; ++i) worst = std::max(worst, rres(i));
        if (worst <= ttol || ks.done) {
            // ---- 4. Rayleigh-Ritz with A on the span of the converged Ritz vectors: the want first
            // and those of the next keep that have converged too.  An eigenvalue of T is shared by
            // A's lambda and -lambda (and nearly so by close pairs); a span that holds one of them
            // without the other is not A-invariant, so partners beyond the want-th are taken
            // along once they converge.
            std::vector<int> sel;
            for (int i = 0; i < std::min(want + keep, ne); ++i)
                if (i < want || ks.done || rres(i) <= ttol) sel.push_back(ord[i]);
            const int wx = (int)sel.size();
            std::vector<cd> Qw((size_t)ne * wx);
            for (int i = 0; i < wx; ++i)
                for (int r = 0; r < ne; ++r) Qw[(size_t)i * ne + r] = Z[(size_t)r * ne + sel[i]];
            if (!host_orthonormalise(Qw, ne, wx)) return fail(c, OVL_ENOCONV, "Ritz vectors are dependent");
            double2* X = w.W;  // wx orthonormal vectors spanning the converged invariant subspace
            int r = rotate(c, w, w.V, ne, Qw, ne, wx, X);
            if (r) return r;
            double2* HAd = w.Hd;  // wx x wx, column-major
            for (int i = 0; i < wx; ++i) {
                applyA(X + (size_t)i * n, w.t0);
                ovl::launch_multidot(X, n, wx, w.t0, HAd + (size_t)i * wx, 0, w.part, n, st);
            }
            std::vector<cd> HA((size_t)wx * wx);
            OVL_CUDA_TRY(c, cudaMemcpyAsync(HA.data(), HAd, sizeof(double2) * wx * wx, cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
            std::vector<cd> Br((size_t)wx * wx), lam, Zs;
            for (int i = 0; i < wx; ++i)
                for (int jj = 0; jj < wx; ++jj) Br[(size_t)i * wx + jj] = HA[i + (size_t)jj * wx];
            if (ovl::host_eig(wx, Br, lam, Zs) != 0) return fail(c, OVL_ENOCONV, "Rayleigh-Ritz eigensolver failed");
            // the want A pairs of smallest |lambda|
            std::vector<int> oa(wx);
            std::iota(oa.begin(), oa.end(), 0);
            std::sort(oa.begin(), oa.end(), [&](int a, int b) { return std::abs(lam[a]) < std::abs(lam[b]); });
            std::vector<cd> Zc((size_t)want * wx);
            for (int i = 0; i < want; ++i)
                for (int l = 0; l < wx; ++l) Zc[(size_t)i * wx + l] = Zs[(size_t)l * wx + oa[i]];
            r = rotate(c, w, X, wx, Zc, wx, want, out);
            if (r) return r;
            run.theta.assign(want, 0.0);
            run.resid.assign(want, 0.0);
            double wr = 0.0;
            for (int i = 0; i < want; ++i) {
                run.theta[i] = lam[oa[i]];
                applyA(out + (size_t)i * n, w.t0);
                const double2 thd = make_double2(lam[oa[i]].real(), lam[oa[i]].imag());
                k_resid<<<grid_n(n), 256, 0, st>>>(w.t0, out + (size_t)i * n, thd, w.ks, w.part, c->counter, n);
                double2 rv;
                OVL_CUDA_TRY(c, cudaMemcpyAsync(&rv, &w.ks->red[0], sizeof(double2), cudaMemcpyDeviceToHost, st));
                OVL_CUDA_TRY(c, cudaStreamSynchronize(st));
                run.resid[i] = std::sqrt(rv.x);
                wr = std::max(wr, run.resid[i]);
            }
            run.tcut = std::norm(lam[oa[want - 1]]);
            if (mode == 1 && !ks.done && run.tcut > acut) {
                // a wanted eigenvalue lies outside the amplified region: widen the filter and
                // start over from the current eigenvectors' sum
                set_filter(2.0 * run.tcut);
                std::vector<cd> ones((size_t)want, 1.0);
                r = rotate(c, w, out, want, ones, want, 1, w.V);
                if (r) return r;
                ovl::launch_multidot(w.V, n, 1, w.V, w.h1, 0, w.part, n, st);
                k_normalize<<<grid_n(n), 256, 0, st>>>(w.V, w.h1, n);
                std::fill(Hh.begin(), Hh.end(), cd(0.0));
                kk = 0;
                ttol = tol;
                continue;
            }
            if (wr <= tol * run.anorm) return OVL_OK;
            if (ks.done) return fail(c, OVL_ENOCONV, "invariant Krylov space without accurate eigenpairs");
            // not yet accurate for A: tighten the criterion and go on from the same basis
            ttol = std::max(ttol * 0.1, 1e-14);
        }
        // ---- thick restart: the want + keep wanted-end Ritz vectors and the last basis vector
        std::vector<cd> Q((size_t)ne * kk2);
        for (int i = 0; i < kk2; ++i)
            for (int r = 0; r < ne; ++r) Q[(size_t)i * ne + r] = Z[(size_t)r * ne + ord[i]];
        if (!host_orthonormalise(Q, ne, kk2)) return fail(c, OVL_ENOCONV, "Ritz vectors are dependent");
        int r = rotate(c, w, w.V, ne, Q, ne, kk2, w.W);
        if (r) return r;
        OVL_CUDA_TRY(c, cudaMemcpyAsync(w.V, w.W, sizeof(double2) * n * kk2, cudaMemcpyDeviceToDevice, st));
        OVL_CUDA_TRY(c, cudaMemcpyAsync(w.V + (size_t)kk2 * n, w.V + (size_t)ne * n, sizeof(double2) * n,
                                        cudaMemcpyDeviceToDevice, st));
        // H <- [Q^dag H Q ; h e_ne^T Q]
        std::vector<cd> HQ((size_t)ne * kk2, 0.0);
        for (int i = 0; i < kk2; ++i)
            for (int l = 0; l < ne; ++l) {
                const cd q = Q[(size_t)i * ne + l];
                if (q == cd(0.0)) continue;
                for (int rr = 0; rr < ne; ++rr) HQ[(size_t)i * ne + rr] += Hsq[(size_t)rr * ne + l] * q;
            }
        std::fill(Hh.begin(), Hh.end(), cd(0.0));
        for (int i = 0; i < kk2; ++i) {
            for (int l = 0; l < kk2; ++l) {
                cd sdot = 0.0;
                for (int rr = 0; rr < ne; ++rr) sdot += std::conj(Q[(size_t)l * ne + rr]) * HQ[(size_t)i * ne + rr];
                Hh[l + (size_t)i * ldH] = sdot;
            }
            Hh[kk2 + (size_t)i * ldH] = hlast * Q[(size_t)i * ne + (ne - 1)];
        }
        kk = kk2;
    }
    return fail(c, OVL_ENOCONV, "deflation eigensolver did not converge");
}

}  // namespace

extern "C" int ovl_deflation_eigs(ovl_ctx* c, double mu, double kappa, int m, int nextra, double tol, int nkrylov,
                                  int maxit, ovl_eiginfo* info) {
    if (!c || m < 1 || nextra < 0 || m + nextra > 512 || nkrylov < 0 || maxit < 1 || !(tol > 0))
        return fail(c, OVL_EINVAL, "bad argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    const size_t n = c->n;
    const int want = m + nextra;
    if ((size_t)want > n) return fail(c, OVL_EINVAL, "more eigenpairs than the dimension");
    // default basis: wide enough that the restart buffer spans well past the wanted cluster (the
    // small eigenvalues of A^2 crowd at the bottom of its spectrum on larger lattices)
    int nk = nkrylov > 0 ? nkrylov : std::min(512, std::max(3 * want + 40, 10 * want));
    nk = (int)std::min<size_t>((size_t)std::max(nk, want + 8), n);
    // device memory: basis, rotation target, two output blocks (at most 64 GiB, else a smaller basis)
    auto bytes_for = [&](int k) { return sizeof(double2) * n * ((size_t)2 * k + 2 * want + 5); };
    while (nk > want + 8 && bytes_for(nk) > ((size_t)64 << 30)) --nk;
    const int keep = std::max(8, (nk - want) / 3);
    int r = ensure_base(c);
    if (r) return r;
    const int mdb = ovl::multidot_blocks(n);
    const size_t part_bytes = std::max<size_t>((size_t)mdb * (nk + 2) * sizeof(double2), (size_t)1 << 16);
    ArnWork w = {};
    double2 *XR = nullptr, *XL = nullptr;
    void* ptrs[14] = {};
    auto cleanup = [&]() {
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
    const size_t sizes[14] = {sizeof(double2) * n * (nk + 1), sizeof(double2) * n * nk, sizeof(double2) * n,
                              sizeof(double2) * (size_t)(nk + 1) * nk, sizeof(double2) * (nk + 2),
                              sizeof(double2) * (nk + 2), sizeof(double2) * (size_t)nk * nk, part_bytes,
                              sizeof(KState), sizeof(double2) * n * want, sizeof(double2) * n * want,
                              sizeof(double2) * n, sizeof(double2) * n, sizeof(double2) * n};
    for (int i = 0; i < 14; ++i)
        if (cudaMalloc(&ptrs[i], sizes[i]) != cudaSuccess) {
            ptrs[i] = nullptr;
            cleanup();
            return fail(c, OVL_ENOMEM, "eigensolver workspace");
        }
    w.V = (double2*)ptrs[0], w.W = (double2*)ptrs[1], w.t0 = (double2*)ptrs[2], w.Hd = (double2*)ptrs[3];
    w.h1 = (double2*)ptrs[4], w.h2 = (double2*)ptrs[5], w.Qd = (double2*)ptrs[6], w.part = (double*)ptrs[7];
    w.ks = (KState*)ptrs[8];
    XR = (double2*)ptrs[9], XL = (double2*)ptrs[10];
    for (int q = 0; q < 3; ++q) w.cb[q] = (double2*)ptrs[11 + q];
    EigRun right, left;
    r = krylov_schur(c, mu, kappa, 0, want, nk, keep, tol, maxit, w, XR, right);
    if (!r) r = krylov_schur(c, mu, kappa, 1, want, nk, keep, tol, maxit, w, XL, left);
    auto fill_info = [&](int mm, const EigRun& e, double wr) {
        if (!info) return;
        info->m = mm;
        info->iterations = right.cycles + left.cycles;
        info->matvecs = right.matvecs + left.matvecs;
        info->max_residual = wr;
        info->lambda_cut = std::sqrt(e.tcut);
    };
    if (r) {
        // progress of the side that stopped: cycles, matvecs, the last residual check
        const EigRun& e = left.cycles ? left : right;
        double wr = 0.0;
        for (double x : e.resid) wr = std::max(wr, x);
        fill_info(0, e, wr);
        cleanup();
        return r;
    }
    // select the m right pairs of smallest |Re lambda| among the computed ones, pair with left
    std::vector<int> ord(want);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(),
              [&](int a, int b) { return std::fabs(right.theta[a].real()) < std::fabs(right.theta[b].real()); });
    std::vector<double> lam(2 * m);
    double2* Rsel = w.V;  // the basis is free now: m selected right vectors, then m left ones
    double2* Lsel = w.W;
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
        cudaMemcpyAsync(Rsel + (size_t)q * n, XR + (size_t)j * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(Lsel + (size_t)q * n, XL + (size_t)best * n, sizeof(double2) * n, cudaMemcpyDeviceToDevice,
                        c->st);
    }
    if (worst_pair > 1e-6) {
        fill_info(0, right, 0.0);
        cleanup();
        return fail(c, OVL_ENOCONV, "left and right eigenvalues do not pair up");
    }
    r = install_deflation(c, mu, kappa, m, lam.data(), Rsel, Lsel);
    cudaStreamSynchronize(c->st);
    double wr = 0.0;
    for (int q = 0; q < m; ++q) wr = std::max(wr, right.resid[ord[q]]);
    fill_info(r ? 0 : m, right, wr);
    cleanup();
    return r;
}
