// Dense eigen-decomposition of small complex matrices on the host, used by
// the deflation set-up (Rayleigh-Ritz step of the eigensolver of the
// critical eigenpairs, Sec. 3 and Sec. 5).  Plain C++, FP64:
//   1. Householder reduction to upper Hessenberg form, H = Q^dag A Q;
//   2. shifted QR iteration with Givens rotations (Wilkinson shift, exceptional
//      shifts on stagnation) to the complex Schur form T = Z^dag A Z;
//   3. eigenvectors of T by back substitution, mapped back by Z, unit norm.
// The matrices are tens to a few hundred rows; nothing here is on the timed path.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace ovl {

using cd = std::complex<double>;

static inline double cabs1(cd z) { return std::fabs(z.real()) + std::fabs(z.imag()); }
// products without the IEEE special-value handling of std::complex's operator* (the inputs are finite)
static inline cd cm(cd a, cd b) {
    return cd(a.real() * b.real() - a.imag() * b.imag(), a.real() * b.imag() + a.imag() * b.real());
}
static inline cd cmc(cd a, cd b) {  // conj(a) b
    return cd(a.real() * b.real() + a.imag() * b.imag(), a.real() * b.imag() - a.imag() * b.real());
}

// A: n x n row-major, overwritten.  w: eigenvalues.  X: right eigenvectors as
// columns, row-major n x n.  Returns 0, or -1 if the QR iteration did not converge.
// The accumulated unitary Z is kept column-major so that its column rotations are contiguous.
int host_eig(int n, std::vector<cd>& A, std::vector<cd>& w, std::vector<cd>& X) {
    auto a = [&](int i, int j) -> cd& { return A[(size_t)i * n + j]; };
    std::vector<cd> Z((size_t)n * n, 0.0);
    auto z = [&](int i, int j) -> cd& { return Z[(size_t)j * n + i]; };
    for (int i = 0; i < n; ++i) z(i, i) = 1.0;
    w.assign(n, 0.0);
    X.assign((size_t)n * n, 0.0);
    if (n == 0) return 0;
    // 1. Hessenberg reduction
    std::vector<cd> v(n), sv(n);
    for (int k = 0; k < n - 2; ++k) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += std::norm(a(i, k));
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        const cd x0 = a(k + 1, k);
        const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        v[k + 1] = x0 + ph * alpha;
        for (int i = k + 2; i < n; ++i) v[i] = a(i, k);
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        const double f = 2.0 / vn;
        // A <- (I - f v v^dag) A: s_j = sum_i conj(v_i) a(i, j), accumulated row by row
        for (int j = 0; j < n; ++j) sv[j] = 0.0;
        for (int i = k + 1; i < n; ++i) {
            const cd vi = v[i];
            const cd* ai = &A[(size_t)i * n];
            for (int j = 0; j < n; ++j) sv[j] += cmc(vi, ai[j]);
        }
        for (int i = k + 1; i < n; ++i) {
            const cd vi = f * v[i];
            cd* ai = &A[(size_t)i * n];
            for (int j = 0; j < n; ++j) ai[j] -= cm(vi, sv[j]);
        }
        // A <- A (I - f v v^dag)
        for (int i = 0; i < n; ++i) {
            cd* ai = &A[(size_t)i * n];
            cd t = 0.0;
            for (int j = k + 1; j < n; ++j) t += cm(ai[j], v[j]);
            t *= f;
            for (int j = k + 1; j < n; ++j) ai[j] -= cm(t, std::conj(v[j]));
        }
        // Z <- Z (I - f v v^dag), column by column
        for (int i = 0; i < n; ++i) sv[i] = 0.0;
        for (int j = k + 1; j < n; ++j) {
            const cd vj = v[j];
            const cd* zj = &Z[(size_t)j * n];
            for (int i = 0; i < n; ++i) sv[i] += cm(zj[i], vj);
        }
        for (int j = k + 1; j < n; ++j) {
            const cd cj = f * std::conj(v[j]);
            cd* zj = &Z[(size_t)j * n];
            for (int i = 0; i < n; ++i) zj[i] -= cm(sv[i], cj);
        }
        for (int i = k + 2; i < n; ++i) a(i, k) = 0.0;
    }
    // 2. shifted QR on the active block [lo, hi]
    const double eps = 2.220446049250313e-16;
    double anorm = 0.0;
    for (size_t e = 0; e < A.size(); ++e) anorm = std::max(anorm, cabs1(A[e]));
    int hi = n - 1, iter = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            --hi;
            continue;
        }
        // find lo: the smallest l with negligible subdiagonal a(l, l-1)
        int lo = hi;
        while (lo > 0) {
            const double s = cabs1(a(lo - 1, lo - 1)) + cabs1(a(lo, lo));
            if (cabs1(a(lo, lo - 1)) <= eps * (s > 0 ? s : anorm)) {
                a(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 100 * n) return -1;
        ++iter;
        // Wilkinson shift from the trailing 2x2 block
        cd mu;
        if (iter % 11 == 10) {
            mu = a(hi, hi) + cd(0.75 * std::abs(a(hi, hi - 1)), 0.0);  // exceptional shift
        } else {
            const cd p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), s = a(hi, hi);
            const cd tr = p + s, det = p * s - q * r;
            const cd disc = std::sqrt(tr * tr - 4.0 * det);
            const cd l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
            mu = std::abs(l1 - s) < std::abs(l2 - s) ? l1 : l2;
        }
        // QR step on H[lo..hi] - mu I via Givens rotations, applied to the full matrix
        std::vector<cd> gc(hi - lo), gs(hi - lo);
        std::vector<double> gcr(hi - lo);
        for (int k = lo; k <= hi; ++k) a(k, k) -= mu;
        for (int k = lo; k < hi; ++k) {
            const cd x = a(k, k), y = a(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            double c;
            cd sn;
            if (r == 0.0) {
                c = 1.0;
                sn = 0.0;
            } else {
                c = std::abs(x) / r;
                const cd ph = std::abs(x) > 0 ? x / std::abs(x) : cd(1.0);
                sn = ph * std::conj(y) / r;
            }
            gcr[k - lo] = c;
            gs[k - lo] = sn;
            // rows k, k+1: [c, s; -conj(s), c]
            cd* ak = &A[(size_t)k * n];
            cd* ak1 = &A[(size_t)(k + 1) * n];
            const cd snc = std::conj(sn);
            for (int j = k; j < n; ++j) {
                const cd t1 = ak[j], t2 = ak1[j];
                ak[j] = c * t1 + cm(sn, t2);
                ak1[j] = c * t2 - cm(snc, t1);
            }
        }
        for (int k = lo; k < hi; ++k) {
            const double c = gcr[k - lo];
            const cd sn = gs[k - lo];
            // columns k, k+1 from the right with the conjugate transpose
            const int rmax = std::min(hi, k + 2);
            const cd snc = std::conj(sn);
            for (int i = 0; i <= rmax; ++i) {
                const cd t1 = a(i, k), t2 = a(i, k + 1);
                a(i, k) = c * t1 + cm(snc, t2);
                a(i, k + 1) = c * t2 - cm(sn, t1);
            }
            cd* zk = &Z[(size_t)k * n];
            cd* zk1 = &Z[(size_t)(k + 1) * n];
            for (int i = 0; i < n; ++i) {
                const cd t1 = zk[i], t2 = zk1[i];
                zk[i] = c * t1 + cm(snc, t2);
                zk1[i] = c * t2 - cm(sn, t1);
            }
        }
        for (int k = lo; k <= hi; ++k) a(k, k) += mu;
    }
    for (int i = 0; i < n; ++i) w[i] = a(i, i);
    // 3. eigenvectors of the upper triangular T, then X = Z Y
    std::vector<cd> y(n);
    const double small = std::max(anorm, 1e-300) * eps;
    for (int k = 0; k < n; ++k) {
        for (int i = 0; i < n; ++i) y[i] = 0.0;
        y[k] = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            cd s = 0.0;
            const cd* ai = &A[(size_t)i * n];
            for (int j = i + 1; j <= k; ++j) s += cm(ai[j], y[j]);
            cd d = a(i, i) - w[k];
            if (std::abs(d) < small) d = small;
            y[i] = -s / d;
        }
        std::vector<cd> col(n, 0.0);
        for (int j = 0; j <= k; ++j) {
            const cd yj = y[j];
            const cd* zj = &Z[(size_t)j * n];
            for (int i = 0; i < n; ++i) col[i] += cm(zj[i], yj);
        }
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm += std::norm(col[i]);
        nrm = std::sqrt(nrm);
        for (int i = 0; i < n; ++i) X[(size_t)i * n + k] = col[i] / nrm;
    }
    return 0;
}

}  // namespace ovl
