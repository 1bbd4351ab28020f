// C ABI of the overlap library (include/ovl.h): context, gauge field, the
// Wilson operator, deflation set-up and the Krylov sign solve.  Host code only
// orders kernels; every arithmetic step of a solve runs in the device kernels
// of stencil.cu, krylov.cu and inner_sign.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "ctx.h"

using ovl::Geom;
using ovl::KState;
using namespace ovl_priv;

namespace {

const char* kclass_name[ovl_priv::KC_COUNT] = {"setup", "deflate_split", "dslash_pair", "lanczos_step", "inner_sign",
                                     "dslash_regen", "combine", "dslash", "multidot", "multiaxpy",
                                     "arnoldi_normalize", "convert", "pass1_persistent", "pass2_persistent"};
const int kclass_kernels[ovl_priv::KC_COUNT] = {1, 1, 1, 1, 0, 1, 1, 1, 2, 1, 1, 1, 1, 1};

}  // namespace

namespace ovl_priv {

int fail(ovl_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CUDA_TRY OVL_CUDA_TRY

template <class T>
int dalloc(ovl_ctx* c, T** p, size_t bytes) {
    if (*p) return OVL_OK;
    cudaError_t e = cudaMalloc((void**)p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, OVL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return OVL_OK;
}

template <class T>
void dfree(T** p) {
    if (*p) cudaFree((void*)*p);
    *p = nullptr;
}

void free_solve(ovl_ctx* c) {
    dfree(&c->V64);
    for (int i = 0; i < 3; ++i) dfree(&c->W64[i]), dfree(&c->R64[i]), dfree(&c->v32[i]), dfree(&c->w32[i]);
    dfree(&c->alpha), dfree(&c->beta), dfree(&c->gamma), dfree(&c->vscale), dfree(&c->cvec);
    dfree(&c->H), dfree(&c->h1), dfree(&c->h2);
    dfree(&c->partials);
    dfree(&c->inner);
    c->kcap = 0;
    c->inner_elems = 0;
    c->partials_bytes = 0;
}

void drop_solve_graph(ovl_ctx* c) {
    if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
    c->graph = GraphEntry();
}

void drop_graph(ovl_ctx* c) {
    drop_solve_graph(c);
    // the one-sequence batch captured the context's buffers and settings as well
    if (c->self_batch) ovl_batch_destroy(c->self_batch);
    c->self_batch = nullptr;
}

// fixed-size buffers (independent of k)
int ensure_base(ovl_ctx* c) {
    const size_t vb = c->n * sizeof(double2);
    int r;
    // the grid-reduction ticket and the barrier counter start at zero (the last block of every
    // reduction resets its ticket)
    const bool fresh = c->counter == nullptr || c->bar == nullptr;
    if (fresh && ((r = dalloc(c, &c->counter, 64)) || (r = dalloc(c, &c->bar, 64)))) return r;
    if (fresh) {
        CUDA_TRY(c, cudaMemsetAsync(c->counter, 0, 64, c->st));
        CUDA_TRY(c, cudaMemsetAsync(c->bar, 0, 64, c->st));
    }
    if ((r = dalloc(c, &c->b64, vb)) || (r = dalloc(c, &c->y64, vb)) || (r = dalloc(c, &c->bR, vb)) ||
        (r = dalloc(c, &c->bL, vb)) || (r = dalloc(c, &c->t64, vb)) || (r = dalloc(c, &c->s64, vb)) ||
        (r = dalloc(c, &c->t32, c->n * sizeof(float2))) || (r = dalloc(c, &c->s32, c->n * sizeof(float2))) ||
        (r = dalloc(c, &c->ks, sizeof(KState))) || (r = dalloc(c, &c->counter, 64)) || (r = dalloc(c, &c->bar, 64)) ||
        (r = dalloc(c, &c->stage_in, vb)) || (r = dalloc(c, &c->stage_out, vb)) ||
        (r = dalloc(c, &c->nat_a, vb)) || (r = dalloc(c, &c->nat_b, vb)) || (r = dalloc(c, &c->pq, 4096 * sizeof(double2))))
        return r;
    for (int i = 0; i < 3; ++i) {
        if ((r = dalloc(c, &c->W64[i], vb)) || (r = dalloc(c, &c->R64[i], vb)) ||
            (r = dalloc(c, &c->v32[i], c->n * sizeof(float2))) || (r = dalloc(c, &c->w32[i], c->n * sizeof(float2))))
            return r;
    }
    return OVL_OK;
}

int ensure_solve(ovl_ctx* c, int k) {
    int r = ensure_base(c);
    if (r) return r;
    const int mdb = ovl::multidot_blocks(c->n);
    const size_t need_part = std::max<size_t>((size_t)(k + 2 + 2 * std::max(c->m, 1)) * mdb * sizeof(double2),
                                              (size_t)1 << 19);
    if (k <= c->kcap && c->partials_bytes >= need_part) return OVL_OK;
    drop_graph(c);
    dfree(&c->V64);
    dfree(&c->alpha), dfree(&c->beta), dfree(&c->gamma), dfree(&c->vscale), dfree(&c->cvec);
    dfree(&c->H), dfree(&c->h1), dfree(&c->h2), dfree(&c->partials), dfree(&c->inner);
    const int kc = std::max(k, c->kcap);
    const size_t vb = c->n * sizeof(double2);
    const size_t kb = (size_t)(kc + 1) * sizeof(double2);
    const size_t ie = std::max({ovl::inner_work_elems(kc, 0), ovl::inner_work_elems(kc, 1),
                                ovl::inner_work_elems(kc, 2)});
    if ((r = dalloc(c, &c->V64, vb * (kc + 1))) || (r = dalloc(c, &c->alpha, kb)) || (r = dalloc(c, &c->beta, kb)) ||
        (r = dalloc(c, &c->gamma, kb)) || (r = dalloc(c, &c->vscale, kb)) || (r = dalloc(c, &c->cvec, kb)) ||
        (r = dalloc(c, &c->H, kb * (kc + 1))) || (r = dalloc(c, &c->h1, kb)) || (r = dalloc(c, &c->h2, kb)) ||
        (r = dalloc(c, &c->partials, need_part)) || (r = dalloc(c, &c->inner, ie * sizeof(double2)))) {
        free_solve(c);
        return r;
    }
    CUDA_TRY(c, cudaMemsetAsync(c->counter, 0, 64, c->st));
    CUDA_TRY(c, cudaMemsetAsync(c->bar, 0, 64, c->st));
    c->kcap = kc;
    c->partials_bytes = need_part;
    c->inner_elems = ie;
    return OVL_OK;
}

// restarted Arnoldi: the accumulated Hessenberg matrix of K columns and its inner-sign workspace
int ensure_restart(ovl_ctx* c, int K) {
    if (K <= c->krs_cap) return OVL_OK;
    drop_graph(c);
    dfree(&c->Hrs), dfree(&c->cvrs), dfree(&c->innrs);
    c->krs_cap = 0;
    const size_t ie = std::max(ovl::inner_work_elems(K, 1), ovl::inner_work_elems(K, 2));
    int r;
    if ((r = dalloc(c, &c->Hrs, sizeof(double2) * (size_t)(K + 1) * (K + 1))) ||
        (r = dalloc(c, &c->cvrs, sizeof(double2) * (size_t)(K + 1))) || (r = dalloc(c, &c->innrs, sizeof(double2) * ie)))
        return r;
    c->krs_cap = K;
    c->innrs_elems = ie;
    return OVL_OK;
}

// small dense complex inverse (Gauss-Jordan, partial pivoting) on the host; returns false if singular
bool host_inverse(std::vector<std::complex<double>>& A, int m) {
    std::vector<int> piv(m);
    std::vector<std::complex<double>> X(A);
    std::vector<std::complex<double>> I((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
    for (int p = 0; p < m; ++p) {
        int r = p;
        for (int i = p + 1; i < m; ++i)
            if (std::abs(X[(size_t)i * m + p]) > std::abs(X[(size_t)r * m + p])) r = i;
        if (std::abs(X[(size_t)r * m + p]) < 1e-300) return false;
        if (r != p)
            for (int j = 0; j < m; ++j) std::swap(X[(size_t)r * m + j], X[(size_t)p * m + j]), std::swap(I[(size_t)r * m + j], I[(size_t)p * m + j]);
        const std::complex<double> ip = 1.0 / X[(size_t)p * m + p];
        for (int j = 0; j < m; ++j) X[(size_t)p * m + j] *= ip, I[(size_t)p * m + j] *= ip;
        for (int i = 0; i < m; ++i) {
            if (i == p) continue;
            const std::complex<double> f = X[(size_t)i * m + p];
            if (f == 0.0) continue;
            for (int j = 0; j < m; ++j) X[(size_t)i * m + j] -= f * X[(size_t)p * m + j], I[(size_t)i * m + j] -= f * I[(size_t)p * m + j];
        }
    }
    A = I;
    return true;
}

// Bi-orthonormalise and install m eigenpairs given in the device layout.
int install_deflation(ovl_ctx* c, double mu, double kappa, int m, const double* lambda, const double2* Rdev,
                      const double2* Ldev) {
    const size_t n = c->n, vb = n * sizeof(double2);
    int r = ensure_base(c);
    if (r) return r;
    drop_graph(c);
    // sgn is undefined on the imaginary axis (Sec. 1, Eq. 1.4)
    double lmax = 0;
    for (int j = 0; j < m; ++j) lmax = std::max(lmax, std::hypot(lambda[2 * j], lambda[2 * j + 1]));
    for (int j = 0; j < m; ++j)
        if (std::fabs(lambda[2 * j]) <= 1e-12 * lmax)
            return fail(c, OVL_ESINGULAR, "deflated eigenvalue on the imaginary axis");
    if (m > 64) return fail(c, OVL_EINVAL, "at most 64 deflated eigenpairs");
    if (m > c->mcap) {
        dfree(&c->R), dfree(&c->L), dfree(&c->lam), dfree(&c->R32), dfree(&c->L32);
        if ((r = dalloc(c, &c->R, vb * m)) || (r = dalloc(c, &c->L, vb * m)) ||
            (r = dalloc(c, &c->lam, sizeof(double2) * m)) || (r = dalloc(c, &c->R32, n * sizeof(float2) * m)) ||
            (r = dalloc(c, &c->L32, n * sizeof(float2) * m)))
            return r;
        c->mcap = m;
    }
    if (Rdev != c->R) CUDA_TRY(c, cudaMemcpyAsync(c->R, Rdev, vb * m, cudaMemcpyDeviceToDevice, c->st));
    if (Ldev != c->L) CUDA_TRY(c, cudaMemcpyAsync(c->L, Ldev, vb * m, cudaMemcpyDeviceToDevice, c->st));
    CUDA_TRY(c, cudaMemcpyAsync(c->lam, lambda, sizeof(double2) * m, cudaMemcpyHostToDevice, c->st));
    c->m = m;
    r = ensure_solve(c, std::max(c->kcap, std::max(m, 1)));
    if (r) return r;
    // M = L^dag R, column-major: M[i + j*m] = l_i^dag r_j
    double2* Md = c->inner;
    for (int j = 0; j < m; ++j)
        ovl::launch_multidot(c->L, n, m, c->R + (size_t)j * n, Md + (size_t)j * m, 0, c->partials, n, c->st);
    std::vector<std::complex<double>> M((size_t)m * m);
    CUDA_TRY(c, cudaMemcpyAsync(M.data(), Md, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    std::vector<std::complex<double>> A((size_t)m * m);  // row-major M
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = M[i + (size_t)j * m];
    if (!host_inverse(A, m)) return fail(c, OVL_ESINGULAR, "L^dag R is singular");
    // L_new = L (M^-1)^dag:  l'_j = sum_i conj(Minv[j][i]) l_i, formed in V64 scratch
    r = ensure_solve(c, std::max(c->kcap, m));
    if (r) return r;
    CUDA_TRY(c, cudaMemsetAsync(c->V64, 0, vb * m, c->st));
    KState zero;
    std::memset(&zero, 0, sizeof(zero));
    CUDA_TRY(c, cudaMemcpyAsync(c->ks, &zero, sizeof(KState), cudaMemcpyHostToDevice, c->st));
    std::vector<std::complex<double>> neg((size_t)m * m);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) neg[(size_t)j * m + i] = -std::conj(A[(size_t)j * m + i]);
    CUDA_TRY(c, cudaMemcpyAsync(c->inner, neg.data(), sizeof(double2) * m * m, cudaMemcpyHostToDevice, c->st));
    for (int j = 0; j < m; ++j)
        ovl::launch_multiaxpy(c->L, n, m, c->inner + (size_t)j * m, c->V64 + (size_t)j * n, c->partials, c->counter,
                              c->ks, 0, n, c->st);
    CUDA_TRY(c, cudaMemcpyAsync(c->L, c->V64, vb * m, cudaMemcpyDeviceToDevice, c->st));
    // check bi-orthonormality
    for (int j = 0; j < m; ++j)
        ovl::launch_multidot(c->L, n, m, c->R + (size_t)j * n, Md + (size_t)j * m, 0, c->partials, n, c->st);
    CUDA_TRY(c, cudaMemcpyAsync(M.data(), Md, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    double dev = 0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) dev = std::max(dev, std::abs(M[i + (size_t)j * m] - (i == j ? 1.0 : 0.0)));
    if (dev > 1e-8) {
        c->m = 0;
        return fail(c, OVL_ESINGULAR, "L^dag R not bi-orthonormal after normalisation");
    }
    ovl::launch_native_f64_to_f32(c->R, c->R32, c->g, m, c->st);
    ovl::launch_native_f64_to_f32(c->L, c->L32, c->g, m, c->st);
    c->dmu = mu;
    c->dkappa = kappa;
    return OVL_OK;
}

cudaEvent_t prof_event(ovl_ctx* c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// Runs `launch` (one kernel class) bracketed by two events when profiling.
template <class F>
void prof(ovl_ctx* c, int cls, F&& launch, int kernels = -1) {
    if (!c->prof_on) {
        launch();
        return;
    }
    ProfRec r;
    r.cls = cls;
    r.kernels = kernels >= 0 ? kernels : kclass_kernels[cls];
    r.a = prof_event(c);
    r.b = prof_event(c);
    cudaEventRecord(r.a, c->st);
    launch();
    cudaEventRecord(r.b, c->st);
    c->recs.push_back(r);
}

void prof_collect(ovl_ctx* c) {
    for (const ProfRec& r : c->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_launches[r.cls] += 1;
        c->prof_kernels[r.cls] += r.kernels;
        c->prof_ms[r.cls] += ms;
    }
    c->recs.clear();
    c->ev_used = 0;
}

// Queue the whole solve (everything between packing b and unpacking y).
// c = |b_perp| sgn(H_k) e_1 for Arnoldi: the resolvent quadrature with Givens-rotation solves of
// the shifted Hessenberg systems, and Roberts/Newton only if it did not converge (or on request)
int arnoldi_inner_sign(ovl_ctx* c, int ldH, int flags) {
    cudaStream_t st = c->st;
    if (!(flags & OVL_INNER_NEWTON)) {
        const int q = ovl::launch_inner_quadrature_hess(c->H, ldH, c->ks, c->cvec, c->inner, c->inner_elems,
                                                        c->kcap, c->partials, c->counter, st);
        if (q == 0)
            return ovl::launch_inner_newton(nullptr, nullptr, nullptr, c->H, ldH, 0, c->ks, c->cvec, c->inner,
                                            c->inner_elems, c->kcap, c->num_sms, st, 1);
    }
    return ovl::launch_inner_newton(nullptr, nullptr, nullptr, c->H, ldH, 0, c->ks, c->cvec, c->inner,
                                    c->inner_elems, c->kcap, c->num_sms, st);
}

int enqueue_solve(ovl_ctx* c, int method, int k, double mu, double kappa, int flags) {
    cudaStream_t st = c->st;
    const size_t n = c->n;
    const Geom& g = c->g;
    KState* ks = c->ks;
    double* part = c->partials;
    unsigned int* cnt = c->counter;
    const bool mixed = (flags & OVL_MIXED) != 0;
    const bool twopass = mixed || (flags & OVL_TWO_PASS);
    const int m = c->m;
    const int mproj = (flags & OVL_REPROJ) ? m : 0;
    const int rperiod = (flags & OVL_REPROJ) ? std::max(1, (flags >> 24) & 0x7f) : 1;  // OVL_REPROJ_PERIOD

    prof(c, KC_SETUP, [&] { ovl::launch_state_init(ks, st); });
    if (m > 0) {
        prof(c, KC_DEFLATE, [&] {
            ovl::launch_multidot(c->L, n, m, c->b64, c->pq, 0, part, n, st);
            ovl::launch_multidot(c->R, n, m, c->b64, c->pq + m, 0, part, n, st);
        }, 4);
    }
    if (method == OVL_LANCZOS2) {
        double2* v0 = twopass ? c->bR : c->V64;
        double2* w0 = twopass ? c->bL : c->W64[0];
        prof(c, KC_DEFLATE, [&] {
            ovl::launch_deflate_split(c->b64, c->R, c->L, c->lam, m, c->pq, v0, w0, c->y64, ks, c->vscale, part,
                                      cnt, n, st);
        });
        if (mixed) {
            prof(c, KC_CONVERT, [&] {
                ovl::launch_native_f64_to_f32(c->bR, c->v32[0], g, 1, st);
                ovl::launch_native_f64_to_f32(c->bL, c->w32[0], g, 1, st);
            }, 2);
        } else if (twopass) {
            cudaMemcpyAsync(c->R64[0], c->bR, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(c->W64[0], c->bL, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
        }
        // pass 1: basis (stored for one-pass FP64) and coefficients
        const bool persist = mixed && !(flags & OVL_STEPWISE) && rperiod == 1 && ovl::persistent_ok(g, c->num_sms);
        if (persist) {
            cudaMemsetAsync(c->bar, 0, 64, st);
            int lr = 0;
            prof(c, KC_PASS1, [&] {
                float4* vv[3] = {(float4*)c->v32[0], (float4*)c->v32[1], (float4*)c->v32[2]};
                float4* ww[3] = {(float4*)c->w32[0], (float4*)c->w32[1], (float4*)c->w32[2]};
                lr = ovl::launch_pass1_persistent(c->U12, vv, ww, ks, c->alpha, c->beta, c->gamma, c->R32, c->L32,
                                                  mproj, mu, kappa, k, part, c->bar, g, c->num_sms, st,
                                                  c->wait_polls, c->wait_unreachable);
            });
            if (lr) return fail(c, OVL_ECUDA, std::string("persistent pass 1 launch: ") +
                                                   cudaGetErrorString((cudaError_t)lr));
        }
        for (int i = 0; i < (persist ? 0 : k); ++i) {
            if (mixed) {
                prof(c, KC_PAIR, [&] {
                    ovl::launch_dslash_pair(c->U12, 1, c->v32[i % 3], c->w32[i % 3], c->t32, c->s32, mu, kappa, ks,
                                            c->alpha, i, k - 1, part, cnt, g, st);
                });
                // optional re-projection of the deflated directions (p = L^dag t, q = R^dag s), at the
                // steps the period selects
                double2* pq2 = c->pq + 2048;
                const int mp = (i + 1) % rperiod == 0 ? mproj : 0;
                if (i + 1 < k && mp > 0)
                    prof(c, KC_DEFLATE, [&] {
                        ovl::launch_multidot_f32(c->L32, n, mp, c->t32, pq2, part, n, st, ks);
                        ovl::launch_multidot_f32(c->R32, n, mp, c->s32, pq2 + mp, part, n, st, ks);
                    }, 4);
                if (i + 1 < k)
                    prof(c, KC_LSTEP, [&] {
                        ovl::launch_lanczos_step(1, c->t32, c->s32, c->v32[i % 3], c->w32[i % 3],
                                                 c->v32[(i + 2) % 3], c->w32[(i + 2) % 3], c->v32[(i + 1) % 3],
                                                 c->w32[(i + 1) % 3], ks, c->alpha, c->beta, c->gamma, c->vscale, i,
                                                 k, part, cnt, n, st, c->R32, c->L32, pq2, mp);
                    });
            } else {
                const double2* vi = twopass ? c->R64[i % 3] : c->V64 + (size_t)i * n;
                const double2* vim1 = twopass ? c->R64[(i + 2) % 3] : (i > 0 ? c->V64 + (size_t)(i - 1) * n : c->V64);
                double2* vn = twopass ? c->R64[(i + 1) % 3] : c->V64 + (size_t)(i + 1) * n;
                prof(c, KC_PAIR, [&] {
                    ovl::launch_dslash_pair(c->U64, 0, vi, c->W64[i % 3], c->t64, c->s64, mu, kappa, ks, c->alpha, i,
                                            k - 1, part, cnt, g, st);
                });
                if (i + 1 < k)
                    prof(c, KC_LSTEP, [&] {
                        ovl::launch_lanczos_step(0, c->t64, c->s64, vi, c->W64[i % 3], vim1, c->W64[(i + 2) % 3], vn,
                                                 c->W64[(i + 1) % 3], ks, c->alpha, c->beta, c->gamma, c->vscale, i,
                                                 k, part, cnt, n, st);
                    });
            }
        }
        // inner sign
        int r = 0;
        if (flags & OVL_INNER_NEWTON)
            prof(c, KC_INNER, [&] {
                r = ovl::launch_inner_newton(c->alpha, c->beta, c->gamma, nullptr, 0, 1, ks, c->cvec, c->inner,
                                             c->inner_elems, c->kcap, c->num_sms, st);
            }, 2);
        else
            prof(c, KC_INNER, [&] {
                r = ovl::launch_inner_quadrature(c->alpha, c->beta, c->gamma, ks, c->cvec, c->inner,
                                                 c->inner_elems, c->kcap, part, cnt, st);
                // Roberts/Newton only if the quadrature did not converge (Ritz values near the axis)
                if (!r)
                    r = ovl::launch_inner_newton(c->alpha, c->beta, c->gamma, nullptr, 0, 1, ks, c->cvec, c->inner,
                                                 c->inner_elems, c->kcap, c->num_sms, st, 1);
            }, 15);
        if (r) return fail(c, OVL_ECUDA, "inner sign launch failed");
        // combination y += |b_perp^R| V_k sgn(G_k) e_1
        if (twopass && persist) {
            prof(c, KC_COMBINE, [&] { ovl::launch_scale_start(c->bR, c->R64[0], c->y64, c->cvec, ks, n, st); });
            int lr = 0;
            prof(c, KC_PASS2, [&] {
                double2* rr[3] = {c->R64[0], c->R64[1], c->R64[2]};
                const float4* udf = (mixed && (flags & OVL_PASS2_DF)) ? c->Udf : nullptr;
                lr = ovl::launch_pass2_persistent(c->U64, udf, rr, c->y64, ks, c->alpha, c->beta, c->gamma, c->cvec,
                                                  c->H, c->kcap, mu, kappa, c->bar, &ks->timeout, g, c->num_sms,
                                                  st);
            });
            if (lr) return fail(c, OVL_ECUDA, std::string("persistent pass 2 launch: ") +
                                                   cudaGetErrorString((cudaError_t)lr));
        } else if (twopass) {
            prof(c, KC_COMBINE, [&] { ovl::launch_scale_start(c->bR, c->R64[0], c->y64, c->cvec, ks, n, st); });
            for (int i = 0; i + 1 < k; ++i)
                prof(c, KC_REGEN, [&] {
                    ovl::launch_dslash_regen(c->U64, c->R64[i % 3], c->R64[(i + 2) % 3], c->R64[(i + 1) % 3],
                                             c->y64, mu, kappa, ks, c->alpha, c->beta, c->gamma, c->cvec, i, g, st);
                });
        } else {
            prof(c, KC_COMBINE, [&] { ovl::launch_combine(c->V64, n, c->vscale, c->cvec, ks, c->kcap, c->y64, n, st); });
        }
    } else if (flags & OVL_MIXED) {  // Arnoldi, double-float basis (csrc/arnoldi_df.cu)
        prof(c, KC_DEFLATE, [&] {
            ovl::launch_deflate_split(c->b64, c->R, c->L, c->lam, m, c->pq, c->bR, nullptr, c->y64, ks, nullptr,
                                      part, cnt, n, st);
        });
        // V64 holds kcap + 1 double-float vectors (same 16 bytes per complex element); the
        // two-sided Lanczos coefficient arrays (kcap + 1 entries each, unused by Arnoldi) hold the
        // double-float copies of h1, h2 and of the combination coefficients
        float4* Vd = reinterpret_cast<float4*>(c->V64);
        float4* h1d = reinterpret_cast<float4*>(c->alpha);
        float4* h2d = reinterpret_cast<float4*>(c->beta);
        float4* cdf = reinterpret_cast<float4*>(c->gamma);
        double2* x64 = c->s64;  // FP64 value of v_j, the stencil's input
        prof(c, KC_ANORM, [&] { ovl::launch_adf_start(c->bR, Vd, x64, ks, n, st); });
        const int ldH = c->kcap + 1;
        // default: delayed CGS2 (two basis sweeps per step); OVL_ARNOLDI_CGS2: the classical form below
        if (!(flags & OVL_ARNOLDI_CGS2)) {
            for (int j = 0; j < k; ++j) {
                float4* uj = Vd + (size_t)j * n;
                float4* un = Vd + (size_t)(j + 1) * n;
                prof(c, KC_ADSLASH, [&] { ovl::launch_dslash(c->U64, 0, x64, c->t64, mu, kappa, 1, g, st, ks); });
                prof(c, KC_ADOT, [&] {
                    ovl::launch_adf_dot2(Vd, n, j + 1, uj, c->t64, c->h1, c->h2, part, n, c->num_sms, ks, st);
                }, 2);
                prof(c, KC_ANORM, [&] { ovl::launch_adf_dcgs(c->H, ldH, c->h1, c->h2, h1d, h2d, ks, j, 0, st); });
                prof(c, KC_AAXPY, [&] {
                    ovl::launch_adf_update2(Vd, n, j, h1d, h2d, uj, un, c->t64, x64, c->H, ldH, c->h1, c->h2, n, ks,
                                            st);
                });
            }
            // re-orthogonalise u_k against V_0..V_{k-1}: finishes column k - 1 of H
            prof(c, KC_ADOT, [&] {
                ovl::launch_adf_dot(Vd, n, k + 1, Vd + (size_t)k * n, c->h1, h1d, part, n, c->num_sms, ks, st);
            }, 2);
            prof(c, KC_ANORM, [&] { ovl::launch_adf_dcgs(c->H, ldH, c->h1, c->h2, h1d, h2d, ks, k, 1, st); });
        } else
        for (int j = 0; j < k; ++j) {
            float4* t = Vd + (size_t)(j + 1) * n;
            prof(c, KC_ADSLASH, [&] {
                ovl::launch_dslash(c->U64, 0, x64, c->t64, mu, kappa, 1, g, st, ks);
                ovl::launch_adf_todf(c->t64, t, ks, n, st);
            }, 2);
            prof(c, KC_ADOT, [&] { ovl::launch_adf_dot(Vd, n, j + 1, t, c->h1, h1d, part, n, c->num_sms, ks, st); }, 2);
            prof(c, KC_AAXPY, [&] { ovl::launch_adf_update(Vd, n, j + 1, h1d, t, n, ks, part, cnt, st); });
            prof(c, KC_ADOT, [&] { ovl::launch_adf_dot(Vd, n, j + 1, t, c->h2, h2d, part, n, c->num_sms, ks, st); }, 2);
            prof(c, KC_AAXPY, [&] {
                ovl::launch_adf_update_fin(Vd, n, j + 1, h2d, t, c->H, ldH, c->h1, c->h2, j, k - 1, part, cnt, ks,
                                           n, st);
            });
            prof(c, KC_ANORM, [&] { ovl::launch_adf_normalize(t, x64, ks, n, st); });
        }
        int r = 0;
        prof(c, KC_INNER, [&] { r = arnoldi_inner_sign(c, ldH, flags); }, (flags & OVL_INNER_NEWTON) ? 2 : 15);
        if (r) return fail(c, OVL_ECUDA, "inner sign launch failed");
        prof(c, KC_COMBINE, [&] { ovl::launch_adf_combine(Vd, n, c->cvec, cdf, ks, c->kcap, c->y64, n, st); }, 2);
    } else {  // Arnoldi
        prof(c, KC_DEFLATE, [&] {
            ovl::launch_deflate_split(c->b64, c->R, c->L, c->lam, m, c->pq, c->bR, nullptr, c->y64, ks, nullptr,
                                      part, cnt, n, st);
        });
        prof(c, KC_ANORM, [&] { ovl::launch_scale_start(c->bR, c->V64, nullptr, nullptr, ks, n, st); });
        const int ldH = c->kcap + 1;
        for (int j = 0; j < k; ++j) {
            double2* vj = c->V64 + (size_t)j * n;
            double2* t = c->V64 + (size_t)(j + 1) * n;
            prof(c, KC_ADSLASH, [&] { ovl::launch_dslash(c->U64, 0, vj, t, mu, kappa, 1, g, st, ks); });
            prof(c, KC_ADOT, [&] { ovl::launch_multidot(c->V64, n, j + 1, t, c->h1, 0, part, n, st, ks); });
            prof(c, KC_AAXPY, [&] { ovl::launch_multiaxpy(c->V64, n, j + 1, c->h1, t, part, cnt, ks, 0, n, st); });
            prof(c, KC_ADOT, [&] { ovl::launch_multidot(c->V64, n, j + 1, t, c->h2, 0, part, n, st, ks); });
            prof(c, KC_AAXPY, [&] {
                ovl::launch_arnoldi_orth2(c->V64, n, j + 1, c->h2, t, c->H, ldH, c->h1, j, k - 1, part, cnt, ks, n,
                                          st);
            });
            prof(c, KC_ANORM, [&] { ovl::launch_arnoldi_normalize(t, ks, n, st); });
        }
        int r = 0;
        prof(c, KC_INNER, [&] { r = arnoldi_inner_sign(c, ldH, flags); }, (flags & OVL_INNER_NEWTON) ? 2 : 15);
        if (r) return fail(c, OVL_ECUDA, "inner sign launch failed");
        prof(c, KC_COMBINE, [&] { ovl::launch_combine(c->V64, n, nullptr, c->cvec, ks, c->kcap, c->y64, n, st); });
    }
    return OVL_OK;
}

int enqueue_restarted(ovl_ctx* c, int rs, int cycles, double mu, double kappa, int flags) {
    cudaStream_t st = c->st;
    const size_t n = c->n;
    const Geom& g = c->g;
    KState* ks = c->ks;
    double* part = c->partials;
    unsigned int* cnt = c->counter;
    const int m = c->m;
    const int K = rs * cycles, ldH = c->krs_cap + 1;
    prof(c, KC_SETUP, [&] { ovl::launch_state_init(ks, st); });
    if (m > 0) {
        prof(c, KC_DEFLATE, [&] {
            ovl::launch_multidot(c->L, n, m, c->b64, c->pq, 0, part, n, st);
            ovl::launch_multidot(c->R, n, m, c->b64, c->pq + m, 0, part, n, st);
        }, 4);
    }
    prof(c, KC_DEFLATE, [&] {
        ovl::launch_deflate_split(c->b64, c->R, c->L, c->lam, m, c->pq, c->bR, nullptr, c->y64, ks, nullptr, part, cnt,
                                  n, st);
    });
    // double-float basis in V64's slots 0..rs; the two-sided Lanczos coefficient arrays hold the
    // double-float coefficient copies (see the unrestarted double-float Arnoldi)
    float4* Vd = reinterpret_cast<float4*>(c->V64);
    float4* h1d = reinterpret_cast<float4*>(c->alpha);
    float4* h2d = reinterpret_cast<float4*>(c->beta);
    float4* cdf = reinterpret_cast<float4*>(c->gamma);
    double2* x64 = c->s64;
    // the accumulated matrix is block lower bidiagonal: everything outside the blocks and their
    // coupling entries is zero
    CUDA_TRY(c, cudaMemsetAsync(c->Hrs, 0, sizeof(double2) * (size_t)ldH * K, st));
    prof(c, KC_ANORM, [&] { ovl::launch_adf_start(c->bR, Vd, x64, ks, n, st); });
    for (int cyc = 0; cyc < cycles; ++cyc) {
        double2* Hc = c->Hrs + (size_t)cyc * rs * (1 + (size_t)ldH);
        prof(c, KC_SETUP, [&] { ovl::launch_rs_begin(ks, cyc, st); });
        for (int j = 0; j < rs; ++j) {
            float4* uj = Vd + (size_t)j * n;
            float4* un = Vd + (size_t)(j + 1) * n;
            prof(c, KC_ADSLASH, [&] { ovl::launch_dslash(c->U64, 0, x64, c->t64, mu, kappa, 1, g, st, ks); });
            prof(c, KC_ADOT, [&] {
                ovl::launch_adf_dot2(Vd, n, j + 1, uj, c->t64, c->h1, c->h2, part, n, c->num_sms, ks, st);
            }, 2);
            prof(c, KC_ANORM, [&] { ovl::launch_adf_dcgs(Hc, ldH, c->h1, c->h2, h1d, h2d, ks, j, 0, st); });
            prof(c, KC_AAXPY, [&] {
                ovl::launch_adf_update2(Vd, n, j, h1d, h2d, uj, un, c->t64, x64, Hc, ldH, c->h1, c->h2, n, ks, st);
            });
        }
        // re-orthogonalise u_rs: finishes the cycle's last column and its coupling entry
        prof(c, KC_ADOT, [&] {
            ovl::launch_adf_dot(Vd, n, rs + 1, Vd + (size_t)rs * n, c->h1, h2d, part, n, c->num_sms, ks, st);
        }, 2);
        prof(c, KC_ANORM, [&] { ovl::launch_adf_dcgs(Hc, ldH, c->h1, c->h2, h1d, h2d, ks, rs, 2, st); });
        prof(c, KC_SETUP, [&] { ovl::launch_rs_mid(ks, st); });
        // inner sign of the accumulated matrix, then this cycle's share of the combination
        int r = 0;
        prof(c, KC_INNER, [&] {
            if (!(flags & OVL_INNER_NEWTON)) {
                const int q = ovl::launch_inner_quadrature_hess(c->Hrs, ldH, ks, c->cvrs, c->innrs, c->innrs_elems,
                                                                c->krs_cap, part, cnt, st);
                r = q ? q
                      : ovl::launch_inner_newton(nullptr, nullptr, nullptr, c->Hrs, ldH, 0, ks, c->cvrs, c->innrs,
                                                 c->innrs_elems, c->krs_cap, c->num_sms, st, 1);
            } else {
                r = ovl::launch_inner_newton(nullptr, nullptr, nullptr, c->Hrs, ldH, 0, ks, c->cvrs, c->innrs,
                                             c->innrs_elems, c->krs_cap, c->num_sms, st);
            }
        }, (flags & OVL_INNER_NEWTON) ? 2 : 15);
        if (r) return fail(c, OVL_ECUDA, "inner sign launch failed");
        prof(c, KC_COMBINE, [&] { ovl::launch_rs_combine(Vd, n, c->cvrs, cyc * rs, cdf, ks, rs, c->y64, n, st); }, 2);
        prof(c, KC_ANORM, [&] { ovl::launch_rs_restart(Vd, n, rs, h1d, x64, ks, n, cyc + 1 == cycles, st); });
    }
    return OVL_OK;
}

}  // namespace

extern "C" {

int ovl_create(ovl_ctx** out, const int dims[4], int bc_t, void* stream) {
    if (!out || !dims) return OVL_EINVAL;
    *out = nullptr;
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2) return OVL_EINVAL;
    if (dims[3] % 2) return OVL_EINVAL;
    if (bc_t != 1 && bc_t != -1) return OVL_EINVAL;
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (1ll << 28)) return OVL_EINVAL;
    ovl_ctx* c = new ovl_ctx();
    for (int d = 0; d < 4; ++d) c->g.L[d] = dims[d];
    c->g.L4h = dims[3] / 2;
    c->g.V = (int)V;
    c->g.Vh = (int)(V / 2);
    c->g.bc_t = bc_t;
    c->n = (size_t)12 * V;
    c->st = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return OVL_ECUDA;
    }
    *out = c;
    return OVL_OK;
}

int ovl_destroy(ovl_ctx* c) {
    if (!c) return OVL_OK;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    drop_graph(c);
    free_solve(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    dfree(&c->U64), dfree(&c->U12), dfree(&c->U18), dfree(&c->Udf), dfree(&c->nbr);
    dfree(&c->R), dfree(&c->L), dfree(&c->lam), dfree(&c->R32), dfree(&c->L32);
    dfree(&c->b64), dfree(&c->y64), dfree(&c->bR), dfree(&c->bL), dfree(&c->t64), dfree(&c->s64);
    dfree(&c->t32), dfree(&c->s32), dfree(&c->ks), dfree(&c->counter), dfree(&c->bar), dfree(&c->stage_in),
        dfree(&c->stage_out);
    dfree(&c->nat_a), dfree(&c->nat_b), dfree(&c->pq);
    dfree(&c->gwork), dfree(&c->tadj);
    dfree(&c->Hrs), dfree(&c->cvrs), dfree(&c->innrs);
    for (int i = 0; i < 3; ++i) dfree(&c->W64[i]), dfree(&c->R64[i]), dfree(&c->v32[i]), dfree(&c->w32[i]);
    delete c;
    return OVL_OK;
}

const char* ovl_last_error(const ovl_ctx* c) { return c ? c->err.c_str() : "null context"; }

int ovl_set_stream(ovl_ctx* c, void* stream) {
    if (!c) return OVL_EINVAL;
    if (c->st != (cudaStream_t)stream) drop_graph(c);
    c->st = (cudaStream_t)stream;
    return OVL_OK;
}

size_t ovl_vector_bytes(const ovl_ctx* c, int prec) {
    if (!c) return 0;
    return c->n * (prec == 0 ? sizeof(double2) : sizeof(float2));
}

int ovl_set_gauge(ovl_ctx* c, const void* U, int flags) {
    if (!c || !U) return fail(c, OVL_EINVAL, "null argument");
    const size_t V = c->g.V;
    int r;
    if ((r = dalloc(c, &c->U64, V * 36 * sizeof(double2))) || (r = dalloc(c, &c->U12, V * 12 * sizeof(float4))) ||
        (r = dalloc(c, &c->U18, V * 36 * sizeof(float2))) || (r = dalloc(c, &c->Udf, V * 36 * sizeof(float4))) ||
        (r = dalloc(c, &c->nbr, V * 8 * sizeof(int))))
        return r;
    const double2* src = (const double2*)U;
    double2* tmp = nullptr;
    if (flags & OVL_HOST) {
        if ((r = dalloc(c, &tmp, V * 36 * sizeof(double2)))) return r;
        CUDA_TRY(c, cudaMemcpyAsync(tmp, U, V * 36 * sizeof(double2), cudaMemcpyHostToDevice, c->st));
        src = tmp;
    }
    ovl::launch_pack_gauge(src, c->U64, c->U12, c->U18, c->Udf, c->g, c->st);
    ovl::launch_build_nbr(c->nbr, c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());
    if (tmp) {
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
        cudaFree(tmp);
    }
    c->have_gauge = true;
    drop_graph(c);
    return OVL_OK;
}

int ovl_pack(ovl_ctx* c, const void* canon, void* native, int prec) {
    if (!c || !canon || !native || prec < 0 || prec > 1) return fail(c, OVL_EINVAL, "bad argument");
    ovl::launch_pack_spinor((const double2*)canon, native, prec, c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());
    return OVL_OK;
}

int ovl_unpack(ovl_ctx* c, const void* native, void* canon, int prec) {
    if (!c || !canon || !native || prec < 0 || prec > 1) return fail(c, OVL_EINVAL, "bad argument");
    ovl::launch_unpack_spinor(native, prec, (double2*)canon, nullptr, 0, c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());
    return OVL_OK;
}

int ovl_apply_Dw(ovl_ctx* c, double mu, double kappa, const void* x, void* y, int flags) {
    if (!c || !x || !y) return fail(c, OVL_EINVAL, "null argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    if (x == y) return fail(c, OVL_EINVAL, "x and y must not overlap");
    const int prec = (flags & OVL_F32) ? 1 : (flags & OVL_F32_FULL) ? 2 : 0;
    const void* U = prec == 0 ? (const void*)c->U64 : prec == 1 ? (const void*)c->U12 : (const void*)c->U18;
    const int g5 = (flags & (OVL_GAMMA5 | OVL_DAGGER)) ? 1 : 0;
    const double m = (flags & OVL_DAGGER) ? -mu : mu;
    struct VariantGuard {
        explicit VariantGuard(int f) { ovl::set_dslash_variant(f & OVL_STENCIL_SITE ? 0 : f & OVL_STENCIL_SPLIT ? 1 : -1); }
        ~VariantGuard() { ovl::set_dslash_variant(-1); }
    } vg(flags);
    if (flags & OVL_NATIVE) {
        if (flags & OVL_HOST) return fail(c, OVL_EINVAL, "OVL_NATIVE vectors must be device memory");
        ovl::launch_dslash(U, prec, x, y, m, kappa, g5, c->g, c->st);
        CUDA_TRY(c, cudaGetLastError());
        return OVL_OK;
    }
    int r = ensure_base(c);
    if (r) return r;
    const size_t cb = c->n * sizeof(double2);
    const double2* xin = (const double2*)x;
    if (flags & OVL_HOST) {
        CUDA_TRY(c, cudaMemcpyAsync(c->stage_in, x, cb, cudaMemcpyHostToDevice, c->st));
        xin = c->stage_in;
    }
    const int vprec = prec == 0 ? 0 : 1;
    ovl::launch_pack_spinor(xin, c->nat_a, vprec, c->g, c->st);
    ovl::launch_dslash(U, prec, c->nat_a, c->nat_b, m, kappa, g5, c->g, c->st);
    double2* yout = (flags & OVL_HOST) ? c->stage_out : (double2*)y;
    ovl::launch_unpack_spinor(c->nat_b, vprec, yout, nullptr, 0, c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());
    if (flags & OVL_HOST) {
        CUDA_TRY(c, cudaMemcpyAsync(y, c->stage_out, cb, cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
    return OVL_OK;
}

int ovl_apply_pair(ovl_ctx* c, double mu, double kappa, int prec, const void* v, const void* w, void* t, void* s,
                   double* alpha_host) {
    if (!c || !v || !w || !t || !s || prec < 0 || prec > 1) return fail(c, OVL_EINVAL, "bad argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    int r = ensure_solve(c, std::max(c->kcap, 1));
    if (r) return r;
    ovl::launch_state_init(c->ks, c->st);
    ovl::launch_dslash_pair(prec == 0 ? (const void*)c->U64 : (const void*)c->U12, prec, v, w, t, s, mu, kappa, c->ks,
                            c->alpha, 0, 1 << 30, c->partials, c->counter, c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());
    if (alpha_host) {
        CUDA_TRY(c, cudaMemcpyAsync(alpha_host, c->alpha, sizeof(double2), cudaMemcpyDeviceToHost, c->st));
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
    return OVL_OK;
}

int ovl_set_deflation(ovl_ctx* c, double mu, double kappa, int m, const double* lambda, const void* R, const void* L,
                      int flags) {
    if (!c || m < 0 || m > 1024) return fail(c, OVL_EINVAL, "bad argument");
    drop_graph(c);
    if (m == 0) {
        c->m = 0;
        return OVL_OK;
    }
    if (!lambda || !R || !L) return fail(c, OVL_EINVAL, "null argument");
    int r = ensure_base(c);
    if (r) return r;
    const size_t n = c->n, vb = n * sizeof(double2);
    double2 *Rt = nullptr, *Lt = nullptr;
    if ((r = dalloc(c, &Rt, vb * m)) || (r = dalloc(c, &Lt, vb * m))) {
        dfree(&Rt);
        return r;
    }
    // pack the eigenvectors into the device layout
    for (int j = 0; j < m && !r; ++j) {
        for (int side = 0; side < 2; ++side) {
            const double2* src = (const double2*)(side == 0 ? R : L) + (size_t)j * n;
            if (flags & OVL_HOST) {
                if (cudaMemcpyAsync(c->stage_in, src, vb, cudaMemcpyHostToDevice, c->st) != cudaSuccess) {
                    r = fail(c, OVL_ECUDA, "copy of an eigenvector failed");
                    break;
                }
                src = c->stage_in;
            }
            ovl::launch_pack_spinor(src, (side == 0 ? Rt : Lt) + (size_t)j * n, 0, c->g, c->st);
            if (flags & OVL_HOST) cudaStreamSynchronize(c->st);
        }
    }
    if (!r) r = install_deflation(c, mu, kappa, m, lambda, Rt, Lt);
    cudaStreamSynchronize(c->st);
    dfree(&Rt);
    dfree(&Lt);
    return r;
}

int ovl_get_deflation(ovl_ctx* c, int* m_out, double* lambda, void* R, void* L, int flags) {
    if (!c) return OVL_EINVAL;
    if (m_out) *m_out = c->m;
    const size_t n = c->n, vb = n * sizeof(double2);
    if (lambda && c->m) CUDA_TRY(c, cudaMemcpyAsync(lambda, c->lam, sizeof(double2) * c->m, cudaMemcpyDeviceToHost, c->st));
    for (int j = 0; j < c->m; ++j) {
        for (int side = 0; side < 2; ++side) {
            void* dst = side == 0 ? R : L;
            if (!dst) continue;
            double2* d = (flags & OVL_HOST) ? c->stage_out : (double2*)dst + (size_t)j * n;
            ovl::launch_unpack_spinor((side == 0 ? c->R : c->L) + (size_t)j * n, 0, d, nullptr, 0, c->g, c->st);
            if (flags & OVL_HOST) {
                CUDA_TRY(c, cudaMemcpyAsync((double2*)dst + (size_t)j * n, c->stage_out, vb, cudaMemcpyDeviceToHost,
                                            c->st));
                CUDA_TRY(c, cudaStreamSynchronize(c->st));
            }
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return OVL_OK;
}

}  // extern "C"

namespace {

// the common body of ovl_sign_krylov (rs = 0) and ovl_sign_arnoldi_restarted (rs = cycle length,
// k = rs x cycles): pack, queue (or replay the captured graph), unpack, read the status
int sign_solve(ovl_ctx* c, int method, int k, int rs, double mu, double kappa, const void* b, void* out, int flags,
               ovl_info* info) {
    int r = rs > 0 ? ensure_solve(c, rs) : ensure_solve(c, k);
    if (!r && rs > 0) r = ensure_restart(c, k);
    if (r) return r;
    const size_t cb = c->n * sizeof(double2);
    const double2* bin = (const double2*)b;
    if (flags & OVL_HOST) {
        CUDA_TRY(c, cudaMemcpyAsync(c->stage_in, b, cb, cudaMemcpyHostToDevice, c->st));
        bin = c->stage_in;
    }
    ovl::launch_pack_spinor(bin, c->b64, 0, c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());

    const int gflags = flags & (OVL_MIXED | OVL_TWO_PASS | OVL_INNER_NEWTON | OVL_REPROJ | OVL_REPROJ_PERIOD(0x7f) |
                                OVL_STEPWISE | OVL_PASS2_F64 | OVL_PASS2_DF | OVL_ARNOLDI_CGS2);
    bool ran = false;
    c->prof_on = (flags & OVL_PROFILE) != 0;
    if (!(flags & (OVL_NO_GRAPH | OVL_PROFILE))) {
        GraphEntry& ge = c->graph;
        if (!(ge.valid && ge.method == method && ge.k == k && ge.rs == rs && ge.flags == gflags && ge.m == c->m &&
              ge.mu == mu && ge.kappa == kappa)) {
            drop_solve_graph(c);
            cudaGraph_t graph = nullptr;
            // capture on a private stream (the caller's may be the legacy default stream, which
            // cannot be captured); the graph is then launched on the caller's stream
            if (!c->cap_st) cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking);
            cudaStream_t user_st = c->st;
            if (c->cap_st && cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                c->st = c->cap_st;
                const int er = rs > 0 ? enqueue_restarted(c, rs, k / rs, mu, kappa, gflags)
                                      : enqueue_solve(c, method, k, mu, kappa, gflags);
                const cudaError_t ec = cudaStreamEndCapture(c->cap_st, &graph);
                c->st = user_st;
                if (er == OVL_OK && ec == cudaSuccess && graph) {
                    cudaGraphExec_t exec = nullptr;
                    if (cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
                        ge.valid = true;
                        ge.method = method, ge.k = k, ge.rs = rs, ge.flags = gflags, ge.m = c->m, ge.mu = mu,
                        ge.kappa = kappa;
                        ge.exec = exec;
                    }
                }
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();  // a failed capture must not poison later calls
            }
        }
        if (ge.valid) {
            CUDA_TRY(c, cudaGraphLaunch(ge.exec, c->st));
            ran = true;
        }
    }
    if (!ran) {
        r = rs > 0 ? enqueue_restarted(c, rs, k / rs, mu, kappa, gflags) : enqueue_solve(c, method, k, mu, kappa, gflags);
        c->prof_on = false;
        if (r) return r;
    }
    double2* yout = (flags & OVL_HOST) ? c->stage_out : (double2*)out;
    ovl::launch_unpack_spinor(c->y64, 0, yout, (flags & OVL_OVERLAP) ? bin : nullptr, (flags & OVL_OVERLAP) ? 1 : 0,
                              c->g, c->st);
    CUDA_TRY(c, cudaGetLastError());
    if (flags & OVL_HOST) CUDA_TRY(c, cudaMemcpyAsync(out, c->stage_out, cb, cudaMemcpyDeviceToHost, c->st));
    KState ks;
    CUDA_TRY(c, cudaMemcpyAsync(&ks, c->ks, sizeof(KState), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (!c->recs.empty()) prof_collect(c);
    if (info) {
        info->k_used = ks.kused;
        info->breakdown_step = ks.bdstep;
        info->inner_iters = ks.inner_iters;
        info->inner_method = ks.inner_method;
        info->bperp_norm = ks.nR;
        info->inner_err = ks.inner_err;
    }
    if (ks.timeout) return fail(c, OVL_ETIMEOUT, "a bounded device wait gave up");
    if (ks.status == OVL_ESINGULAR) return fail(c, OVL_ESINGULAR, "singular projected matrix");
    if (ks.status == OVL_ENOCONV) return fail(c, OVL_ENOCONV, "inner sign did not converge");
    if (ks.status) return fail(c, ks.status, "solve failed");
    if (ks.bdstep >= 0) return fail(c, OVL_EBREAKDOWN, "two-sided Lanczos serious breakdown");
    return OVL_OK;
}

}  // namespace

extern "C" {

int ovl_sign_krylov(ovl_ctx* c, int method, int k, double mu, double kappa, const void* b, void* out, int flags,
                    ovl_info* info) {
    if (!c || !b || !out) return fail(c, OVL_EINVAL, "null argument");
    if (method != OVL_ARNOLDI && method != OVL_LANCZOS2) return fail(c, OVL_EINVAL, "unknown method");
    if (k < 1 || k > 8192) return fail(c, OVL_EINVAL, "k out of range [1, 8192]");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    if (b == out) return fail(c, OVL_EINVAL, "b and out must not overlap");
    if (c->m > 0 && (mu != c->dmu || kappa != c->dkappa))
        return fail(c, OVL_EINVAL, "mu/kappa differ from those of the installed deflation");
    if (method == OVL_ARNOLDI && (flags & OVL_TWO_PASS))
        return fail(c, OVL_EINVAL, "two-pass is defined for two-sided Lanczos only");
    // mixed two-sided Lanczos on a lattice too large for the persistent passes: the batched kernels
    // as a batch of one (the stepwise path's FP64 regeneration is bound by the FP64 pipe; the
    // batch regenerates in double-float).  Options only the stepwise path has keep it.
    if (method == OVL_LANCZOS2 && (flags & OVL_MIXED) && !(flags & ~(OVL_MIXED | OVL_OVERLAP | OVL_HOST)) &&
        !ovl::persistent_ok(c->g, c->num_sms)) {
        if (!c->self_batch) {
            const int one = 1;
            ovl_ctx* self = c;
            const int rb = ovl_batch_create(&c->self_batch, &self, 1, &one);
            if (rb) {
                c->self_batch = nullptr;
                return fail(c, rb, "one-sequence batch");
            }
        }
        const int rs = ovl_batch_solve(c->self_batch, k, mu, kappa, &b, &out, flags, info);
        if (rs) return fail(c, rs, ovl_batch_last_error(c->self_batch));
        return OVL_OK;
    }
    return sign_solve(c, method, k, 0, mu, kappa, b, out, flags, info);
}

int ovl_sign_arnoldi_restarted(ovl_ctx* c, int m, int cycles, double mu, double kappa, const void* b, void* out,
                               int flags, ovl_info* info) {
    if (!c || !b || !out) return fail(c, OVL_EINVAL, "null argument");
    if (m < 1 || cycles < 1 || (long long)m * cycles > 8192)
        return fail(c, OVL_EINVAL, "m >= 1, cycles >= 1 and m x cycles <= 8192 required");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    if (b == out) return fail(c, OVL_EINVAL, "b and out must not overlap");
    if (c->m > 0 && (mu != c->dmu || kappa != c->dkappa))
        return fail(c, OVL_EINVAL, "mu/kappa differ from those of the installed deflation");
    if (flags & (OVL_TWO_PASS | OVL_REPROJ | OVL_STEPWISE))
        return fail(c, OVL_EINVAL, "flags: two-pass, re-projection and stepwise are two-sided Lanczos options");
    return sign_solve(c, OVL_ARNOLDI, m * cycles, m, mu, kappa, b, out, flags | OVL_MIXED, info);
}

int ovl_profile_get(ovl_ctx* c, ovl_kstat* out, int max, int* count) {
    if (!c || !count || (max > 0 && !out)) return fail(c, OVL_EINVAL, "bad argument");
    int q = 0;
    for (int i = 0; i < KC_COUNT; ++i) {
        if (!c->prof_launches[i]) continue;
        if (q < max) {
            std::memset(&out[q], 0, sizeof(ovl_kstat));
            std::strncpy(out[q].name, kclass_name[i], sizeof(out[q].name) - 1);
            out[q].launches = c->prof_launches[i];
            out[q].kernels = c->prof_kernels[i];
            out[q].ms = c->prof_ms[i];
        }
        ++q;
    }
    *count = q;
    return OVL_OK;
}

int ovl_set_wait_limit(ovl_ctx* c, long long polls, int unreachable) {
    if (!c || polls < 0) return fail(c, OVL_EINVAL, "bad argument");
    c->wait_polls = polls;
    c->wait_unreachable = unreachable ? 1 : 0;
    drop_graph(c);  // a captured solve holds the old limits
    return OVL_OK;
}

int ovl_profile_reset(ovl_ctx* c) {
    if (!c) return OVL_EINVAL;
    for (int i = 0; i < KC_COUNT; ++i) c->prof_launches[i] = 0, c->prof_kernels[i] = 0, c->prof_ms[i] = 0.0;
    return OVL_OK;
}

}  // extern "C"
