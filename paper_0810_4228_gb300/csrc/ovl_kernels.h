// Host-side launchers of the library's kernels (internal C++ interface between
// the translation units; the public C ABI is include/ovl.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ovl_common.cuh"

namespace ovl {

// Device-side scalar state of one Krylov solve.  Coefficients follow the
// paper's notation (Sec. 4, Eq. 4.1-4.2): alpha on the diagonal of G_k, beta
// below, gamma above.  Basis vectors are stored unnormalised (v~_i = v_i /
// vscale[i]); consumers multiply by the recorded scales.
struct KState {
    int status;        // 0 = running/ok, else an ovl_status code
    int done;          // 1 after a lucky breakdown or the last step
    int kused;         // Krylov steps completed (size of G_k / H_k)
    int bdstep;        // serious-breakdown step, -1 if none
    int timeout;       // a bounded wait gave up
    int inner_iters;
    int inner_method;
    int inner_done;    // the inner sign has converged (quadrature or Newton)
    double anorm;      // running max |A v_i|, breakdown tolerance scale
    double nR;         // |b_perp^R|
    double inner_err;
    double pad2;
    double2 sv, sw;    // scale of the current v~, w~ (v = sv v~, w = sw w~)
    double2 svp, swp;  // scale of the previous v~, w~
    double2 red[8];    // scratch results of the last grid reduction
};

struct Workspace;   // defined in api.cu

// ---- stencil.cu
// Udf: the double-float copy of the links (float4 {re.hi, re.lo, im.hi, im.lo} in the FP64 layout)
void launch_pack_gauge(const double2* U_canon, double2* U64, float4* U12, float2* U18, float4* Udf, const Geom& g,
                       cudaStream_t st);
// in place: FP64 vectors (double2) -> double-float (float4 {hi, lo, hi, lo}), n complex each; and back
void launch_f64_to_df(void* x, size_t n, cudaStream_t st);
void launch_df_to_f64(void* x, size_t n, cudaStream_t st);
void launch_pack_spinor(const double2* canon, void* native, int prec, const Geom& g, cudaStream_t st);
// out_canon = b_canon (if given) + (g5 ? gamma5 : 1) * native
void launch_unpack_spinor(const void* native, int prec, double2* canon, const double2* b_canon, int g5,
                          const Geom& g, cudaStream_t st);
// y = [gamma5] D_w(mu) x  (single application), prec 0 = FP64, 1 = FP32-12, 2 = FP32-18;
// skipped when ks is given and the solve is finished.
void launch_dslash(const void* U, int prec, const void* x, void* y, double mu, double kappa, int gamma5,
                   const Geom& g, cudaStream_t st, const KState* ks = nullptr);
// pair: t = sv * A v~, s = sw * A^dag w~, alpha[step] = w^dag t (fused grid reduction),
// kused = step + 1, done after step klast.
void launch_dslash_pair(const void* U, int prec, const void* v, const void* w, void* t, void* s,
                        double mu, double kappa, KState* ks, double2* alpha, int step, int klast,
                        double* partials, unsigned int* counter, const Geom& g, cudaStream_t st);
// FP64 regeneration step of the two-pass 2sL (Sec. 5): v_{i+1} = ((A - alpha_i) v_i - gamma_{i-1} v_{i-1})
// / beta_i and y += c_{i+1} v_{i+1}, no reductions.
void launch_dslash_regen(const double2* U, const double2* vi, const double2* vim1, double2* vip1, double2* y,
                         double mu, double kappa, const KState* ks, const double2* alpha, const double2* beta,
                         const double2* gamma, const double2* c, int step, const Geom& g, cudaStream_t st);
int dslash_grid(const Geom& g, int threads);
// thread blocks launch_dslash_pair launches on g (= the partial-sum slots its reduction writes)
int dslash_pair_blocks(const Geom& g);
// nvec FP64 device-layout vectors to the FP32 device layout (component pairs in float4)
void launch_native_f64_to_f32(const double2* x, void* y, const Geom& g, int nvec, cudaStream_t st);
void launch_native_f32_to_f64(const void* x, double2* y, const Geom& g, int nvec, cudaStream_t st);
// nbr[h][i]: internal index of the hop-h neighbour of site i (h < 4 forward, else backward in nu = h & 3),
// bit-inverted where the hop takes the antiperiodic phase -1
void launch_build_nbr(int* nbr, const Geom& g, cudaStream_t st);
// stencil thread layout: -1 automatic (by volume), 0 one thread per site, 1 direction split
void set_dslash_variant(int mode);

// ---- krylov.cu
void launch_state_init(KState* ks, cudaStream_t st);
// 2sL recurrence of Sec. 4, Eq. 4.2 with fused reductions (w^^dag v^, |v^|^2, |w^|^2);
// the last block sets beta[step], gamma[step], the scales and vscale[step+1].
// With m > 0, v^ -= R p and w^ -= L q (p = pq[0..m), q = pq[m..2m)) in the same pass (re-projection of
// the deflated directions); R, L in the vectors' precision, m <= 64.
void launch_lanczos_step(int prec, const void* t, const void* s, const void* vi, const void* wi,
                         const void* vim1, const void* wim1, void* vnext, void* wnext, KState* ks,
                         const double2* alpha, double2* beta, double2* gamma, double2* vscale, int step, int kmax,
                         double* partials, unsigned int* counter, size_t n, cudaStream_t st,
                         const void* Rp = nullptr, const void* Lp = nullptr, const double2* pq = nullptr, int m = 0);
// h[l] = V_l^dag x for FP32 V and x (FP32 products, FP64 reduction)
void launch_multidot_f32(const float2* V, size_t ld, int nvec, const float2* x, double2* h, double* partials,
                         size_t n, cudaStream_t st, const KState* ks = nullptr);
// h[l] (+)= V_l^dag x for l < nvec (V_l = V + l*ld), deterministic two-stage reduction.
int multidot_blocks(size_t n);
void launch_multidot(const double2* V, size_t ld, int nvec, const double2* x, double2* h, int acc,
                     double* partials, size_t n, cudaStream_t st, const KState* ks = nullptr, int step = -1);
// x -= sum_l h[l] V_l
void launch_multiaxpy(const double2* V, size_t ld, int nvec, const double2* h, double2* x, double* partials,
                      unsigned int* counter, KState* ks, int norm_out, size_t n, cudaStream_t st, int step = -1);
// second Gram-Schmidt update of Arnoldi step j, then H[0..j, j] = h1 + h2, H[j+1, j] = |x|,
// kused = j + 1, done on a lucky breakdown or at j = jlast.
void launch_arnoldi_orth2(const double2* V, size_t ld, int nvec, const double2* h2, double2* x, double2* H, int ldH,
                          const double2* h1, int j, int jlast, double* partials, unsigned int* counter, KState* ks,
                          size_t n, cudaStream_t st);
void launch_arnoldi_normalize(double2* t, const KState* ks, size_t n, cudaStream_t st);
// Deflation split (Sec. 3, Eq. 3.2-3.4; Sec. 4, Eq. 4.5): bR = b - R p, bL = b - L q (bL may be null),
// y = R (sgn(lambda) p), with p = pq[0..m), q = pq[m..2m); sets nR = |bR|, sv = 1/nR, sw = 1/conj(bL^dag v_1).
void launch_deflate_split(const double2* b, const double2* R, const double2* L, const double2* lam, int m,
                          const double2* pq, double2* bR, double2* bL, double2* y, KState* ks, double2* vscale,
                          double* partials, unsigned int* counter, size_t n, cudaStream_t st);
// v = sv * x; if y: y += c[0] * v
void launch_scale_start(const double2* x, double2* v, double2* y, const double2* c, const KState* ks, size_t n,
                        cudaStream_t st);
// y += sum_{l < kused} c_l vscale_l V_l
void launch_combine(const double2* V, size_t ld, const double2* vscale, const double2* c, const KState* ks,
                    int kmax, double2* y, size_t n, cudaStream_t st);

// ---- arnoldi_df.cu: Arnoldi with the basis as double-float pairs (float4 {re.hi, re.lo, im.hi, im.lo}
// per complex element, n per vector, ld = n) and the Gram-Schmidt sweeps in double-float arithmetic
void launch_adf_todf(const double2* x, float4* xdf, const KState* ks, size_t n, cudaStream_t st);
// V_0 = x / nR (double-float) and its FP64 value into x64
void launch_adf_start(const double2* x, float4* v, double2* x64, const KState* ks, size_t n, cudaStream_t st);
int adf_dot_blocks(size_t n);
// h[l] = V_l^dag x for l < nvec (FP64 and double-float copies); partials: nvec * adf_dot_blocks(n) double2
void launch_adf_dot(const float4* V, size_t ld, int nvec, const float4* x, double2* h, float4* hdf,
                    double* partials, size_t n, int num_sms, const KState* ks, cudaStream_t st);
// x -= sum_{l < nvec} h[l] V_l
void launch_adf_update(const float4* V, size_t ld, int nvec, const float4* hdf, float4* x, size_t n, KState* ks,
                       double* partials, unsigned int* counter, cudaStream_t st);
// second update of Arnoldi step j, then H[0..j, j] = h1 + h2, H[j+1, j] = |x|, kused = j + 1, done on a
// lucky breakdown or at j = jlast
void launch_adf_update_fin(const float4* V, size_t ld, int nvec, const float4* hdf, float4* x, double2* H, int ldH,
                           const double2* h1, const double2* h2, int j, int jlast, double* partials,
                           unsigned int* counter, KState* ks, size_t n, cudaStream_t st);
// t <- t / |t| (|t| from the last update) and its FP64 value into x64
void launch_adf_normalize(float4* t, double2* x64, const KState* ks, size_t n, cudaStream_t st);
// y += sum_{l < kused} c_l V_l; cdf: kmax float4 scratch
// delayed CGS2 (low-synch Arnoldi, csrc/arnoldi_df.cu): h1[l] = V_l^dag x1, h2[l] = V_l^dag x2 for l < nvec in
// one sweep (x1 double-float, x2 FP64); the step's scalar work; the fused update of v_j and u_{j+1}
void launch_adf_dot2(const float4* V, size_t ld, int nvec, const float4* x1, const double2* x2, double2* h1,
                     double2* h2, double* partials, size_t n, int num_sms, const KState* ks, cudaStream_t st);
void launch_adf_dcgs(double2* H, int ldH, const double2* h1, const double2* h2, float4* cdf, float4* qdf, KState* ks,
                     int j, int fin, cudaStream_t st);
void launch_adf_update2(const float4* V, size_t ld, int j, const float4* cdf, const float4* qdf, float4* uj,
                        float4* unext, const double2* w, double2* x64, double2* H, int ldH, const double2* h1,
                        const double2* h2, size_t n, KState* ks, cudaStream_t st);
// restarted Arnoldi (csrc/arnoldi_df.cu): cycle bookkeeping, the cycle's combination y += V c[off ..] and the next
// cycle's start vector
void launch_rs_begin(KState* ks, int cyc, cudaStream_t st);
void launch_rs_mid(KState* ks, cudaStream_t st);
void launch_rs_combine(const float4* V, size_t ld, const double2* c, int off, float4* cdf, const KState* ks, int m,
                       double2* y, size_t n, cudaStream_t st);
void launch_rs_restart(float4* V, size_t ld, int m, const float4* cdf, double2* x64, KState* ks, size_t n, int last,
                       cudaStream_t st);
void launch_adf_combine(const float4* V, size_t ld, const double2* c, float4* cdf, const KState* ks, int kmax,
                        double2* y, size_t n, cudaStream_t st);

// ---- persistent.cu
bool persistent_ok(const Geom& g, int num_sms);
int launch_pass1_persistent(const float4* U12, float4* const v[3], float4* const w[3], KState* ks, double2* alpha,
                            double2* beta, double2* gamma, const float2* R32, const float2* L32, int m, double mu,
                            double kappa, int k, double* partials, unsigned int* bar, const Geom& g, int num_sms,
                            cudaStream_t st, long long spin = 0, int unreachable = 0);
// coef_work: 4 (kmax + 1) double2 of scratch for the per-step regeneration coefficients.
// Udf non-null: double-float arithmetic (links Udf; v[] are converted to double-float in place, so
// v[0] must hold the FP64 start vector and all three are left in double-float); else FP64 (links U64).
int launch_pass2_persistent(const double2* U64, const float4* Udf, double2* const v[3], double2* y, const KState* ks,
                            const double2* alpha, const double2* beta, const double2* gamma, const double2* c,
                            double2* coef_work, int kmax, double mu, double kappa, unsigned int* bar, int* err,
                            const Geom& g, int num_sms, cudaStream_t st);

// ---- inner_sign.cu
// c[0..n) = nR * sgn(H) e_1 for the upper Hessenberg H (column-major, leading dimension ldH) of
// size ks->kused, by the same quadrature with Givens-rotation solves of the shifted Hessenberg
// systems; needs inner_work_elems(kmax, 2) elements of work and kmax * 16 bytes of shared memory
// per node (-1: too small / too large, nothing launched).
int launch_inner_quadrature_hess(const double2* H, int ldH, KState* ks, double2* c, double2* work,
                                 size_t work_elems, int kmax, double* partials, unsigned int* counter,
                                 cudaStream_t st);
// c[0..n) = nR * sgn(G) e_1 for the tridiagonal G (alpha, beta, gamma) of size ks->kused, by the
// resolvent quadrature sgn(G) = (2/pi) int_0^inf G (G^2 + t^2)^-1 dt (see inner_sign.cu).
int launch_inner_quadrature(const double2* alpha, const double2* beta, const double2* gamma, KState* ks,
                            double2* c, double2* work, size_t work_elems, int kmax, double* partials,
                            unsigned int* counter, cudaStream_t st);
// the same for nseq independent problems at once; sequence j's alpha, beta, gamma, c start at
// j coef_stride, its state at ks + j, its scratch at j work_stride (>= inner_work_elems(kmax, 0)),
// its reduction buffers at j part_stride and counters + j.
int launch_inner_quadrature_batched(int nseq, const double2* alpha, const double2* beta, const double2* gamma,
                                    KState* ks, double2* c, size_t coef_stride, double2* work, size_t work_stride,
                                    int kmax, double* partials, size_t part_stride, unsigned int* counters,
                                    cudaStream_t st);
// c = nR * sgn(M) e_1 by Roberts' iteration (Sec. 2) with determinant scaling, M dense n x n
// (n = ks->kused) built from the tridiagonal (tri = 1) or taken as the Hessenberg H (ld = ldH).
// fallback = 1: run only if the quadrature before it did not converge (status 6 is then cleared).
int launch_inner_newton(const double2* alpha, const double2* beta, const double2* gamma, const double2* H,
                        int ldH, int tri, KState* ks, double2* c, double2* work, size_t work_elems, int kmax,
                        int num_sms, cudaStream_t st, int fallback = 0);
size_t inner_work_elems(int kmax, int method);

}  // namespace ovl
