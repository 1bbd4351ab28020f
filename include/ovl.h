/*
 * ovl.h -- C ABI of the GB300 library computing the overlap Dirac operator at
 * nonzero chemical potential,
 *
 *     D_ov(mu) b = b + gamma5 sgn(gamma5 D_w(mu)) b            (Sec. 1, Eq. 1.1)
 *
 * with the Arnoldi (Sec. 2, Eq. 2.6) and two-sided Lanczos (Sec. 4, Eq. 4.4)
 * Krylov approximations of sgn(A) b, A = gamma5 D_w(mu), and LR deflation of
 * the critical eigenvalues (Sec. 3, Eq. 3.4; Sec. 4, Eq. 4.5).
 *
 * Conventions (fixed by this library; the paper leaves them open):
 *   - lattice dims[4] = (L1, L2, L3, L4), L4 = Euclidean time; every extent
 *     >= 2 and L4 even (the device layout is even/odd ordered).
 *   - canonical site index s = ((x1*L2 + x2)*L3 + x3)*L4 + x4 (time fastest).
 *   - gauge field: complex128 U[V][4][3][3], U[s][nu] = link from x to x+nu.
 *   - spinor: complex128 psi[V][4][3] (spin, colour), gamma matrices in the
 *     chiral basis, gamma5 = diag(1, 1, -1, -1).
 *   - hops of Eq. 1.2: (T_nu^+ psi)(x) = (1 + gamma_nu) U_{x,nu} psi(x + nu),
 *     (T_nu^- psi)(x) = (1 - gamma_nu) U_{x-nu,nu}^dag psi(x - nu);
 *     e^{+mu} multiplies T_4^+, e^{-mu} multiplies T_4^-.
 *   - boundary: periodic in space, bc_t = -1 (antiperiodic) or +1 in time.
 *   - complex numbers are interleaved (re, im) pairs of double.
 *
 * Memory: unless OVL_HOST is given, every pointer argument that names a
 * field is a DEVICE pointer owned by the caller, which keeps it alive until
 * the work queued on the context's stream has finished.  The library owns
 * only its workspace (device memory it allocates with cudaMalloc on first
 * use and frees in ovl_destroy).  All work is queued on the stream given to
 * ovl_create; calls that return results to the host (info structs, status)
 * synchronise that stream.
 *
 * Errors: every function returns an ovl_status; OVL_OK is 0.  On failure
 * ovl_last_error(ctx) returns a message; outputs are then unspecified.
 * A context is not thread safe: one host thread at a time.
 */
#ifndef OVL_H
#define OVL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OVL_OK = 0,
    OVL_EINVAL = 1,      /* bad argument (sizes, flags, null pointer, mismatched mu/kappa) */
    OVL_ENOMEM = 2,      /* device allocation failed */
    OVL_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    OVL_EBREAKDOWN = 4,  /* serious breakdown of two-sided Lanczos: w_hat^dag v_hat = 0 */
    OVL_ESINGULAR = 5,   /* sgn undefined (eigenvalue on the imaginary axis) or singular matrix */
    OVL_ENOCONV = 6,     /* the inner sign iteration did not converge */
    OVL_ETIMEOUT = 7,    /* a bounded device-side wait gave up; the context stays usable */
    OVL_ESTATE = 8       /* call order: gauge field or deflation not set */
} ovl_status;

typedef struct ovl_ctx ovl_ctx;

/* Methods of sgn(A) b. */
#define OVL_ARNOLDI   0   /* Sec. 2, Eq. 2.6 (with deflation Eq. 3.4) */
#define OVL_LANCZOS2  1   /* Sec. 4, Eq. 4.4 (with deflation Eq. 4.5)  */

/* Flags (bit set). */
#define OVL_GAMMA5       0x0001  /* apply_Dw: y = gamma5 D_w(mu) x  (A x)                  */
#define OVL_DAGGER       0x0002  /* apply_Dw: y = A^dag x = gamma5 D_w(-mu) x              */
#define OVL_NATIVE       0x0004  /* x, y in the device layout (see ovl_vector_bytes)       */
#define OVL_HOST         0x0008  /* field pointers are host memory (canonical layout)      */
#define OVL_F32          0x0010  /* apply_Dw: FP32 stencil with 12-real links (NATIVE FP32 vectors) */
#define OVL_F32_FULL     0x0020  /* apply_Dw: FP32 stencil with 18-real links              */
#define OVL_OVERLAP      0x0100  /* sign_krylov: out = D_ov b = b + gamma5 sgn(A) b,
                                    otherwise out = sgn(A) b                               */
#define OVL_MIXED        0x0200  /* sign_krylov LANCZOS2: FP32 basis + 12-real links in pass 1, FP64
                                    coefficients, FP64 regeneration pass (two-pass, Sec. 5).
                                    ARNOLDI: the stored basis as double-float pairs (about 48
                                    significant bits, 16 bytes per complex element as in FP64) and
                                    both Gram-Schmidt sweeps in double-float arithmetic on the FP32
                                    pipe; FP64 stencil, H and inner sign.  Results agree with the
                                    FP64 Arnoldi run to about 1e-12                          */
#define OVL_TWO_PASS     0x0400  /* sign_krylov LANCZOS2: do not store the basis, regenerate it
                                    from alpha, beta, gamma in a second pass (Sec. 5)       */
#define OVL_INNER_NEWTON 0x1000  /* inner sgn(G_k) / sgn(H_k): Roberts/Newton (Sec. 2) instead of
                                    the resolvent quadrature (tridiagonal solves for 2sL,
                                    Givens-rotation Hessenberg solves for Arnoldi); without the
                                    flag Newton still runs if the quadrature does not converge */
#define OVL_REPROJ       0x8000  /* sign_krylov MIXED with deflation: project the deflated directions
                                    out of every FP32 pass-1 vector (v^ -= R L^dag v^, w^ -= L R^dag w^).
                                    Off by default: with FP32 copies of R, L the projected operator
                                    differs from A at the 1e-8 level, which then bounds the accuracy */
/* OVL_REPROJ applied every p-th step only (1 <= p <= 127): the pass-1 vectors of the steps i with
 * (i + 1) % p == 0 are projected; p = 1 is OVL_REPROJ.  p > 1 runs the stepwise kernels. */
#define OVL_REPROJ_PERIOD(p) (OVL_REPROJ | (((p) & 0x7f) << 24))
#define OVL_STEPWISE     0x40000 /* sign_krylov MIXED: one kernel per recurrence step instead of the
                                    persistent cooperative kernels (default on small lattices)   */
#define OVL_PASS2_F64    0x80000 /* MIXED: regeneration pass in native FP64                       */
#define OVL_NO_TUNE      0x200000 /* batch_solve: keep the current launch shapes, no autotuning     */
#define OVL_ARNOLDI_CGS2 0x400000 /* sign_krylov ARNOLDI with MIXED: classical Gram-Schmidt applied
                                     twice, four sweeps over the basis per step.  The default is the
                                     delayed form (the second Gram-Schmidt pass of step j fused with
                                     the first of step j + 1): two sweeps per step, the same Arnoldi
                                     process (Sec. 2, Eq. 2.2-2.3) in exact arithmetic             */
#define OVL_PASS2_DF     0x100000 /* MIXED: regeneration pass in double-float arithmetic (FP32 pairs,
                                    about 48 significant bits, on the FP32 pipe).  Default: double-
                                    float in batched solves and in single mixed 2sL solves on lattices
                                    above the persistent limit (run as a batch of one), FP64 in the
                                    other single solves (one source per tile is latency bound, where
                                    double-float's longer dependency chains cost more than the
                                    narrow FP64 pipe)                                              */
#define OVL_NO_GRAPH     0x2000  /* sign_krylov: launch kernels directly, no CUDA graph     */
#define OVL_STENCIL_SITE  0x10000 /* apply_Dw: force one thread per site (default: by volume)    */
#define OVL_STENCIL_SPLIT 0x20000 /* apply_Dw: force the direction-split layout (4 threads/site)   */
#define OVL_PROFILE      0x4000  /* sign_krylov: time every kernel class with CUDA events on the
                                    context's stream (implies OVL_NO_GRAPH); read the totals with
                                    ovl_profile_get                                        */

/* Information returned by ovl_sign_krylov. */
typedef struct {
    int    k_used;          /* Krylov steps taken (< k after a lucky breakdown)          */
    int    breakdown_step;  /* step of a serious breakdown, -1 if none                   */
    int    inner_iters;     /* Newton iterations, or quadrature nodes, of the inner sign */
    int    inner_method;    /* 0 = quadrature, 1 = Newton                                */
    double bperp_norm;      /* |b_perp^R| (|b| without deflation)                         */
    double inner_err;       /* a-posteriori estimate of the inner sign's relative error  */
} ovl_info;

/* --- context ---------------------------------------------------------------------------- */

/* Create a context for one lattice on the current CUDA device; stream is a
 * cudaStream_t (NULL = legacy default stream).  Fails with OVL_EINVAL if an
 * extent is < 2 or L4 is odd, or bc_t is not +-1. */
int ovl_create(ovl_ctx** ctx, const int dims[4], int bc_t, void* stream);
int ovl_destroy(ovl_ctx* ctx);
const char* ovl_last_error(const ovl_ctx* ctx);
/* Change the stream later work is queued on. */
int ovl_set_stream(ovl_ctx* ctx, void* stream);
/* Bytes of one vector in the device layout: prec 0 = FP64 (12V complex128),
 * 1 = FP32 (12V complex64).  The layout is site-major in even/odd order with
 * 16-byte components [component-chunk][site] (see the implementation). */
size_t ovl_vector_bytes(const ovl_ctx* ctx, int prec);

/* --- gauge field ------------------------------------------------------------------------- */

/* Install U (canonical complex128 [V][4][3][3], SU(3) links).  The library
 * keeps an FP64 copy and FP32 copies (12-real: rows 0,1; 18-real) in the
 * device layout.  flags: OVL_HOST if U is host memory. */
int ovl_set_gauge(ovl_ctx* ctx, const void* U, int flags);

/* --- the Wilson operator (Sec. 1, Eq. 1.2) ---------------------------------------------- */

/* y = D_w(mu) x, gamma5 D_w(mu) x (OVL_GAMMA5) or gamma5 D_w(-mu) x (OVL_DAGGER), with
 * kappa = 1/(8 + 2 m_w).  Canonical complex128 vectors by default; with OVL_NATIVE
 * x and y are device-layout vectors (FP64, or FP32 with OVL_F32 / OVL_F32_FULL).
 * x and y must not overlap. */
int ovl_apply_Dw(ovl_ctx* ctx, double mu, double kappa, const void* x, void* y, int flags);

/* Pair application of the two-sided Lanczos step (Sec. 4, Eq. 4.2): t = A v and s = A^dag w
 * in one pass over the links, plus alpha = w^dag t (FP64 accumulation) written to
 * *alpha_host (2 doubles) if non-NULL.  Device-layout vectors; prec 0 = FP64,
 * 1 = FP32 with 12-real links. */
int ovl_apply_pair(ovl_ctx* ctx, double mu, double kappa, int prec,
                   const void* v, const void* w, void* t, void* s, double* alpha_host);

/* The same pair application as ovl_apply_pair, for callers that must not allocate device
 * memory when they call it -- code capturing a CUDA graph (allocation is illegal there), or
 * a caller whose memory belongs to its own pool or arena.  It calls no cudaMalloc, cudaFree
 * or allocating library routine: the reduction's scratch is a static device array of the
 * library (768 KiB, resident on every GPU that loads the library).  The paper has no
 * counterpart; this is a calling convention of this library.
 *   - alpha_dev: DEVICE pointer to 2 doubles receiving alpha = w^dag t; nothing is copied
 *     to the host and the call does not synchronise (read alpha after the stream's work).
 *   - the context and its gauge field must exist already (they allocate when created).
 *   - lattices whose pair kernel needs more than 32768 thread blocks (more than 4194304
 *     sites; ovl_apply_pair_noalloc_blocks tells) are rejected with OVL_EINVAL before any
 *     launch.
 *   - the first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     no allocation); make that first call before any stream capture that includes it.
 *   - all calls share the array and it keeps the last call's contents; each call resets
 *     what must start at zero, but calls that overlap on the GPU (e.g. on two streams at
 *     once) race on it and give wrong results. */
int ovl_apply_pair_noalloc(ovl_ctx* ctx, double mu, double kappa, int prec,
                           const void* v, const void* w, void* t, void* s, double* alpha_dev);

/* Host-only size check for ovl_apply_pair_noalloc (no GPU call, no context): *blocks = the
 * number of thread blocks the pair kernel launches on a lattice of extents dims[4] (the same
 * function decides the launch), *max_blocks (may be NULL) = the most the static scratch holds
 * (32768).  Returns OVL_OK when the lattice fits, OVL_EINVAL when it does not or when dims is
 * not a valid lattice (an extent below 2 or an odd time extent; *blocks is then 0).  The paper
 * has no counterpart. */
int ovl_apply_pair_noalloc_blocks(const int dims[4], int* blocks, int* max_blocks);

/* Adjoint of y = A x, A = gamma5 D_w(mu; U) (Eq. 1.2), for a real function l(y), in PyTorch's
 * convention for complex gradients (g_z = dl/dRe z + i dl/dIm z, so dl = Re <g_z, dz>): given
 * g = g_y, writes
 *   grad_U[x][nu] = g_{U_{x,nu}}     (canonical complex128 [V][4][3][3], device; may be NULL)
 *   *grad_mu      = dl/dmu = Re <g, (dA/dmu) x>, dA/dmu = -kappa gamma5 (e^mu T_4^+ - e^-mu T_4^-)
 * (host double; may be NULL).  x, g: canonical complex128 device vectors.  grad_x = A^dag g is
 * ovl_apply_Dw with OVL_DAGGER.  Uses the installed gauge field U.  flags: 0 (FP64) or OVL_F32
 * (the link force in FP32 arithmetic, relative error about 1e-7; d/dmu stays FP64). */
int ovl_dw_grad(ovl_ctx* ctx, double mu, double kappa, const void* x, const void* g, void* grad_U,
                double* grad_mu, int flags);

/* ---- batched solves (one launch sequence for many right-hand sides and configurations) ----
 * A batch groups nctx contexts (each with its own lattice size, gauge field and installed
 * deflation set) and nrhs[j] right-hand sides for context j.  Every sequence (context, rhs)
 * runs the two-sided Lanczos solve of ovl_sign_krylov (Sec. 4, Eq. 4.2-4.5), but each batched
 * kernel covers all sequences in one launch, with per-sequence reductions, and the whole solve
 * is captured as one CUDA graph (re-captured when k, mu, kappa, the precision or a context's
 * deflation size change).
 * Precision: OVL_MIXED = FP32 pass 1 and a regeneration pass in double-float arithmetic (about
 * 48 significant bits; native FP64 with OVL_PASS2_F64) (Sec. 5); otherwise FP64, one
 * pass with the basis stored, or two passes with OVL_TWO_PASS or when the stored basis would
 * exceed 32 GiB.  The contexts must share one stream (the first's); the batch
 * owns its workspace (for n = 12 V summed over sequences: about 8 n FP32 + 7 n FP64 complex
 * values mixed, (k + 9) n FP64 otherwise). */
typedef struct ovl_batch ovl_batch;
int ovl_batch_create(ovl_batch** out, ovl_ctx* const* ctxs, int nctx, const int* nrhs);
int ovl_batch_destroy(ovl_batch* batch);
const char* ovl_batch_last_error(const ovl_batch* batch);
/* b[j], out[j]: nrhs[j] canonical complex128 vectors of context j, one after another (device,
 * or host with OVL_HOST).  flags: OVL_MIXED, OVL_TWO_PASS, OVL_PASS2_F64, OVL_STEPWISE (pass 1
 * one launch per step even when the batch fits one resident grid), OVL_NO_TUNE, OVL_OVERLAP,
 * OVL_HOST, OVL_NO_GRAPH, OVL_PROFILE.  info: one
 * entry per sequence in (context, rhs) order (may be NULL).  OVL_PROFILE: eager launches with
 * per-phase events (see ovl_batch_profile).  Returns the first failing
 * sequence's status (the others' results are still written). */
int ovl_batch_solve(ovl_batch* batch, int k, double mu, double kappa, const void* const* b, void* const* out,
                    int flags, ovl_info* info);
/* Totals of the solves run with OVL_PROFILE (eager launches, CUDA events around each phase):
 * ms3[0] pass 1 (the Krylov recurrence), ms3[1] the inner sign, ms3[2] the regeneration pass or the
 * combination; *nsolves the number of such solves.  reset != 0 clears the totals. */
int ovl_batch_profile(ovl_batch* batch, double* ms3, int* nsolves, int reset);
/* Launch shapes of the batched kernels.  The first solve in each precision times the candidates
 * (pass-1 site blocks of 64, 128 or 256 sites; the regeneration kernel at 3 to 6 blocks per SM
 * with one sequence per block, or at 2 to 4 blocks per SM with two sequences of one lattice per
 * block) with short eager solves of the batch itself and keeps the fastest (OVL_NO_TUNE skips
 * this).  The choice is cached per (GPU model, SM count, precision, lattice extents and
 * right-hand sides of every context): later batches of the same shape in the process take it
 * without timing, and when the environment variable OVL_TUNE_CACHE names a file the choices are
 * appended there ("key shape blocks_per_sm pair" lines) and read by later processes.  Writes the
 * chosen shapes (NULL pointers are skipped); returns OVL_ESTATE before the first tuning. */
int ovl_batch_tuning(const ovl_batch* batch, int* pass1_block_sites, int* regen_blocks_per_sm,
                     int* regen_seqs_per_block);
/* Pins the launch shapes (pass1_block_sites 64, 128 or 256; regen_blocks_per_sm 2 to 6;
 * regen_seqs_per_block 1 or 2) and turns the autotuner off for this batch.  OVL_EINVAL for any
 * other value (nothing changed). */
int ovl_batch_set_tuning(ovl_batch* batch, int pass1_block_sites, int regen_blocks_per_sm,
                         int regen_seqs_per_block);
/* create + solve + destroy (no graph reuse); errors are reported on ctxs[0]. */
int ovl_sign_krylov_batched(ovl_ctx* const* ctxs, int nctx, const int* nrhs, int k, double mu, double kappa,
                            const void* const* b, void* const* out, int flags, ovl_info* info);

/* Derivatives of l = Re <g, y>, y = sgn(A) b (Sec. 1, Eq. 1.3), A = gamma5 D_w(mu; U) (Eq. 1.2),
 * for the upstream gradient g = g_y in PyTorch's convention (dl = Re <g_z, dz> for every
 * complex z).  The derivative of the exact function: with the resolvent form of sgn,
 * dl/dtheta = -(1/pi) int e^u sum_+- Re <R_+-^dag g, (dA/dtheta) R_+- b> du, R_+- = (A +- i e^u)^-1,
 * and one k-step FP64 two-sided Lanczos process (Sec. 4, Eq. 4.2) started from v_1 = b / |b|,
 * w_1 = g / conj(g^dag v_1) approximates R b in K_k(A, b) and R^dag g in K_k(A^dag, g).
 * The installed deflation set is not used (its eigenvectors would depend on U and mu).
 * Writes, each may be NULL:
 *   y       sgn(A) b                           (canonical complex128 [V][12], device)
 *   grad_U  g_U                                (canonical complex128 [V][4][3][3], device)
 *   grad_mu dl/dmu                             (host double)
 *   grad_b  g_b = sgn(A)^dag g                 (canonical complex128 [V][12], device)
 * b, g: canonical complex128 device vectors.  The two Krylov bases (k + 1 vectors each) and
 * k more vectors stay in device memory for the call.  Errors as ovl_sign_krylov;
 * OVL_EBREAKDOWN also if g^dag b = 0 (the process cannot start); OVL_ENOCONV if the
 * quadrature of the k x k part does not settle.  flags: 0 = FP64 process (the N k^2 combination
 * Z = W conj(M) in double-float arithmetic, about 48 bits, on the FP32 pipe); OVL_MIXED = the
 * two-sided Lanczos process in FP32 with 12-real links (FP64 reductions, coefficients and the
 * k x k quadrature), the combination and the link force in FP32: relative error about 1e-6
 * against the FP64 path.  info: as ovl_sign_krylov (may be NULL).  Synchronises the context's
 * stream. */
int ovl_sign_grad(ovl_ctx* ctx, int k, double mu, double kappa, const void* b, const void* g, void* y,
                  void* grad_U, double* grad_mu, void* grad_b, int flags, ovl_info* info);

/* Convert a canonical complex128 vector (device) into the device layout (prec 0 or 1)
 * and back. */
int ovl_pack(ovl_ctx* ctx, const void* canon, void* native, int prec);
int ovl_unpack(ovl_ctx* ctx, const void* native, void* canon, int prec);

/* --- deflation (Sec. 3, Eq. 3.1; Sec. 5) ------------------------------------------------- */

/* Install m critical eigenpairs of A = gamma5 D_w(mu) for the given (mu, kappa):
 * lambda: host array of m complex (2m doubles); R, L: canonical complex128 [m][12V]
 * right and left eigenvectors (A r_j = lambda_j r_j, l_j^dag A = lambda_j l_j^dag).
 * The library makes them bi-orthonormal, L <- L (L^dag R)^-H, and returns OVL_ESINGULAR
 * if L^dag R is numerically singular.  m = 0 removes the deflation.  Later sign_krylov
 * calls must use the same mu and kappa (else OVL_EINVAL). */
int ovl_set_deflation(ovl_ctx* ctx, double mu, double kappa, int m, const double* lambda,
                      const void* R, const void* L, int flags);

/* Result of ovl_deflation_eigs. */
typedef struct {
    int       m;             /* eigenpairs installed                                     */
    int       iterations;    /* Arnoldi restart cycles (right + left side)                */
    long long matvecs;       /* applications of A or A^dag                                */
    double    max_residual;  /* max |A r_j - lambda_j r_j| of the installed right pairs  */
    double    lambda_cut;    /* largest |lambda| among the m + nextra computed pairs      */
} ovl_eiginfo;

/* Deflation phase on the GPU (Sec. 3 and Sec. 5, where ARPACK plays this role): compute the
 * m + nextra eigenvalues of A = gamma5 D_w(mu) nearest 0 with right and left eigenvectors
 * (thick-restart Arnoldi on a Chebyshev polynomial of A^2 that amplifies its smallest
 * eigenvalues, with a basis of nkrylov vectors, 0 = 10 (m + nextra) within
 * [3 (m + nextra) + 40, 512], at
 * most maxit restart cycles, then Rayleigh-Ritz with A and with A^dag; residual
 * |A r - lambda r| <= tol |A|), keep the m of smallest |Re lambda|, and install them as by
 * ovl_set_deflation.  Returns OVL_ENOCONV if the iteration did not converge (nothing
 * installed; info, if given, then holds m = 0 and the progress: cycles, matvecs, the last
 * residual check of the side that stopped).  Uses its own temporary device memory
 * (about 2 nkrylov + 2 (m + nextra) vectors). */
int ovl_deflation_eigs(ovl_ctx* ctx, double mu, double kappa, int m, int nextra, double tol, int nkrylov,
                       int maxit, ovl_eiginfo* info);

/* Copy the installed (bi-orthonormalised) deflation out: *m_out = m; lambda (host, 2m
 * doubles), R and L canonical complex128 [m][12V] (device, or host with OVL_HOST).  NULL
 * output pointers are skipped (pass R = L = lambda = NULL to query m). */
int ovl_get_deflation(ovl_ctx* ctx, int* m_out, double* lambda, void* R, void* L, int flags);

/* --- sgn(A) b and D_ov(mu) b ------------------------------------------------------------- */

/* out = sgn(A) b (or D_ov(mu) b with OVL_OVERLAP), A = gamma5 D_w(mu), by the method
 * (OVL_ARNOLDI / OVL_LANCZOS2) with Krylov size k >= 1 and the installed deflation.
 * b, out: canonical complex128 (device, or host with OVL_HOST), may not overlap.
 * info may be NULL.  OVL_EINVAL for OVL_TWO_PASS with OVL_ARNOLDI (the Arnoldi basis is always
 * stored: k + 1 vectors of 16 bytes per complex element, FP64 or double-float with OVL_MIXED).
 * Returns OVL_EBREAKDOWN on a serious 2sL breakdown (out holds the
 * approximation from the steps before it), OVL_ESINGULAR if the projected matrix has an
 * eigenvalue on the imaginary axis, OVL_ENOCONV if the inner sign did not converge.
 * OVL_LANCZOS2 with OVL_MIXED (and no flags but OVL_OVERLAP, OVL_HOST) on a lattice whose tiles do
 * not fit the persistent passes (more than 8 tiles of 32 sites per SM) runs as a batch of one
 * (ovl_batch_solve: double-float regeneration, autotuned launch shapes); the context keeps that
 * batch and its graph until its gauge field, deflation set, stream or buffers change. */
int ovl_sign_krylov(ovl_ctx* ctx, int method, int k, double mu, double kappa,
                    const void* b, void* out, int flags, ovl_info* info);

/* --- eigenvalues of the overlap operator ------------------------------------------------------ */
typedef struct {
    int       nconv;          /* eigenpairs returned (nev on success)                        */
    int       restarts;       /* Arnoldi cycles                                              */
    long long sign_solves;    /* applications of D_ov (each one sign solve of k steps)       */
    double    ritz_residual;  /* largest |h| |e^T z| of the returned Ritz pairs              */
    double    max_residual;   /* largest |D_ov x - lambda x| of the unit eigenvectors        */
} ovl_ovinfo;

/* The nev eigenvalues of D_ov(mu) = 1 + gamma5 sgn(gamma5 D_w(mu)) (Eq. 1.1) nearest 0, the
 * application Sec. 5 names as the next use of the sign function (the paper gives no method for
 * it): thick-restart Arnoldi with a basis of nkrylov vectors (0 = automatic, max(2 nev + 20, 40))
 * in which every application of D_ov is one ovl_sign_krylov solve by `method` (OVL_ARNOLDI or
 * OVL_LANCZOS2) with Krylov size k, the installed deflation and `flags` (OVL_MIXED, OVL_TWO_PASS,
 * OVL_INNER_NEWTON, OVL_ARNOLDI_CGS2; OVL_OVERLAP is implied; OVL_HOST and OVL_PROFILE are
 * rejected).  The eigenvalues are accurate to about the sign solves' relative error.
 *   - converged when every returned Ritz pair has |h| |e^T z| <= tol (|D_ov| <= 2 at mu = 0);
 *   - lambda: HOST array of 2 nev doubles (re, im), sorted by modulus, nearest 0 first;
 *   - vecs: DEVICE array of nev canonical complex128 unit eigenvectors (12V each), or NULL;
 *   - at most maxit restart cycles, else OVL_ENOCONV (info tells how far it got);
 *   - a failing sign solve ends the run with its status (OVL_EBREAKDOWN included);
 *   - allocates its own workspace ((2 nkrylov + 2) vectors) and frees it before returning. */
int ovl_overlap_eigs(ovl_ctx* ctx, int method, int k, double mu, double kappa, int flags, int nev,
                     int nkrylov, double tol, int maxit, double* lambda, void* vecs, ovl_ovinfo* info);

/* out = sgn(A) b (or D_ov b with OVL_OVERLAP) by the Arnoldi approximation restarted every m steps,
 * at most `cycles` cycles: the basis holds m + 1 vectors instead of k + 1 (Sec. 5 names the N k^2
 * cost of Arnoldi's basis; the paper gives no restart).  Cycle c continues from the last basis
 * vector of cycle c - 1; its Hessenberg block joins the accumulated matrix H (block lower
 * bidiagonal, upper Hessenberg, m cycles x m columns at most), and y gains |b_perp| V_c times the
 * rows of cycle c of sgn(H) e_1 (the restart of Eiermann and Ernst, SIAM J. Numer. Anal. 44, 2006),
 * with the installed LR deflation (Sec. 3, Eq. 3.4).  The basis and its Gram-Schmidt sweeps are
 * double-float (as with OVL_MIXED for OVL_ARNOLDI, delayed CGS2 within a cycle), the inner sign
 * the resolvent quadrature of H (Roberts' iteration with OVL_INNER_NEWTON or as the fallback).
 * A lucky breakdown ends the process after that cycle.  info->k_used = columns of H used.
 * flags: OVL_OVERLAP, OVL_HOST, OVL_NO_GRAPH, OVL_PROFILE, OVL_INNER_NEWTON; OVL_EINVAL for
 * m < 1, cycles < 1, m x cycles > 8192 or the two-sided Lanczos options. */
int ovl_sign_arnoldi_restarted(ovl_ctx* ctx, int m, int cycles, double mu, double kappa,
                               const void* b, void* out, int flags, ovl_info* info);

/* Limits of the bounded device waits of the persistent FP32 pass 1 (the grid barriers of
 * OVL_MIXED two-sided Lanczos solves on lattices that fit the GPU): a wait gives up after
 * `polls` polls (0 restores the default, 2e7), sets the solve's timeout flag and every block
 * leaves, so the call returns OVL_ETIMEOUT and the context stays usable.  unreachable != 0 adds
 * one arrival to every barrier's target, so every wait runs out: a test of the timeout path
 * without a fault (use a small `polls`).  Drops the captured solve graph.  The paper has no
 * counterpart. */
int ovl_set_wait_limit(ovl_ctx* ctx, long long polls, int unreachable);

/* --- per-kernel profile -------------------------------------------------------------------- */

/* One kernel class of a profiled solve: its name, how many times it was queued, how many
 * kernels those launches contain and their total device time (CUDA events). */
typedef struct {
    char      name[24];
    int       launches;
    long long kernels;
    double    ms;
} ovl_kstat;

/* Accumulated per-class totals of every OVL_PROFILE solve since the last reset.  Writes at
 * most max entries to out and the number of classes with data to *count. */
int ovl_profile_get(ovl_ctx* ctx, ovl_kstat* out, int max, int* count);
int ovl_profile_reset(ovl_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* OVL_H */
