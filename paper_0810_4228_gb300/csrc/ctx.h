// Private definition of the library context (shared by the translation units
// that implement the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/ovl.h"
#include "ovl_kernels.h"

namespace ovl_priv {

// kernel classes of the per-kernel profile (OVL_PROFILE)
enum KClass {
    KC_SETUP = 0, KC_DEFLATE, KC_PAIR, KC_LSTEP, KC_INNER, KC_REGEN, KC_COMBINE, KC_ADSLASH, KC_ADOT, KC_AAXPY,
    KC_ANORM, KC_CONVERT, KC_PASS1, KC_PASS2, KC_COUNT
};

struct ProfRec {
    int cls;
    int kernels;
    cudaEvent_t a, b;
};

struct GraphEntry {
    bool valid = false;
    int method = -1, k = -1, flags = 0, m = -1, rs = 0;
    double mu = 0, kappa = 0;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace ovl_priv

struct ovl_ctx {
    ovl::Geom g{};
    size_t n = 0;  // 12 V complex per vector
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;  // private stream the solve graph is captured on
    // one-sequence batch that runs mixed two-sided Lanczos solves on lattices too large for the
    // persistent passes (its regeneration is the double-float kernel), created on first use
    ovl_batch* self_batch = nullptr;
    int device = 0, num_sms = 0;
    std::string err;

    // gauge field in the device layout
    double2* U64 = nullptr;
    float4* U12 = nullptr;
    float2* U18 = nullptr;
    float4* Udf = nullptr;  // double-float links (regeneration pass of mixed solves)
    int* nbr = nullptr;     // [8][V] neighbour table of the regeneration kernel (ovl::launch_build_nbr)
    bool have_gauge = false;

    // deflation
    int m = 0;
    double dmu = 0, dkappa = 0;
    double2* R = nullptr;
    double2* L = nullptr;
    double2* lam = nullptr;
    float2* R32 = nullptr;  // FP32 copies for re-projection in the FP32 pass
    float2* L32 = nullptr;
    int mcap = 0;

    // solve workspace
    int kcap = 0;
    double2 *b64 = nullptr, *y64 = nullptr, *bR = nullptr, *bL = nullptr, *t64 = nullptr, *s64 = nullptr;
    double2* V64 = nullptr;  // kcap + 1 vectors
    double2* W64[3] = {nullptr, nullptr, nullptr};
    double2* R64[3] = {nullptr, nullptr, nullptr};  // FP64 regeneration (two-pass)
    float2* v32[3] = {nullptr, nullptr, nullptr};
    float2* w32[3] = {nullptr, nullptr, nullptr};
    float2 *t32 = nullptr, *s32 = nullptr;
    double2 *alpha = nullptr, *beta = nullptr, *gamma = nullptr, *vscale = nullptr, *cvec = nullptr;
    double2 *H = nullptr, *h1 = nullptr, *h2 = nullptr, *pq = nullptr;
    ovl::KState* ks = nullptr;
    double* partials = nullptr;
    size_t partials_bytes = 0;
    unsigned int* counter = nullptr;
    unsigned int* bar = nullptr;  // grid barrier of the persistent kernels
    double2* inner = nullptr;
    size_t inner_elems = 0;
    double2* stage_in = nullptr;   // canonical staging (host transfers, apply_Dw)
    double2* stage_out = nullptr;
    void* nat_a = nullptr;         // device-layout temporaries (apply_Dw)
    void* nat_b = nullptr;

    ovl_priv::GraphEntry graph;

    // bounded device waits of the persistent pass 1 (ovl_set_wait_limit; 0 = the default limit)
    long long wait_polls = 0;
    int wait_unreachable = 0;

    // restarted Arnoldi: the accumulated Hessenberg matrix ((krs + 1) x krs), its combination
    // coefficients and inner-sign workspace (the basis is V64's first m + 1 slots)
    int krs_cap = 0;
    double2* Hrs = nullptr;
    double2* cvrs = nullptr;
    double2* innrs = nullptr;
    size_t innrs_elems = 0;

    // gradient of the Krylov sign (grad_krylov.cu): basis checkpoints and adjoint vectors, and the
    // scratch of the small-problem adjoint
    void* gwork = nullptr;
    size_t gwork_bytes = 0;
    double2* tadj = nullptr;
    size_t tadj_elems = 0;

    // per-kernel profile (OVL_PROFILE)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ovl_priv::ProfRec> recs;
    int prof_launches[ovl_priv::KC_COUNT] = {};
    long long prof_kernels[ovl_priv::KC_COUNT] = {};
    double prof_ms[ovl_priv::KC_COUNT] = {};
};


namespace ovl_priv {
int fail(ovl_ctx* c, int code, const std::string& msg);
int ensure_base(ovl_ctx* c);
int ensure_solve(ovl_ctx* c, int k);
void drop_graph(ovl_ctx* c);
bool host_inverse(std::vector<std::complex<double>>& A, int m);
// queue one solve of the C ABI's sign_krylov (b already packed into c->b64)
int enqueue_solve(ovl_ctx* c, int method, int k, double mu, double kappa, int flags);
// queue one restarted Arnoldi solve: k / rs cycles of rs steps (b already packed into c->b64)
int enqueue_restarted(ovl_ctx* c, int rs, int cycles, double mu, double kappa, int flags);
int ensure_restart(ovl_ctx* c, int K);
// install m eigenpairs already in the device layout (R, L: m device vectors each, lam: host)
int install_deflation(ovl_ctx* c, double mu, double kappa, int m, const double* lambda, const double2* Rdev,
                      const double2* Ldev);
}  // namespace ovl_priv

#define OVL_CUDA_TRY(ctx, call)                                                                         \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return ovl_priv::fail(ctx, OVL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
