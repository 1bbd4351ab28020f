// An entry point that allocates no device memory: the pair application
// t = A v, s = A^dag w with alpha = w^dag t of ovl_apply_pair, whose grid
// reduction scratch (per-block partial sums, the block counter and the small
// solve-state record the kernel reads and writes) lives in a file-scope
// static __device__ array instead of the context's cudaMalloc'ed workspace.
//
// Who needs it: code that must not call cudaMalloc at the point where it runs
// -- for example a caller in the middle of capturing a CUDA graph (allocation
// calls are illegal there), a caller whose memory is owned by a pool or
// arena that forbids allocations outside its own, or a real-time loop that
// must not block on the driver.  Such a caller creates the context and
// installs the gauge field beforehand; this call then only launches kernels.
//
// Limits and sharing: the static array holds the partial sums of at most
// 32768 thread blocks (768 KiB in total, resident on every
// GPU that loads the library until the process exits).  The block count is
// the pair kernel's own grid (dslash_pair_blocks, the function its launcher
// uses): one block per 64 sites of each parity on large lattices, so at most
// 4194304 sites.  Every call shares
// the array and it keeps the last call's contents; the counter and state
// record are cleared at the start of each call, so calls must not overlap on
// the GPU (two concurrent calls on different streams race on the array).
#include <cuda_runtime.h>

#include <mutex>

#include "ctx.h"

using namespace ovl_priv;

namespace {

constexpr int kMaxBlocks = 32768;                     // partial sums of at most this many blocks
constexpr size_t kStateBytes = 256;                   // ovl::KState
constexpr size_t kCounterBytes = 256;                 // block counter (padded)
constexpr size_t kPartialDoubles = 3 * (size_t)kMaxBlocks;
constexpr size_t kScratchDoubles = (kStateBytes + kCounterBytes) / sizeof(double) + kPartialDoubles;

static_assert(sizeof(ovl::KState) <= kStateBytes, "state record does not fit its slot");

// The scratch itself: state record | counter | partial sums.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of the array, one per device (taken once, with that device current).
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return OVL_EINVAL;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return OVL_ECUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return OVL_OK;
}

// clear the counter and put the state record in its initial state (unit scales)
__global__ void k_noalloc_reset(double* scratch) {
    ovl::KState* ks = reinterpret_cast<ovl::KState*>(scratch);
    unsigned int* counter = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(scratch) + kStateBytes);
    ovl::KState z = {};
    z.bdstep = -1;
    z.sv = z.sw = z.svp = z.swp = make_double2(1.0, 0.0);
    *ks = z;
    *counter = 0u;
}

}  // namespace

extern "C" int ovl_apply_pair_noalloc_blocks(const int dims[4], int* blocks, int* max_blocks) {
    if (max_blocks) *max_blocks = kMaxBlocks;
    if (!dims || !blocks) return OVL_EINVAL;
    *blocks = 0;
    long long V = 1;
    for (int d = 0; d < 4; ++d) {
        if (dims[d] < 2) return OVL_EINVAL;
        V *= dims[d];
    }
    if (dims[3] % 2 || V > (1ll << 28)) return OVL_EINVAL;
    ovl::Geom g = {};
    for (int d = 0; d < 4; ++d) g.L[d] = dims[d];
    g.L4h = dims[3] / 2;
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.bc_t = -1;
    *blocks = ovl::dslash_pair_blocks(g);
    return *blocks <= kMaxBlocks ? OVL_OK : OVL_EINVAL;
}

extern "C" int ovl_apply_pair_noalloc(ovl_ctx* c, double mu, double kappa, int prec, const void* v, const void* w,
                                      void* t, void* s, double* alpha_dev) {
    if (!c || prec < 0 || prec > 1) return fail(c, OVL_EINVAL, "bad argument");
    // the grid the pair launcher will use: one partial-sum slot per block
    const int blocks = ovl::dslash_pair_blocks(c->g);
    if (blocks > kMaxBlocks)
        return fail(c, OVL_EINVAL,
                    "lattice too large for ovl_apply_pair_noalloc: at most 4194304 sites (its static scratch "
                    "holds the partial sums of 32768 thread blocks, one per 64 sites of each parity)");
    if (!v || !w || !t || !s || !alpha_dev) return fail(c, OVL_EINVAL, "null argument");
    if (!c->have_gauge) return fail(c, OVL_ESTATE, "gauge field not set");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(c, OVL_ECUDA, "cudaGetDevice failed");
    double* scratch = nullptr;
    if (scratch_address(dev, &scratch) != OVL_OK)
        return fail(c, OVL_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
    ovl::KState* ks = reinterpret_cast<ovl::KState*>(scratch);
    unsigned int* counter = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(scratch) + kStateBytes);
    double* partials = scratch + (kStateBytes + kCounterBytes) / sizeof(double);
    k_noalloc_reset<<<1, 1, 0, c->st>>>(scratch);
    ovl::launch_dslash_pair(prec == 0 ? (const void*)c->U64 : (const void*)c->U12, prec, v, w, t, s, mu, kappa, ks,
                            reinterpret_cast<double2*>(alpha_dev), 0, 1 << 30, partials, counter, c->g, c->st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, OVL_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return OVL_OK;
}
