// noalloc.cu -- one proximal mean-field step on caller-owned buffers, with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc: code running under a memory pool or
// allocator that owns the whole device (a serving framework that reserved
// HBM up front), code inside a region where allocation is forbidden or would
// synchronise the device, and embedded integrations that must not touch the
// allocator after start-up.  For them this file offers a variant of the grid
// step whose only scratch memory -- the per-tile free-energy partials, the
// tile counter, the status word, the step size and the table of mu pairs --
// lives in a file-scope
// device array that the library holds from load time until the process exits,
// on every GPU that loads it.
//
// In host code the array's name is not a device address, so the address is
// fetched once per device with cudaGetSymbolAddress (with that device
// current) and cached; the first call on a device does this set-up, so make
// that first call before any stream capture.  Every call shares the array:
// calls that overlap on the GPU (different streams, different threads) race
// on it and must be serialised by the caller.
//
// A call is three kernel launches on the caller's stream and nothing else:
// a set-up kernel that receives the mu pair table and the step size by value
// (kernel parameters, so no host buffer has to outlive the call) and clears
// the counter and status word; the grid step; and a finishing kernel that
// turns F_out into NaN when the step reported an error or F is not finite.
#include <cmath>
#include <mutex>

#include "../../include/proxmf.h"
#include "nvtx_range.h"
#include "internal.h"

namespace {

// 512 KiB: 64480 FP64 tile partials, then the counter, status word and step
// (256 bytes), then the table of mu pairs (8 KiB).
constexpr size_t kScratchBytes = 512 * 1024;
constexpr size_t kPairBytes = 8 * 1024;
constexpr int kMaxTiles = (int)((kScratchBytes - kPairBytes) / sizeof(double)) - 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Everything the set-up kernel writes, carried in its parameters (8 KiB of
// pairs plus the step; kernel parameters may take up to 32 KiB).
struct NoallocSetup {
    float2 pairs[2 * proxmf::kMaxLabels * 16];
    int npairs;
    float eta;
};

__global__ void noalloc_setup_kernel(const __grid_constant__ NoallocSetup p, float2 *mu_dev, float *eta_dev,
                                     unsigned *counter, int *status) {
    for (int i = threadIdx.x; i < p.npairs; i += blockDim.x) mu_dev[i] = p.pairs[i];
    if (threadIdx.x == 0) {
        *eta_dev = p.eta;
        *counter = 0u;
        *status = 0;
    }
}

// The step records a non-finite F as status -6; the caller sees it as NaN.
__global__ void noalloc_finish_kernel(const int *status, double *F_out) {
    if (*status != 0 || !isfinite(*F_out)) *F_out = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace

extern "C" crf_status mf_grid_step_noalloc(int32_t topology, int32_t n_labels, int64_t height,
                                           int64_t width, const float *U, const float *w,
                                           const float *mu, const float *logq_in, float *logq_out,
                                           double eta, double *F_out, void *stream) {
    PROXMF_RANGE("mf_grid_step_noalloc");
    using namespace proxmf;
    if (topology != CRF_GRID4 && topology != CRF_GRID8) return CRF_E_INVALID;
    if (n_labels < 1 || n_labels > kMaxLabels || height < 1 || width < 1) return CRF_E_INVALID;
    if (!U || !w || !mu || !logq_in || !logq_out || !F_out) return CRF_E_INVALID;
    if (logq_in == logq_out) return CRF_E_INVALID;
    if (!(eta > 0.0) || eta > 1.0) return CRF_E_INVALID;
    if (height > 65535ll * GY || width > (1 << 24)) return CRF_E_INVALID;
    int nbx, nby;
    grid_tiles((int)height, (int)width, &nbx, &nby);
    if ((long long)nbx * nby > kMaxTiles) return CRF_E_INVALID;
    for (int i = 0; i < n_labels * n_labels; ++i)
        if (!std::isfinite(mu[i])) return CRF_E_INVALID;
    bool sym = true;
    for (int i = 0; i < n_labels; ++i)
        for (int k = i + 1; k < n_labels; ++k)
            if (mu[i * n_labels + k] != mu[k * n_labels + i]) sym = false;

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        (void)cudaGetLastError();
        return CRF_E_CUDA;
    }
    double *partial = (double *)base;
    unsigned *counter = (unsigned *)(partial + kMaxTiles);
    int *status = (int *)(counter + 1);
    float *eta_dev = (float *)(status + 1);
    float2 *mu_dev = (float2 *)((unsigned char *)base + kScratchBytes - kPairBytes);
    cudaStream_t st = (cudaStream_t)stream;

    // mu as the step kernel's column / row pairs (see mu_pair_slots), passed
    // by value to the set-up kernel, which writes them into the scratch array
    const int LT = kernel_labels(n_labels), NPP = mu_pair_slots(LT);
    NoallocSetup setup;
    static_assert(sizeof(setup.pairs) <= kPairBytes, "pair table fits its scratch slot");
    build_mu_pairs_host(mu, n_labels, LT, setup.pairs);
    setup.npairs = 2 * LT * NPP;
    setup.eta = (float)eta;
    const float2 *pairs = setup.pairs;
    noalloc_setup_kernel<<<1, 256, 0, st>>>(setup, mu_dev, eta_dev, counter, status);
    cudaError_t e = cudaGetLastError();
    GridStepLaunch a{};
    a.s_in = logq_in;
    a.s_out = logq_out;
    a.U = U;
    a.w = w;
    a.eta = eta_dev;
    a.mu_out = mu_dev;
    a.mu_in = mu_dev + (size_t)LT * NPP;
    a.mu_host = pairs;   // read while the step is launched (symmetric mu in its parameters)
    a.partial = partial;
    a.counter = counter;
    a.f_trace = F_out;   // never written: trace_cap = 0
    a.f_cur = F_out;
    a.done = nullptr;
    a.status = status;
    a.B = 1;
    a.L = n_labels;
    a.H = (int)height;
    a.W = (int)width;
    a.conn = topology == CRF_GRID8 ? 8 : 4;
    a.t = 0;
    a.trace_cap = 0;
    a.update = 1;
    a.rel_tol = 0.0;
    a.mu_sym = sym;
    if (e == cudaSuccess) e = launch_grid_step(a, st);
    if (e == cudaSuccess) {
        noalloc_finish_kernel<<<1, 1, 0, st>>>(status, F_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return CRF_E_CUDA;
    }
    return CRF_OK;
}
