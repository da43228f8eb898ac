// api.cu -- the C ABI (include/proxmf.h): handle, device storage, call order,
// status mapping.  Host code here only sequences device work; every step of
// the method runs in the kernels of grid_step*.cu, layout.cu and lanczos.cu.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/proxmf.h"
#include "nvtx_range.h"
#include "internal.h"

using namespace proxmf;

struct crf_s {
    crf_desc d{};
    int B = 0, L = 0, H = 0, W = 0, nd = 0, conn = 4;
    int LP = 0;                  // labels stored per pixel (padded)
    int LT = 0;                  // label count of the step kernel
    int nblk = 0;
    cudaStream_t st = nullptr;
    float *U = nullptr;          // [B][N][LP] unaries, padding 0
    float *s[2] = {nullptr, nullptr};  // [B][N][LP] log q, ping-pong, padding kPadLogQ
    float *w = nullptr;          // [B][N][nd] edge weights
    float2 *mu_pairs = nullptr;  // device [2][LT][NPP] mu column / row pairs
    std::vector<float2> mu_pairs_host;   // host copy of the same
    uint8_t *mu_tc = nullptr;    // device BF16 operand images of mu, mu^T (grid, BF16 form)
    __nv_bfloat16 *U16 = nullptr;  // [B][N][u16_pitch(LP)] unaries in BF16 (grid, BF16 form)
    // general graph (edge list)
    bool sparse = false;
    int *sp_out_ptr = nullptr, *sp_out_col = nullptr, *sp_in_ptr = nullptr, *sp_in_col = nullptr;
    float *sp_out_w = nullptr, *sp_in_w = nullptr;
    double *sp_nu = nullptr;     // [2] extreme eigenvalues of C mu C
    // fully connected model
    bool dense = false;
    int N = 0;                   // variables per instance
    float *K32 = nullptr;        // [B][N][N]
    __nv_bfloat16 *K16 = nullptr;  // [B][tiles][chunks][128 x 64] swizzled blocks (tensor-core form)
    float *q32[2] = {nullptr, nullptr};            // [B][N][LP] + padding
    __nv_bfloat16 *qt16[2] = {nullptr, nullptr};   // [B][32][N]
    float *feats = nullptr;      // [B][N][5]
    float *featsT = nullptr;     // BF16 dense handles: prescaled features per chunk (on-the-fly K)
    bool dense_fly = false;      // tensor-core steps compute K in the kernel (mf_dense_on_the_fly)
    float *mu_dev = nullptr;     // [L][L]
    double theta[2] = {0.0, 0.0};
    bool bf16 = false;           // tensor-core form
    DenseTcBuffers tcb{nullptr, nullptr};
    float *eta_fixed = nullptr;  // [B]
    float *adapt_d = nullptr;    // [B] d of the adaptive binary step (or d0 of Adam)
    bool adapt_active = false;   // set while mf_iterate runs the adaptive rule
    float *mom = nullptr, *vv = nullptr;   // [B][N][LP] momentum / Adam state (allocated on first use)
    int rule_kernel = 0;         // 1 momentum, 2 Adam, 3 ADHOC while mf_iterate runs them
    float gamma1 = 0.f, gamma2 = 0.f, eps = 0.f;
    float *eta_auto = nullptr;   // [B]
    double *Lambda = nullptr;    // [B]
    double *partial = nullptr;   // [2][B][nblk][kMaxFParts] free-energy partials (two slots: deferred sums)
    unsigned *counter = nullptr; // [B]
    double *ftrace = nullptr;    // [B][trace_cap]
    double *fcur = nullptr;      // [B]
    int *done = nullptr;         // [B]
    int *status = nullptr;       // device error word
    float *staging = nullptr;    // [B][N][L] row-layout staging
    int trace_cap = 0;
    int last_iters = 0;
    int cur = 0;
    std::vector<float> mu;
    bool mu_sym = true;
    bool use_resident = true;    // small grids: one launch per mf_iterate (grid_resident.cu)
    bool has_unary = false, has_pairwise = false, lambda_valid = false, broken = false;
    int lanczos_steps = 0;
    bool profile = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int prof_launches = 0;
    bool prof_valid = false;
    long long launches = 0;
    bool fcur_valid = false;
    // CUDA graphs of the mf_iterate launch sequence, one per configuration
    struct GraphEntry {
        int iters, refine, cur, rule;
        double rel_tol, gamma1, gamma2, eps;
        const float *eta;
        cudaGraphExec_t exec;
        int flushes;   // free-energy flush launches in the recorded loop
    };
    bool use_graphs = false;
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_st = nullptr;   // private stream to record on (the legacy stream cannot be captured)
    // reverse mode (allocated on first mf_unrolled_backward)
    float *adj_gs = nullptr;     // [B][N][LP]
    float *adj_gs2 = nullptr;    // [B][N][LP] (ping-pong with adj_gs)
    float *adj_dU = nullptr;     // [B][N][LP]
    float *adj_dw = nullptr;     // [B][N][nd]
    float *adj_dwx = nullptr;    // [B][nd][H][W] (host-output staging)
    float *adj_part = nullptr;   // [adjoint_blocks][L][L]
    float *adj_mu = nullptr;     // [L][L] (+ [L][L] dmu result)
};

namespace {

// The device address of a host buffer of `bytes` bytes when it lies inside
// one page-locked, mapped allocation (cudaHostAlloc / cudaHostRegister, e.g. a
// pinned tensor), else null: pageable memory, or a range that cannot be
// verified.  The layout kernels then read or write the caller's buffer
// directly over the CPU-GPU link instead of going through a staging copy;
// the range check keeps them inside the allocation.
void *pinned_device_ptr(const void *p, size_t bytes) {
    if (((uintptr_t)p & 3) != 0) return nullptr;   // the kernels access it as floats
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
    static const PFN_cuPointerGetAttribute_v4000 get_attr = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            fn = nullptr;
        }
        return reinterpret_cast<PFN_cuPointerGetAttribute_v4000>(fn);
    }();
    if (!get_attr) return nullptr;
    const CUdeviceptr dp = (CUdeviceptr)(uintptr_t)at.devicePointer;
    CUdeviceptr start = 0;
    size_t size = 0;
    if (get_attr(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS ||
        get_attr(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS)
        return nullptr;
    if (size == 0 || dp < start || dp - start > size || bytes > size - (dp - start)) return nullptr;
    return at.devicePointer;
}


crf_status fail_cuda(crf_t h, cudaError_t e) {
    if (e == cudaSuccess) return CRF_OK;
    if (h) h->broken = true;
    (void)cudaGetLastError();
    return CRF_E_CUDA;
}

#define CK(h, x)                                 \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return fail_cuda(h, e_); \
    } while (0)

crf_status check_handle(crf_t h) {
    if (!h) return CRF_E_INVALID;
    if (h->broken) return CRF_E_STATE;
    return CRF_OK;
}

size_t n_pix(const crf_t h) { return (size_t)h->B * h->H * h->W; }
size_t n_rows(const crf_t h) { return n_pix(h) * h->L; }
size_t n_padded(const crf_t h) { return n_pix(h) * h->LP; }

void free_all(crf_t h) {
    float *fs[] = {h->U, h->s[0], h->s[1], h->w, h->eta_fixed, h->eta_auto, h->staging, h->adapt_d, h->mom, h->vv};
    for (float *p : fs)
        if (p) cudaFree(p);
    double *ds[] = {h->Lambda, h->partial, h->ftrace, h->fcur};
    for (double *p : ds)
        if (p) cudaFree(p);
    if (h->counter) cudaFree(h->counter);
    if (h->done) cudaFree(h->done);
    if (h->status) cudaFree(h->status);
    if (h->mu_pairs) cudaFree(h->mu_pairs);
    if (h->mu_tc) cudaFree(h->mu_tc);
    int *ip[] = {h->sp_out_ptr, h->sp_out_col, h->sp_in_ptr, h->sp_in_col};
    for (int *p : ip)
        if (p) cudaFree(p);
    if (h->sp_out_w) cudaFree(h->sp_out_w);
    if (h->sp_nu) cudaFree(h->sp_nu);
    if (h->sp_in_w) cudaFree(h->sp_in_w);
    float *fd[] = {h->K32, h->q32[0], h->q32[1], h->feats, h->featsT, h->mu_dev};
    for (float *p : fd)
        if (p) cudaFree(p);
    __nv_bfloat16 *bd[] = {h->K16, h->qt16[0], h->qt16[1], h->U16};
    for (__nv_bfloat16 *p : bd)
        if (p) cudaFree(p);
    if (h->tcb.split_part) cudaFree(h->tcb.split_part);
    if (h->tcb.tile_count) cudaFree(h->tcb.tile_count);
    float *ad[] = {h->adj_gs, h->adj_gs2, h->adj_dU, h->adj_dw, h->adj_dwx, h->adj_part, h->adj_mu};
    for (float *p : ad)
        if (p) cudaFree(p);
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
}

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, (n ? n : 1) * sizeof(T));
}

crf_status ensure_trace(crf_t h, int iters) {
    if (iters <= h->trace_cap) return CRF_OK;
    int cap = h->trace_cap > 0 ? h->trace_cap : 64;
    while (cap < iters) cap *= 2;
    double *nt = nullptr;
    if (dalloc(&nt, (size_t)h->B * cap) != cudaSuccess) {
        (void)cudaGetLastError();
        return CRF_E_OOM;
    }
    CK(h, cudaMemsetAsync(nt, 0, (size_t)h->B * cap * sizeof(double), h->st));
    if (h->ftrace) {
        CK(h, cudaStreamSynchronize(h->st));
        cudaFree(h->ftrace);
    }
    h->ftrace = nt;
    h->trace_cap = cap;
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);   // they captured the old trace buffer
    h->graphs.clear();
    return CRF_OK;
}

GridStepLaunch step_args(crf_t h, const float *eta, int t, int update, double rel_tol) {
    GridStepLaunch a{};
    a.s_in = h->s[h->cur];
    a.s_out = h->s[h->cur ^ 1];
    a.U = h->U;
    a.w = h->w;
    a.eta = eta;
    a.mu_out = h->mu_pairs;
    a.mu_in = h->mu_pairs + (size_t)h->LT * mu_pair_slots(h->LT);
    a.mu_tc = reinterpret_cast<const uint4 *>(h->mu_tc);
    a.U16 = h->U16;
    a.mu_host = h->mu_pairs_host.empty() ? nullptr : h->mu_pairs_host.data();
    a.adapt_d = (h->adapt_active || (update && h->rule_kernel == 2)) ? h->adapt_d : nullptr;
    a.rule = update ? h->rule_kernel : 0;
    a.mom = h->mom;
    a.vv = h->vv;
    a.gamma1 = h->gamma1;
    a.gamma2 = h->gamma2;
    a.eps = h->eps;
    a.rule_first = t == 0;
    a.partial = h->partial;
    a.counter = h->counter;
    a.f_trace = h->ftrace;
    a.f_cur = h->fcur;
    a.done = update ? h->done : nullptr;
    a.status = h->status;
    a.B = h->B;
    a.L = h->L;
    a.H = h->H;
    a.W = h->W;
    a.conn = h->conn;
    a.t = t;
    a.trace_cap = h->trace_cap;
    a.update = update;
    a.rel_tol = rel_tol;
    a.mu_sym = h->mu_sym;
    return a;
}

DenseStepLaunch dense_args(crf_t h, const float *eta, int t, int update, double rel_tol) {
    DenseStepLaunch a{};
    a.K32 = h->K32;
    a.K16 = h->K16;
    a.featsT = h->dense_fly ? h->featsT : nullptr;
    a.q_in = h->q32[h->cur];
    a.qt_in = h->qt16[h->cur];
    a.s_in = h->s[h->cur];
    a.U = h->U;
    a.s_out = h->s[h->cur ^ 1];
    a.q_out = h->q32[h->cur ^ 1];
    a.qt_out = h->qt16[h->cur ^ 1];
    a.eta = eta;
    a.mu = h->mu_dev;
    a.partial = h->partial;
    a.counter = h->counter;
    a.f_trace = h->ftrace;
    a.f_cur = h->fcur;
    a.done = update ? h->done : nullptr;
    a.status = h->status;
    a.B = h->B;
    a.N = h->N;
    a.L = h->L;
    a.t = t;
    a.trace_cap = h->trace_cap;
    a.update = update;
    a.rel_tol = rel_tol;
    return a;
}

// One step (update = 1) or a free-energy-only pass (update = 0) of either
// model.  fp32 = 1 forces the FP32 form (refinement steps, and every
// free-energy-only pass, which is evaluated with FP32 messages).
// pending (step loops only): in/out, the partials per tile of a deferring
// grid step whose free energy awaits its sum, else 0 (see
// GridStepLaunch::defer); *flushes counts the flush launches this adds.
cudaError_t launch_step(crf_t h, const float *eta, int t, int update, double rel_tol, int fp32 = 0,
                        int *pending = nullptr, int *flushes = nullptr) {
    if (h->sparse) {
        SparseStepLaunch a{};
        a.s_in = h->s[h->cur];
        a.s_out = h->s[h->cur ^ 1];
        a.q_in = h->q32[h->cur];
        a.q_out = h->q32[h->cur ^ 1];
        a.U = h->U;
        a.out_ptr = h->sp_out_ptr;
        a.out_col = h->sp_out_col;
        a.out_w = h->sp_out_w;
        a.in_ptr = h->sp_in_ptr;
        a.in_col = h->sp_in_col;
        a.in_w = h->sp_in_w;
        a.mu = h->mu_dev;
        a.eta = eta;
        a.partial = h->partial;
        a.counter = h->counter;
        a.f_trace = h->ftrace;
        a.f_cur = h->fcur;
        a.done = (update && rel_tol > 0) ? h->done : nullptr;
        a.status = h->status;
        a.B = h->B;
        a.N = h->N;
        a.L = h->L;
        a.LP = h->LP;
        a.nblk = h->nblk;
        a.t = t;
        a.trace_cap = h->trace_cap;
        a.update = update;
        a.rel_tol = rel_tol;
        a.sym = h->mu_sym;
        return launch_sparse_step(a, h->st);
    }
    if (h->dense) {
        DenseStepLaunch a = dense_args(h, eta, t, update, rel_tol);
        if (!update || rel_tol <= 0) a.done = nullptr;
        const bool tc = h->bf16 && update && !fp32;
        if (pending) {
            // the tensor-core step defers its free energy (one partial per row tile)
            const int d = tc ? 1 : 0;
            if (*pending && !d) {
                const cudaError_t e = launch_dense_f_flush(a, t - 1, h->st);
                if (e != cudaSuccess) return e;
                if (flushes) ++*flushes;
                *pending = 0;
            }
            a.defer = d;
            a.prev_pending = *pending;
            *pending = d;
        }
        if (tc) return launch_dense_step_tc(a, h->tcb, h->st);
        return launch_dense_step_f32(a, h->st);
    }
    GridStepLaunch a = step_args(h, eta, t, update, rel_tol);
    if (!update || rel_tol <= 0) a.done = nullptr;
    a.tc = h->bf16 && update && !fp32;
    if (pending) {
        const int d = update ? grid_step_fparts(a) : 0;
        if (*pending && !d) {
            // the next kernel does not take the pending sum: flush it first
            const cudaError_t e = launch_grid_f_flush(a, t - 1, *pending, h->st);
            if (e != cudaSuccess) return e;
            if (flushes) ++*flushes;
            *pending = 0;
        }
        a.defer = d;
        a.prev_pending = *pending;
        *pending = d;
    }
    return launch_grid_step(a, h->st);
}

// After the state buffer s[cur] changed outside a step: refresh the dense
// model's q copies.
cudaError_t refresh_q(crf_t h) {
    if (!h->dense && !h->sparse) return cudaSuccess;
    h->launches++;
    return launch_dense_export_q(h->s[h->cur], h->q32[h->cur], h->qt16[h->cur], h->B, h->N, h->L, h->LP, h->st);
}

crf_status ensure_lambda(crf_t h) {
    if (h->lambda_valid) return CRF_OK;
    if (h->sparse) return CRF_E_INVALID;   // set by crf_set_graph
    LipschitzJob job{};
    job.w = h->w;
    job.Kdense = h->dense ? h->K32 : nullptr;
    job.mu_host = h->mu.data();
    job.mu_sym = h->mu_sym;
    job.B = h->B;
    job.L = h->L;
    job.H = h->dense ? 1 : h->H;
    job.W = h->dense ? h->N : h->W;
    job.P = job.W;
    job.conn = h->conn;
    job.Lambda = h->Lambda;
    job.eta = h->eta_auto;
    job.max_steps = 4000;
    job.tol = 1e-9;    // relative change of the extreme Ritz values between checks
    int steps = 0;
    long long nl = 0;
    const int rc = estimate_lipschitz_grid(job, h->st, &steps, &nl);
    h->launches += nl;
    if (rc == -5) return CRF_E_TIMEOUT;   // a bounded wait ran out; the handle stays usable
    if (rc != 0) return fail_cuda(h, cudaErrorUnknown);
    h->lanczos_steps = steps;
    h->lambda_valid = true;
    return CRF_OK;
}

crf_status read_status(crf_t h) {
    int s = 0;
    CK(h, cudaMemcpyAsync(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (s != 0) {
        CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
        // a step kernel's bounded wait ran out: copies or MMAs it waited for
        // may still have been in flight, so the handle is not used again
        if (s == CRF_E_TIMEOUT) h->broken = true;
        return (crf_status)s;
    }
    return CRF_OK;
}

}  // namespace

namespace proxmf {

cudaError_t launch_grid_step(const GridStepLaunch &a, cudaStream_t st) {
    switch (kernel_labels(a.L)) {
    case 2: return launch_grid_step_l2(a, st);
    case 4: return launch_grid_step_l4(a, st);
    case 8: return launch_grid_step_l8(a, st);
    case 12: return launch_grid_step_l12(a, st);
    case 16: return launch_grid_step_l16(a, st);
    case 20: return launch_grid_step_l20(a, st);
    case 21: return launch_grid_step_l21(a, st);
    case 24: return launch_grid_step_l24(a, st);
    case 28: return launch_grid_step_l28(a, st);
    default: return launch_grid_step_l32(a, st);
    }
}

// Column pairs (for mu S) and row pairs (for mu^T S) of mu, zero padded to
// the kernel label count (see mu_pair_slots).
void build_mu_pairs_host(const float *mu, int L, int LT, float2 *out) {
    const int NPP = mu_pair_slots(LT);
    auto at = [&](int r, int c) { return (r < L && c < L) ? mu[(size_t)r * L + c] : 0.f; };
    for (int k = 0; k < LT; ++k)
        for (int j = 0; j < NPP; ++j) {
            out[(size_t)k * NPP + j] = make_float2(at(2 * j, k), at(2 * j + 1, k));
            out[(size_t)(LT + k) * NPP + j] = make_float2(at(k, 2 * j), at(k, 2 * j + 1));
        }
}

// BF16 B-operand images for the tensor-core grid step: B[n][k] = mu[n][k]
// (m = mu S_out) followed by B'[n][k] = mu[k][n] (m += mu^T S_in), each
// KP x KP in the core-matrix layout of tc_sbo, zero outside L x L.
void build_mu_tc_image(const std::vector<float> &mu, int L, int KP, std::vector<uint8_t> &out) {
    out.assign((size_t)2 * KP * KP * 2, 0);
    const int sbo = tc_sbo(KP);
    for (int part = 0; part < 2; ++part)
        for (int n = 0; n < L; ++n)
            for (int k = 0; k < L; ++k) {
                const float v = part == 0 ? mu[(size_t)n * L + k] : mu[(size_t)k * L + n];
                const __nv_bfloat16 bv = __float2bfloat16_rn(v);
                const size_t off = (size_t)part * KP * KP * 2 + (size_t)(n / 8) * sbo + (k / 8) * 128 + (n % 8) * 16 +
                                   (k % 8) * 2;
                std::memcpy(out.data() + off, &bv, 2);
            }
}

void build_mu_pairs(const std::vector<float> &mu, int L, int LT, std::vector<float2> &out) {
    out.assign((size_t)2 * LT * mu_pair_slots(LT), make_float2(0.f, 0.f));
    build_mu_pairs_host(mu.data(), L, LT, out.data());
}

}  // namespace proxmf

namespace {

// CSR of a graph given as (src, dst, w) triples: variable i's list holds
// (dst, w) of the edges leaving i and, when `both`, (src, w) of those
// entering it; otherwise `in_*` receives the entering edges separately.
void build_csr(int N, int64_t E, const int32_t *src, const int32_t *dst, const float *w, bool both,
                      std::vector<int> &optr, std::vector<int> &ocol, std::vector<float> &ow, std::vector<int> &iptr,
                      std::vector<int> &icol, std::vector<float> &iw) {
    optr.assign((size_t)N + 1, 0);
    iptr.assign((size_t)N + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        optr[(size_t)src[e] + 1]++;
        if (both)
            optr[(size_t)dst[e] + 1]++;
        else
            iptr[(size_t)dst[e] + 1]++;
    }
    for (int i = 0; i < N; ++i) {
        optr[(size_t)i + 1] += optr[i];
        iptr[(size_t)i + 1] += iptr[i];
    }
    ocol.assign((size_t)optr[N], 0);
    ow.assign((size_t)optr[N], 0.f);
    icol.assign((size_t)iptr[N], 0);
    iw.assign((size_t)iptr[N], 0.f);
    std::vector<int> fo(optr.begin(), optr.end() - 1), fi(iptr.begin(), iptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
        const int a = src[e], b = dst[e];
        ocol[(size_t)fo[a]] = b;
        ow[(size_t)fo[a]++] = w[e];
        if (both) {
            ocol[(size_t)fo[b]] = a;
            ow[(size_t)fo[b]++] = w[e];
        } else {
            icol[(size_t)fi[b]] = a;
            iw[(size_t)fi[b]++] = w[e];
        }
    }
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &v, cudaStream_t st) {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    cudaError_t e = dalloc(dst, v.size());
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    return e;
}

}  // namespace

extern "C" {

const char *crf_version(void) { return "proxmf 0.1 (sm_103a)"; }

const char *crf_error_string(crf_status s) {
    switch (s) {
    case CRF_OK: return "ok";
    case CRF_E_INVALID: return "invalid argument, size or call order";
    case CRF_E_OOM: return "device allocation failed";
    case CRF_E_CUDA: return "CUDA error (handle is now unusable)";
    case CRF_E_STATE: return "handle unusable after an earlier CUDA error";
    case CRF_E_TIMEOUT: return "bounded wait ran out";
    case CRF_E_NUMERIC: return "non-finite free energy";
    case CRF_E_UNSUPPORTED: return "request outside what this build supports";
    }
    return "unknown status";
}

crf_status crf_create(const crf_desc *desc, crf_t *out) {
    PROXMF_RANGE("crf_create");
    if (!out) return CRF_E_INVALID;
    *out = nullptr;
    if (!desc) return CRF_E_INVALID;
    const crf_desc &d = *desc;
    if (d.n_labels < 1 || d.n_labels > kMaxLabels || d.batch < 1 || d.height < 1 || d.width < 1)
        return CRF_E_INVALID;
    if (d.precision != CRF_FP32 && d.precision != CRF_BF16) return CRF_E_INVALID;
    if (d.topology != CRF_GRID4 && d.topology != CRF_GRID8 && d.topology != CRF_DENSE_GAUSS &&
        d.topology != CRF_SPARSE)
        return CRF_E_INVALID;
    const bool dense = d.topology == CRF_DENSE_GAUSS;
    const bool sparse = d.topology == CRF_SPARSE;
    if (sparse) {
        if (d.precision != CRF_FP32) return CRF_E_UNSUPPORTED;
        if ((long long)d.height * d.width >= (1ll << 31) || d.batch > 65535 ||
            (long long)d.batch * d.height * d.width * storage_labels(d.n_labels) > (1ll << 40))
            return CRF_E_INVALID;
    }
    if (dense) {
        // the dense step keeps up to 24 labels per row; N x N weights per instance
        if (d.n_labels > 24) return CRF_E_UNSUPPORTED;
        const long long N = d.height * d.width;
        if (N > 65536 || d.batch > 65535 || (long long)d.batch * N * N * 4 > (64ll << 30)) return CRF_E_INVALID;
    } else if (!sparse) {
        // grid dimensions: y tiles <= 65535, batch <= 65535 (CUDA grid limits)
        if (d.height > 65535ll * GY || d.width > (1 << 24) || d.batch > 65535) return CRF_E_INVALID;
        if ((long long)d.batch * storage_labels(d.n_labels) * d.height * d.width > (1ll << 40))
            return CRF_E_INVALID;
    }

    crf_t h = new (std::nothrow) crf_s();
    if (!h) return CRF_E_OOM;
    h->d = d;
    h->B = d.batch;
    h->L = d.n_labels;
    h->H = (int)d.height;
    h->W = (int)d.width;
    h->LP = storage_labels(h->L);
    h->LT = kernel_labels(h->L);
    h->conn = d.topology == CRF_GRID8 ? 8 : 4;
    h->nd = h->conn == 8 ? 4 : 2;
    h->st = (cudaStream_t)d.stream;
    int nbx, nby;
    grid_tiles(h->H, h->W, &nbx, &nby);
    h->nblk = nbx * nby;
    h->dense = dense;
    h->N = h->H * h->W;
    if (dense) {
        h->nd = 0;
        h->nblk = dense_nblk(h->N);
    }
    h->sparse = sparse;
    if (sparse) {
        h->nd = 0;
        h->nblk = sparse_blocks(h->N);
        h->conn = 0;
    }
    h->mu.assign((size_t)h->L * h->L, 0.f);

    bool ok = true;
    ok = ok && dalloc(&h->U, n_padded(h)) == cudaSuccess;
    ok = ok && dalloc(&h->s[0], n_padded(h)) == cudaSuccess;
    ok = ok && dalloc(&h->s[1], n_padded(h)) == cudaSuccess;
    ok = ok && dalloc(&h->w, n_pix(h) * h->nd) == cudaSuccess;
    if (sparse) {
        ok = ok && dalloc(&h->sp_nu, 2) == cudaSuccess;
        ok = ok && dalloc(&h->q32[0], n_padded(h)) == cudaSuccess;
        ok = ok && dalloc(&h->q32[1], n_padded(h)) == cudaSuccess;
    }
    if (dense) {
        const size_t qn = n_padded(h) + 64 * (size_t)h->LP;   // rows past N read as zero
        ok = ok && dalloc(&h->K32, (size_t)h->B * h->N * h->N) == cudaSuccess;
        ok = ok && dalloc(&h->q32[0], qn) == cudaSuccess;
        ok = ok && dalloc(&h->q32[1], qn) == cudaSuccess;
        ok = ok && dalloc(&h->feats, (size_t)h->B * h->N * 5) == cudaSuccess;
        if (ok) {
            ok = cudaMemsetAsync(h->q32[0], 0, qn * sizeof(float), h->st) == cudaSuccess &&
                 cudaMemsetAsync(h->q32[1], 0, qn * sizeof(float), h->st) == cudaSuccess;
        }
        if (ok && d.precision == CRF_BF16) {
            h->bf16 = true;
            const size_t pitch = dense_tc_pitch(h->N);
            const size_t tiles = (size_t)h->B * dense_tc_tiles(h->N);
            ok = ok && dalloc(&h->K16, tiles * 128 * pitch) == cudaSuccess;   // every instance's tiles x 128 rows
            ok = ok && dalloc(&h->qt16[0], (size_t)h->B * 32 * pitch) == cudaSuccess;
            ok = ok && dalloc(&h->qt16[1], (size_t)h->B * 32 * pitch) == cudaSuccess;
            ok = ok && dalloc(&h->tcb.split_part, tiles * 2 * 128 * 32) == cudaSuccess;
            ok = ok && dalloc(&h->tcb.tile_count, tiles) == cudaSuccess;
            ok = ok && dalloc(&h->featsT, (size_t)h->B * (pitch / 64) * 6 * 64) == cudaSuccess;
            if (ok)
                ok = cudaMemsetAsync(h->qt16[0], 0, (size_t)h->B * 32 * pitch * 2, h->st) == cudaSuccess &&
                     cudaMemsetAsync(h->qt16[1], 0, (size_t)h->B * 32 * pitch * 2, h->st) == cudaSuccess &&
                     cudaMemsetAsync(h->tcb.tile_count, 0, tiles * sizeof(unsigned), h->st) == cudaSuccess;
        }
    }
    ok = ok && dalloc(&h->mu_pairs, (size_t)2 * h->LT * mu_pair_slots(h->LT)) == cudaSuccess;
    ok = ok && dalloc(&h->mu_dev, (size_t)h->L * h->L) == cudaSuccess;
    if (!dense && d.precision == CRF_BF16) {
        h->bf16 = true;
        ok = ok && dalloc(&h->mu_tc, kTcImageBytes) == cudaSuccess;
        if (ok) ok = cudaMemsetAsync(h->mu_tc, 0, kTcImageBytes, h->st) == cudaSuccess;
        if (!sparse) {
            const size_t nu = n_pix(h) * u16_pitch(h->LP);
            ok = ok && dalloc(&h->U16, nu) == cudaSuccess;
            if (ok) ok = cudaMemsetAsync(h->U16, 0, nu * sizeof(__nv_bfloat16), h->st) == cudaSuccess;
        }
    }
    ok = ok && dalloc(&h->eta_fixed, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->adapt_d, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->eta_auto, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->Lambda, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->partial, 2 * (size_t)kMaxFParts * h->B * h->nblk) == cudaSuccess;
    ok = ok && dalloc(&h->counter, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->fcur, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->done, h->B) == cudaSuccess;
    ok = ok && dalloc(&h->status, 1) == cudaSuccess;
    ok = ok && dalloc(&h->staging, n_rows(h)) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        free_all(h);
        delete h;
        return CRF_E_OOM;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemsetAsync(h->U, 0, n_padded(h) * sizeof(float), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->s[0], 0, n_padded(h) * sizeof(float), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->s[1], 0, n_padded(h) * sizeof(float), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->w, 0, n_pix(h) * h->nd * sizeof(float), h->st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->mu_pairs, 0, (size_t)2 * h->LT * mu_pair_slots(h->LT) * sizeof(float2), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->counter, 0, h->B * sizeof(unsigned), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->done, 0, h->B * sizeof(int), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->fcur, 0, h->B * sizeof(double), h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_all(h);
        delete h;
        return CRF_E_CUDA;
    }
    crf_status rc = ensure_trace(h, 64);
    if (rc != CRF_OK) {
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return CRF_OK;
}

crf_status crf_destroy(crf_t h) {
    PROXMF_RANGE("crf_destroy");
    if (!h) return CRF_OK;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
    return CRF_OK;
}

crf_status crf_set_unary(crf_t h, const float *U, int is_device) {
    PROXMF_RANGE("crf_set_unary");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!U) return CRF_E_INVALID;
    const float *src = U;
    if (!is_device) {
        const size_t bytes = n_rows(h) * sizeof(float);
        if (const void *dp = pinned_device_ptr(U, bytes)) {
            src = static_cast<const float *>(dp);   // read in place by the layout kernel
        } else {
            CK(h, cudaMemcpyAsync(h->staging, U, bytes, cudaMemcpyHostToDevice, h->st));
            src = h->staging;
        }
    }
    CK(h, launch_rows_to_padded(src, h->U, (long long)n_pix(h), h->L, h->LP, 0.f, h->st));
    CK(h, launch_init_logq(h->U, h->s[0], (long long)n_pix(h), h->L, h->LP, h->st));
    h->launches += 2;
    if (h->U16) {   // the BF16 form's unaries
        CK(h, launch_to_bf16(h->U, h->U16, (long long)n_pix(h), h->LP, u16_pitch(h->LP), h->st));
        h->launches++;
    }
    h->cur = 0;
    CK(h, refresh_q(h));
    h->fcur_valid = false;
    if (!is_device) CK(h, cudaStreamSynchronize(h->st));
    h->has_unary = true;
    return CRF_OK;
}

// Fully connected model: features and bandwidths in, K (and its BF16 copy
// for the tensor-core form) built on the device.
static crf_status set_pairwise_dense(crf_t h, const std::vector<float> &m, const float *feats,
                                     const float *theta, int is_device) {
    double th[2];
    if (!theta) return CRF_E_INVALID;
    if (is_device) {
        float t2[2];
        CK(h, cudaMemcpyAsync(t2, theta, sizeof(t2), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        th[0] = t2[0];
        th[1] = t2[1];
    } else {
        th[0] = theta[0];
        th[1] = theta[1];
    }
    if (!(th[0] > 0) || !(th[1] > 0) || !std::isfinite(th[0]) || !std::isfinite(th[1])) return CRF_E_INVALID;
    const size_t nf = (size_t)h->B * h->N * 5;
    CK(h, cudaMemcpyAsync(h->feats, feats, nf * sizeof(float),
                          is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->mu_dev, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice, h->st));
    CK(h, launch_dense_kernel_build(h->feats, h->K32, h->K16, h->B, h->N, th[0], th[1], h->st));
    if (h->featsT) CK(h, launch_dense_fly_features(h->feats, h->featsT, h->B, h->N, th[0], th[1], h->st));
    h->launches += h->K16 ? 2 : 1;
    CK(h, cudaStreamSynchronize(h->st));   // m and a host feats buffer are pageable
    h->theta[0] = th[0];
    h->theta[1] = th[1];
    h->mu = m;
    h->mu_sym = true;
    h->has_pairwise = true;
    h->lambda_valid = false;
    h->fcur_valid = false;
    return CRF_OK;
}

crf_status crf_set_pairwise(crf_t h, const float *mu, const float *w_or_feats, const float *theta,
                            int is_device) {
    PROXMF_RANGE("crf_set_pairwise");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!mu || !w_or_feats) return CRF_E_INVALID;
    if (h->sparse) return CRF_E_INVALID;   // crf_set_graph
    const size_t LL = (size_t)h->L * h->L;
    std::vector<float> m(LL);
    if (is_device) {
        CK(h, cudaMemcpyAsync(m.data(), mu, LL * sizeof(float), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
    } else {
        std::memcpy(m.data(), mu, LL * sizeof(float));
    }
    for (float v : m)
        if (!std::isfinite(v)) return CRF_E_INVALID;
    bool sym = true;
    for (int i = 0; i < h->L; ++i)
        for (int k = i + 1; k < h->L; ++k)
            if (m[i * h->L + k] != m[k * h->L + i]) sym = false;
    if (h->dense) {
        // pairs of a fully connected model have no orientation: mu must be symmetric
        if (!sym) return CRF_E_INVALID;
        return set_pairwise_dense(h, m, w_or_feats, theta, is_device);
    }
    const size_t nw = n_pix(h) * h->nd;
    std::vector<float2> pairs;
    build_mu_pairs(m, h->L, h->LT, pairs);
    CK(h, cudaMemcpyAsync(h->mu_pairs, pairs.data(), pairs.size() * sizeof(float2), cudaMemcpyHostToDevice,
                          h->st));
    h->mu_pairs_host = pairs;
    CK(h, cudaMemcpyAsync(h->mu_dev, m.data(), LL * sizeof(float), cudaMemcpyHostToDevice, h->st));
    std::vector<uint8_t> img;
    if (h->bf16) {
        build_mu_tc_image(m, h->L, tc_k(h->LT), img);
        CK(h, cudaMemcpyAsync(h->mu_tc, img.data(), img.size(), cudaMemcpyHostToDevice, h->st));
    }
    const float *src = w_or_feats;
    if (!is_device) {
        // the staging buffer holds B*N*L floats >= B*nd*N only when L >= nd
        if (nw > n_rows(h)) {
            float *tmp = nullptr;
            CK(h, cudaMalloc((void **)&tmp, nw * sizeof(float)));
            cudaError_t e = cudaMemcpyAsync(tmp, w_or_feats, nw * sizeof(float), cudaMemcpyHostToDevice, h->st);
            if (e == cudaSuccess) e = launch_weights_to_pixel_major(tmp, h->w, h->B, h->nd, h->H, h->W, h->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
            cudaFree(tmp);
            CK(h, e);
        } else {
            CK(h, cudaMemcpyAsync(h->staging, w_or_feats, nw * sizeof(float), cudaMemcpyHostToDevice, h->st));
            CK(h, launch_weights_to_pixel_major(h->staging, h->w, h->B, h->nd, h->H, h->W, h->st));
            CK(h, cudaStreamSynchronize(h->st));
        }
    } else {
        CK(h, launch_weights_to_pixel_major(src, h->w, h->B, h->nd, h->H, h->W, h->st));
        CK(h, cudaStreamSynchronize(h->st));   // the pair table above is pageable host memory
    }
    h->launches++;
    h->mu = m;
    h->mu_sym = sym;
    h->fcur_valid = false;
    h->has_pairwise = true;
    h->lambda_valid = false;
    return CRF_OK;
}

crf_status crf_set_graph(crf_t h, const float *mu, int64_t n_edges, const int32_t *src, const int32_t *dst,
                         const float *w, int32_t is_device) {
    PROXMF_RANGE("crf_set_graph");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!h->sparse || !mu || n_edges < 0 || n_edges > (1ll << 30) || (n_edges > 0 && (!src || !dst || !w)))
        return CRF_E_INVALID;
    const size_t LL = (size_t)h->L * h->L, E = (size_t)n_edges;
    std::vector<float> m(LL), wv(E);
    std::vector<int32_t> sv(E), dv(E);
    if (is_device) {
        CK(h, cudaMemcpyAsync(m.data(), mu, LL * sizeof(float), cudaMemcpyDeviceToHost, h->st));
        if (E) {
            CK(h, cudaMemcpyAsync(sv.data(), src, E * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
            CK(h, cudaMemcpyAsync(dv.data(), dst, E * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
            CK(h, cudaMemcpyAsync(wv.data(), w, E * sizeof(float), cudaMemcpyDeviceToHost, h->st));
        }
        CK(h, cudaStreamSynchronize(h->st));
    } else {
        std::memcpy(m.data(), mu, LL * sizeof(float));
        if (E) {
            std::memcpy(sv.data(), src, E * sizeof(int32_t));
            std::memcpy(dv.data(), dst, E * sizeof(int32_t));
            std::memcpy(wv.data(), w, E * sizeof(float));
        }
    }
    for (float v : m)
        if (!std::isfinite(v)) return CRF_E_INVALID;
    for (size_t e = 0; e < E; ++e)
        if (sv[e] < 0 || sv[e] >= h->N || dv[e] < 0 || dv[e] >= h->N || sv[e] == dv[e] || !std::isfinite(wv[e]))
            return CRF_E_INVALID;
    bool sym = true;
    for (int i = 0; i < h->L; ++i)
        for (int j = i + 1; j < h->L; ++j)
            if (m[(size_t)i * h->L + j] != m[(size_t)j * h->L + i]) sym = false;
    std::vector<int> optr, ocol, iptr, icol;
    std::vector<float> ow, iw;
    build_csr(h->N, n_edges, sv.data(), dv.data(), wv.data(), sym, optr, ocol, ow, iptr, icol, iw);
    CK(h, upload(&h->sp_out_ptr, optr, h->st));
    CK(h, upload(&h->sp_out_col, ocol, h->st));
    CK(h, upload(&h->sp_out_w, ow, h->st));
    CK(h, upload(&h->sp_in_ptr, iptr, h->st));
    CK(h, upload(&h->sp_in_col, icol, h->st));
    CK(h, upload(&h->sp_in_w, iw, h->st));
    CK(h, cudaMemcpyAsync(h->mu_dev, m.data(), LL * sizeof(float), cudaMemcpyHostToDevice, h->st));
    // step bound (see proxmf.h): the largest summed |w| per variable, and
    // the spectrum of C mu C (symmetric mu) or ||mu||_F
    unsigned *deg = reinterpret_cast<unsigned *>(h->counter);   // counters are zero between launches
    unsigned bits[2] = {0u, 0u};
    CK(h, launch_sparse_degree(h->sp_out_ptr, h->sp_out_w, h->N, deg, h->st));
    CK(h, cudaMemcpyAsync(&bits[0], deg, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
    if (!sym) {
        CK(h, launch_sparse_degree(h->sp_in_ptr, h->sp_in_w, h->N, deg, h->st));
        CK(h, cudaMemcpyAsync(&bits[1], deg, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
    }
    double nu[2] = {0.0, 0.0};
    if (sym) {
        CK(h, launch_mu_tilde_extremes(h->mu_dev, h->L, h->sp_nu, h->st));
        CK(h, cudaMemcpyAsync(nu, h->sp_nu, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    }
    CK(h, cudaMemsetAsync(h->counter, 0, h->B * sizeof(unsigned), h->st));
    CK(h, cudaStreamSynchronize(h->st));
    float d0, d1;
    std::memcpy(&d0, &bits[0], 4);
    std::memcpy(&d1, &bits[1], 4);
    double lam;
    if (sym) {
        lam = (double)d0 * std::max(std::fabs(nu[0]), std::fabs(nu[1]));
    } else {
        double fro = 0.0;
        for (float v : m) fro += (double)v * v;
        lam = ((double)d0 + (double)d1) * std::sqrt(fro);
    }
    std::vector<double> L(h->B, lam);
    std::vector<float> eta(h->B, (float)(1.0 / (1.0 + std::max(lam, 0.0))));
    CK(h, cudaMemcpyAsync(h->Lambda, L.data(), h->B * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->eta_auto, eta.data(), h->B * sizeof(float), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    h->launches += sym ? 2 : 2;
    h->mu = m;
    h->mu_sym = sym;
    h->lambda_valid = true;
    h->has_pairwise = true;
    h->fcur_valid = false;
    return CRF_OK;
}

crf_status crf_set_state(crf_t h, const float *logq, int is_device) {
    PROXMF_RANGE("crf_set_state");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!logq) return CRF_E_INVALID;
    const float *src = logq;
    if (!is_device) {
        CK(h, cudaMemcpyAsync(h->staging, logq, n_rows(h) * sizeof(float), cudaMemcpyHostToDevice, h->st));
        src = h->staging;
    }
    CK(h, launch_rows_to_padded(src, h->s[h->cur], (long long)n_pix(h), h->L, h->LP, kPadLogQ, h->st));
    h->launches++;
    CK(h, refresh_q(h));
    h->fcur_valid = false;
    if (!is_device) CK(h, cudaStreamSynchronize(h->st));
    return CRF_OK;
}

crf_status mf_iterate(crf_t h, const mf_params *p, int32_t *iters_done) {
    PROXMF_RANGE("mf_iterate");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!p || p->max_iters < 0 || p->rel_tol < 0 || !std::isfinite(p->eta) || p->eta > 1.0)
        return CRF_E_INVALID;
    if (!h->has_unary || !h->has_pairwise) return CRF_E_INVALID;
    if (p->rule < MF_RULE_FIXED || p->rule > MF_RULE_ADHOC) return CRF_E_INVALID;
    if (p->rule == MF_RULE_ADHOC && (h->dense || h->sparse || h->bf16)) return CRF_E_UNSUPPORTED;
    if (p->rule == MF_RULE_MOMENTUM || p->rule == MF_RULE_ADAM) {
        if (h->dense || h->sparse || h->bf16) return CRF_E_UNSUPPORTED;
        if (!(p->gamma1 >= 0 && p->gamma1 <= 1)) return CRF_E_INVALID;
        if (p->rule == MF_RULE_ADAM &&
            (!(p->gamma2 >= 0 && p->gamma2 <= 1) || !(p->epsilon >= 0) || !std::isfinite(p->epsilon) ||
             !std::isfinite(p->d)))
            return CRF_E_INVALID;
        if (!h->mom) {
            if (dalloc(&h->mom, n_padded(h)) != cudaSuccess || dalloc(&h->vv, n_padded(h)) != cudaSuccess) {
                (void)cudaGetLastError();
                return CRF_E_OOM;
            }
        }
        if (p->rule == MF_RULE_ADAM) {
            if (p->d > 0) {
                CK(h, launch_fill_eta(h->adapt_d, h->B, p->d, h->st));
            } else {
                const crf_status lr = ensure_lambda(h);
                if (lr != CRF_OK) return lr;
                CK(h, launch_lambda_to_d(h->Lambda, h->adapt_d, h->B, h->st));
            }
            h->launches++;
        }
    }
    if (p->rule == MF_RULE_ADAPTIVE) {
        if (h->dense || h->sparse || h->L != 2) return CRF_E_UNSUPPORTED;
        if (!std::isfinite(p->d)) return CRF_E_INVALID;
        if (p->d > 0) {
            CK(h, launch_fill_eta(h->adapt_d, h->B, p->d, h->st));
        } else {
            const crf_status lr = ensure_lambda(h);
            if (lr != CRF_OK) return lr;
            CK(h, launch_lambda_to_d(h->Lambda, h->adapt_d, h->B, h->st));
        }
        h->launches++;
    }
    const float *eta = nullptr;
    if (p->rule == MF_RULE_ADAPTIVE || p->rule == MF_RULE_ADAM) {
        eta = h->eta_fixed;   // unused by these epilogues
    } else if (p->eta > 0) {
        CK(h, launch_fill_eta(h->eta_fixed, h->B, p->eta, h->st));
        h->launches++;
        eta = h->eta_fixed;
    } else {
        rc = ensure_lambda(h);
        if (rc != CRF_OK) return rc;
        eta = h->eta_auto;
    }
    if (p->reset) {
        CK(h, launch_init_logq(h->U, h->s[h->cur], (long long)n_pix(h), h->L, h->LP, h->st));
        h->launches++;
        CK(h, refresh_q(h));
    }
    const int refine = (h->bf16 && p->refine_fp32 > 0) ? p->refine_fp32 : 0;
    if (p->refine_fp32 < 0) return CRF_E_INVALID;
    rc = ensure_trace(h, p->max_iters + refine);
    if (rc != CRF_OK) return rc;
    const int nsteps = p->max_iters + refine;
    // the step loop: eager, or captured once per configuration and replayed
    int loop_flushes = 0;   // free-energy flush launches of the loop
    auto body = [&]() -> cudaError_t {
        if (p->rel_tol > 0) {
            cudaError_t e = cudaMemsetAsync(h->done, 0, h->B * sizeof(int), h->st);
            if (e != cudaSuccess) return e;
        }
        int pending = 0;
        loop_flushes = 0;
        for (int t = 0; t < nsteps; ++t) {
            cudaError_t e = launch_step(h, eta, t, 1, p->rel_tol, t >= p->max_iters, &pending, &loop_flushes);
            if (e != cudaSuccess) return e;
            h->cur ^= 1;
        }
        if (pending) {
            cudaError_t e;
            if (h->dense) {
                DenseStepLaunch a = dense_args(h, eta, nsteps - 1, 1, p->rel_tol);
                if (p->rel_tol <= 0) a.done = nullptr;
                e = launch_dense_f_flush(a, nsteps - 1, h->st);
            } else {
                GridStepLaunch a = step_args(h, eta, nsteps - 1, 1, p->rel_tol);
                if (p->rel_tol <= 0) a.done = nullptr;
                e = launch_grid_f_flush(a, nsteps - 1, pending, h->st);
            }
            if (e != cudaSuccess) return e;
            ++loop_flushes;
        }
        return cudaSuccess;
    };
    h->adapt_active = p->rule == MF_RULE_ADAPTIVE;
    h->rule_kernel = p->rule == MF_RULE_MOMENTUM ? 1 : (p->rule == MF_RULE_ADAM ? 2 : (p->rule == MF_RULE_ADHOC ? 3 : 0));
    h->gamma1 = (float)p->gamma1;
    h->gamma2 = (float)p->gamma2;
    h->eps = (float)p->epsilon;
    // small grids: the whole loop in one launch, one thread-block cluster per
    // instance with the iterates in shared memory (fixed rule, FP32)
    const bool resident = h->use_resident && !h->dense && !h->sparse && !h->bf16 && p->rule == MF_RULE_FIXED &&
                          nsteps >= 2 && grid_resident_fits(h->H, h->W, h->L, h->LP);
    cudaGraphExec_t exec = nullptr;
    if (h->use_graphs && nsteps > 0 && !resident) {
        for (auto &g : h->graphs)
            if (g.iters == p->max_iters && g.refine == refine && g.cur == h->cur && g.rel_tol == p->rel_tol &&
                g.eta == eta && g.rule == p->rule && g.gamma1 == p->gamma1 && g.gamma2 == p->gamma2 &&
                g.eps == p->epsilon) {
                exec = g.exec;
                loop_flushes = g.flushes;
            }
        if (!exec) {
            const int cur0 = h->cur;
            if (!h->cap_st) CK(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
            // record the loop on the private stream; the graph is launched on the handle's stream
            cudaStream_t st0 = h->st;
            h->st = h->cap_st;
            cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) e = body();
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(h->st, &graph);
            h->st = st0;
            h->cur = cur0;   // nothing ran yet
            if (e != cudaSuccess || e2 != cudaSuccess) {
                h->adapt_active = false;
                h->rule_kernel = 0;
                if (graph) cudaGraphDestroy(graph);
                return fail_cuda(h, e != cudaSuccess ? e : e2);
            }
            const cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                h->adapt_active = false;
                h->rule_kernel = 0;
            }
            CK(h, e3);
            h->graphs.push_back({p->max_iters, refine, cur0, p->rule, p->rel_tol, p->gamma1, p->gamma2, p->epsilon,
                                 eta, exec, loop_flushes});
        }
    }
    if (h->profile) CK(h, cudaEventRecord(h->ev0, h->st));
    if (resident) {
        h->adapt_active = false;
        h->rule_kernel = 0;
        if (p->rel_tol > 0) CK(h, cudaMemsetAsync(h->done, 0, h->B * sizeof(int), h->st));
        GridResidentLaunch ra{};
        ra.s_in = h->s[h->cur];
        ra.s_out = h->s[h->cur ^ (nsteps & 1)];   // where the step-by-step loop would leave it
        ra.U = h->U;
        ra.w = h->w;
        ra.mu = h->mu_dev;
        ra.eta = eta;
        ra.f_trace = h->ftrace;
        ra.f_cur = h->fcur;
        ra.done = h->done;
        ra.status = h->status;
        ra.B = h->B;
        ra.H = h->H;
        ra.W = h->W;
        ra.L = h->L;
        ra.LP = h->LP;
        ra.conn = h->conn;
        ra.mu_sym = h->mu_sym ? 1 : 0;
        ra.nsteps = nsteps;
        ra.trace_cap = h->trace_cap;
        ra.rel_tol = p->rel_tol;
        CK(h, launch_grid_resident(ra, h->st));
        h->cur ^= nsteps & 1;
    } else if (exec) {
        h->adapt_active = false;
        h->rule_kernel = 0;
        CK(h, cudaGraphLaunch(exec, h->st));
        h->cur ^= nsteps & 1;
    } else {
        const cudaError_t e = body();
        h->adapt_active = false;
        h->rule_kernel = 0;
        CK(h, e);
    }
    h->launches += resident ? 1 : nsteps + loop_flushes;
    if (h->profile) {
        CK(h, cudaEventRecord(h->ev1, h->st));
        h->prof_launches = resident ? 1 : p->max_iters + refine;
        h->prof_valid = true;
    }
    h->last_iters = p->max_iters + refine;
    h->fcur_valid = false;
    if (p->final_free_energy) {
        CK(h, launch_step(h, eta, 0, 0, 0.0, 1));
        h->launches++;
        h->fcur_valid = true;
    }
    if (iters_done) {
        std::vector<int> dn(h->B);
        CK(h, cudaMemcpyAsync(dn.data(), h->done, h->B * sizeof(int), cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        for (int b = 0; b < h->B; ++b) iters_done[b] = dn[b] ? dn[b] : p->max_iters + refine;
    }
    return CRF_OK;
}

crf_status mf_free_energy(crf_t h, double *F) {
    PROXMF_RANGE("mf_free_energy");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!F) return CRF_E_INVALID;
    if (!h->has_unary || !h->has_pairwise) return CRF_E_INVALID;
    if (!h->fcur_valid) {
        CK(h, launch_fill_eta(h->eta_fixed, h->B, 1.0, h->st));
        CK(h, launch_step(h, h->eta_fixed, 0, 0, 0.0, 1));
        h->launches += 2;
        h->fcur_valid = true;
    }
    CK(h, cudaMemcpyAsync(F, h->fcur, h->B * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return read_status(h);
}

crf_status mf_free_energy_trace(crf_t h, double *F, int32_t n) {
    PROXMF_RANGE("mf_free_energy_trace");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!F || n < 0 || n > h->last_iters || n > h->trace_cap) return CRF_E_INVALID;
    if (n == 0) return CRF_OK;
    CK(h, cudaMemcpy2DAsync(F, n * sizeof(double), h->ftrace, h->trace_cap * sizeof(double),
                            n * sizeof(double), h->B, cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return CRF_OK;
}

static crf_status export_state(crf_t h, float *dst, int is_device, int mode) {
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!dst) return CRF_E_INVALID;
    const size_t bytes = n_rows(h) * sizeof(float);
    float *out = dst;
    bool staged = false;
    if (!is_device) {
        // pinned host memory is written in place by the layout kernel
        out = static_cast<float *>(pinned_device_ptr(dst, bytes));
        staged = out == nullptr;
        if (staged) out = h->staging;
    }
    CK(h, launch_padded_to_rows(h->s[h->cur], out, (long long)n_pix(h), h->L, h->LP, mode, h->st));
    h->launches++;
    if (staged) CK(h, cudaMemcpyAsync(dst, h->staging, bytes, cudaMemcpyDeviceToHost, h->st));
    if (!is_device) CK(h, cudaStreamSynchronize(h->st));
    return CRF_OK;
}

crf_status mf_marginals(crf_t h, float *q, int is_device) { return export_state(h, q, is_device, CONV_EXP); }

crf_status mf_log_marginals(crf_t h, float *logq, int is_device) {
    PROXMF_RANGE("mf_log_marginals");
    return export_state(h, logq, is_device, CONV_COPY);
}

crf_status mf_lipschitz(crf_t h, double *Lambda, double *eta) {
    PROXMF_RANGE("mf_lipschitz");
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!h->has_pairwise) return CRF_E_INVALID;
    rc = ensure_lambda(h);
    if (rc != CRF_OK) return rc;
    std::vector<float> e(h->B);
    if (Lambda) CK(h, cudaMemcpyAsync(Lambda, h->Lambda, h->B * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(e.data(), h->eta_auto, h->B * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    if (eta)
        for (int b = 0; b < h->B; ++b) eta[b] = e[b];
    return CRF_OK;
}

crf_status mf_profile(crf_t h, int32_t enable) {
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (enable && !h->ev0) {
        CK(h, cudaEventCreate(&h->ev0));
        CK(h, cudaEventCreate(&h->ev1));
    }
    h->profile = enable != 0;
    h->prof_valid = false;
    return CRF_OK;
}

crf_status mf_profile_read(crf_t h, double *loop_ms, int32_t *launches) {
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!h->prof_valid) return CRF_E_INVALID;
    CK(h, cudaEventSynchronize(h->ev1));
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (loop_ms) *loop_ms = ms;
    if (launches) *launches = h->prof_launches;
    return CRF_OK;
}

crf_status mf_use_resident(crf_t h, int32_t enable) {
    const crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    h->use_resident = enable != 0;
    return CRF_OK;
}

crf_status mf_dense_on_the_fly(crf_t h, int32_t enable) {
    const crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (!h->dense || !h->bf16) return CRF_E_UNSUPPORTED;
    if (h->dense_fly != (enable != 0)) {
        for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);   // they recorded the other kernel
        h->graphs.clear();
    }
    h->dense_fly = enable != 0;
    return CRF_OK;
}

crf_status mf_use_graphs(crf_t h, int32_t enable) {
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    h->use_graphs = enable != 0;
    return CRF_OK;
}

crf_status crf_launch_count(crf_t h, int64_t *n) {
    if (!h || !n) return CRF_E_INVALID;
    *n = h->launches;
    return CRF_OK;
}

// ---- reverse mode through K unrolled steps --------------------------------

static crf_status unrolled_check(crf_t h, int32_t K) {
    crf_status rc = check_handle(h);
    if (rc != CRF_OK) return rc;
    if (h->dense || h->sparse || h->L > kAdjointMaxLabels) return CRF_E_UNSUPPORTED;
    if (h->H > 4 * 65535) return CRF_E_UNSUPPORTED;   // reverse-step grid: 4-row tiles in gridDim.y
    if (K < 1 || K > 4096) return CRF_E_INVALID;
    return CRF_OK;
}

static size_t state_floats(const crf_t h) { return n_padded(h); }

static crf_status unrolled_eta(crf_t h, double eta, const float **out) {
    if (!std::isfinite(eta) || eta > 1.0) return CRF_E_INVALID;
    if (eta > 0) {
        CK(h, launch_fill_eta(h->eta_fixed, h->B, eta, h->st));
        h->launches++;
        *out = h->eta_fixed;
        return CRF_OK;
    }
    crf_status rc = ensure_lambda(h);
    if (rc != CRF_OK) return rc;
    *out = h->eta_auto;
    return CRF_OK;
}

crf_status mf_unrolled_checkpoint_floats(crf_t h, int32_t K, int64_t *n_floats) {
    crf_status rc = unrolled_check(h, K);
    if (rc != CRF_OK) return rc;
    if (!n_floats) return CRF_E_INVALID;
    *n_floats = (int64_t)(K + 1) * (int64_t)state_floats(h);
    return CRF_OK;
}

crf_status mf_unrolled_forward(crf_t h, int32_t K, double eta, float *ckpt) {
    PROXMF_RANGE("mf_unrolled_forward");
    crf_status rc = unrolled_check(h, K);
    if (rc != CRF_OK) return rc;
    if (!ckpt || ((uintptr_t)ckpt & 15)) return CRF_E_INVALID;
    if (!h->has_unary || !h->has_pairwise) return CRF_E_INVALID;
    const float *e = nullptr;
    rc = unrolled_eta(h, eta, &e);
    if (rc != CRF_OK) return rc;
    rc = ensure_trace(h, K);
    if (rc != CRF_OK) return rc;
    const size_t S = state_floats(h);
    CK(h, launch_init_logq(h->U, ckpt, (long long)n_pix(h), h->L, h->LP, h->st));
    if (h->profile) CK(h, cudaEventRecord(h->ev0, h->st));
    int pending = 0, flushes = 0;   // deferred free energy, as in mf_iterate
    for (int t = 0; t < K; ++t) {
        GridStepLaunch a = step_args(h, e, t, 1, 0.0);
        a.done = nullptr;
        a.tc = h->bf16;   // BF16 handles: tensor-core messages in the forward steps
        a.s_in = ckpt + (size_t)t * S;
        a.s_out = ckpt + (size_t)(t + 1) * S;
        const int d = grid_step_fparts(a);
        if (pending && !d) {
            CK(h, launch_grid_f_flush(a, t - 1, pending, h->st));
            ++flushes;
            pending = 0;
        }
        a.defer = d;
        a.prev_pending = pending;
        pending = d;
        CK(h, launch_grid_step(a, h->st));
    }
    if (pending) {
        GridStepLaunch a = step_args(h, e, K - 1, 1, 0.0);
        a.done = nullptr;
        CK(h, launch_grid_f_flush(a, K - 1, pending, h->st));
        ++flushes;
    }
    if (h->profile) {
        CK(h, cudaEventRecord(h->ev1, h->st));
        h->prof_launches = K;
        h->prof_valid = true;
    }
    CK(h, cudaMemcpyAsync(h->s[h->cur], ckpt + (size_t)K * S, S * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    h->launches += 1 + K + flushes;
    h->last_iters = K;
    h->fcur_valid = false;
    return CRF_OK;
}

crf_status mf_unrolled_backward(crf_t h, int32_t K, double eta, const float *ckpt, const float *dlogq,
                                float *dU, float *dmu, float *dw, int32_t is_device) {
    PROXMF_RANGE("mf_unrolled_backward");
    crf_status rc = unrolled_check(h, K);
    if (rc != CRF_OK) return rc;
    if (!ckpt || !dlogq || ((uintptr_t)ckpt & 15)) return CRF_E_INVALID;
    if (!h->has_pairwise) return CRF_E_INVALID;
    const size_t S = state_floats(h);
    const size_t nw = n_pix(h) * h->nd;
    const size_t LL = (size_t)h->L * h->L;
    const int nblk = adjoint_blocks(h->B, h->H, h->W);
    if (!h->adj_gs) {
        bool ok = true;
        ok = ok && dalloc(&h->adj_gs, S) == cudaSuccess;
        ok = ok && dalloc(&h->adj_gs2, S) == cudaSuccess;
        ok = ok && dalloc(&h->adj_dU, S) == cudaSuccess;
        ok = ok && dalloc(&h->adj_dw, nw) == cudaSuccess;
        ok = ok && dalloc(&h->adj_dwx, nw) == cudaSuccess;
        ok = ok && dalloc(&h->adj_part, (size_t)nblk * LL) == cudaSuccess;
        ok = ok && dalloc(&h->adj_mu, LL) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            float *ad[] = {h->adj_gs, h->adj_gs2, h->adj_dU, h->adj_dw, h->adj_dwx, h->adj_part, h->adj_mu};
            for (float *p : ad)
                if (p) cudaFree(p);
            h->adj_gs = h->adj_gs2 = h->adj_dU = h->adj_dw = h->adj_dwx = h->adj_part = h->adj_mu = nullptr;
            return CRF_E_OOM;
        }
    }
    const float *e = nullptr;
    rc = unrolled_eta(h, eta, &e);
    if (rc != CRF_OK) return rc;
    const float *src = dlogq;
    if (!is_device) {
        CK(h, cudaMemcpyAsync(h->staging, dlogq, n_rows(h) * sizeof(float), cudaMemcpyHostToDevice, h->st));
        src = h->staging;
    }
    CK(h, launch_rows_to_padded(src, h->adj_gs, (long long)n_pix(h), h->L, h->LP, 0.f, h->st));
    CK(h, cudaMemsetAsync(h->adj_dU, 0, S * sizeof(float), h->st));
    CK(h, cudaMemsetAsync(h->adj_dw, 0, nw * sizeof(float), h->st));
    CK(h, cudaMemsetAsync(h->adj_part, 0, (size_t)nblk * LL * sizeof(float), h->st));
    h->launches++;
    AdjointStep a{};
    float *gsb[2] = {h->adj_gs, h->adj_gs2};
    a.dU = h->adj_dU;
    a.dw = h->adj_dw;
    a.dmu_part = h->adj_part;
    a.w = h->w;
    a.mu = h->mu_dev;
    a.eta = e;
    a.status = h->status;
    a.B = h->B;
    a.L = h->L;
    a.H = h->H;
    a.W = h->W;
    a.conn = h->conn;
    a.mu_sym = h->mu_sym;
    if (h->profile) CK(h, cudaEventRecord(h->ev0, h->st));
    for (int t = K - 1, c = 0; t >= 0; --t, c ^= 1) {
        a.gs_in = gsb[c];
        a.gs_out = gsb[c ^ 1];
        a.s = ckpt + (size_t)t * S;
        a.s_next = ckpt + (size_t)(t + 1) * S;
        CK(h, launch_adjoint_step(a, h->st));
    }
    if (h->profile) {
        CK(h, cudaEventRecord(h->ev1, h->st));
        h->prof_launches = K;
        h->prof_valid = true;
    }
    h->launches += K;
    AdjointFinish f{};
    f.gs = gsb[K & 1];
    f.s0 = ckpt;
    f.dU = h->adj_dU;
    f.dw = h->adj_dw;
    f.dw_out = (is_device && dw) ? dw : h->adj_dwx;
    f.dmu_part = h->adj_part;
    f.dmu_out = h->adj_mu;
    f.B = h->B;
    f.L = h->L;
    f.H = h->H;
    f.W = h->W;
    f.conn = h->conn;
    CK(h, launch_adjoint_finish(f, h->st));
    h->launches += 3;
    if (dU) {
        float *out = is_device ? dU : h->staging;
        CK(h, launch_padded_to_rows(h->adj_dU, out, (long long)n_pix(h), h->L, h->LP, CONV_COPY, h->st));
        h->launches++;
        if (!is_device)
            CK(h, cudaMemcpyAsync(dU, h->staging, n_rows(h) * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    }
    if (dmu)
        CK(h, cudaMemcpyAsync(dmu, h->adj_mu, LL * sizeof(float),
                              is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
    if (dw && !is_device)
        CK(h, cudaMemcpyAsync(dw, h->adj_dwx, nw * sizeof(float), cudaMemcpyDeviceToHost, h->st));
    if (!is_device) CK(h, cudaStreamSynchronize(h->st));
    return CRF_OK;
}

}  // extern "C"
