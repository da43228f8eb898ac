// serve.cu -- host side of the serving loop (continuous batching).
//
// A server owns one device memory pool of a fixed budget.  Requests (single
// grid CRFs of any size, label count and connectivity) are copied on submit
// and queued; each step the server
//   1. retires the slots whose stopping rule fired (flags in host-mapped
//      memory): copies q out and returns the slot and its pool memory;
//   2. admits queued requests in arrival order while a slot and pool memory
//      (first-fit) are free: uploads and converts the data, builds q^0 and
//      the step size on the device, and registers the slot in its bucket;
//   3. replays a CUDA graph holding one persistent launch per bucket
//      (serve.cuh) for the requested number of iterations.
// Requests therefore join and leave between iterations while the others keep
// running, and every request's arithmetic is that of a solve on its own.
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/proxmf.h"
#include "nvtx_range.h"
#include "serve.cuh"

using namespace proxmf;

namespace {

// First-fit allocator over [0, size) with 256-byte granules and coalescing.
class Pool {
public:
    explicit Pool(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    int H = 0, W = 0, L = 0, conn = 4;
    std::vector<float> U, mu, w;
    mf_params p{};
    float *q_out = nullptr;
    int state = 0;               // 0 queued, 1 running, 2 done
    int slot = -1;
    size_t off = 0, bytes = 0;
    double F = 0.0;
    int iters = 0;
    bool sym = true;
};

constexpr int kMaxBuckets = 64;

}  // namespace

struct mf_server_s {
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;
    size_t budget = 0;
    int max_slots = 0;
    unsigned char *pool_base = nullptr;
    Pool *pool = nullptr;
    ServeSlot *d_slots = nullptr;
    ServeBucket *d_buckets = nullptr;
    ServeResult *h_res = nullptr, *d_res = nullptr;   // host-mapped
    double *d_scratch = nullptr;
    float *staging = nullptr;
    size_t staging_floats = 0;
    std::vector<ServeBucket> h_buckets;
    std::vector<int> bucket_lt, bucket_conn, bucket_sym;
    std::vector<bool> bucket_dirty;
    std::vector<int> slot_ticket;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_stale = true;
    bool broken = false;
    int grid_small = 0, grid_large = 0;
};

namespace {

crf_status srv_cuda(mf_server_t s, cudaError_t e) {
    if (e == cudaSuccess) return CRF_OK;
    s->broken = true;
    (void)cudaGetLastError();
    return CRF_E_CUDA;
}

#define SCK(x)                                          \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) return srv_cuda(s, e_);  \
    } while (0)

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Pool layout of one request (byte offsets from its base).
struct SlotLayout {
    size_t U, s0, s1, w, pairs, mu, partial, counter, eta, total;
};

SlotLayout layout_for(const Request &r) {
    const size_t N = (size_t)r.H * r.W;
    const int LP = storage_labels(r.L), LT = kernel_labels(r.L), nd = r.conn == 8 ? 4 : 2;
    int nbx, nby;
    grid_tiles(r.H, r.W, &nbx, &nby);
    SlotLayout l{};
    size_t o = 0;
    l.U = o; o += align256(N * LP * 4);
    l.s0 = o; o += align256(N * LP * 4);
    l.s1 = o; o += align256(N * LP * 4);
    l.w = o; o += align256(N * nd * 4);
    l.pairs = o; o += align256((size_t)2 * LT * mu_pair_slots(LT) * 8);
    l.mu = o; o += align256((size_t)r.L * r.L * 4);
    l.partial = o; o += align256((size_t)nbx * nby * 8);
    l.counter = o; o += 256;
    l.eta = o; o += 256;
    l.total = o;
    return l;
}

int bucket_for(mf_server_t s, int LT, int conn, bool sym) {
    for (size_t b = 0; b < s->bucket_lt.size(); ++b)
        if (s->bucket_lt[b] == LT && s->bucket_conn[b] == conn && s->bucket_sym[b] == (int)sym) return (int)b;
    if ((int)s->bucket_lt.size() >= kMaxBuckets) return -1;
    s->bucket_lt.push_back(LT);
    s->bucket_conn.push_back(conn);
    s->bucket_sym.push_back(sym ? 1 : 0);
    s->bucket_dirty.push_back(true);
    s->graph_stale = true;
    return (int)s->bucket_lt.size() - 1;
}

void bucket_rebuild(mf_server_t s, int b, const std::vector<ServeSlot> &hs) {
    (void)hs;
    ServeBucket &bk = s->h_buckets[b];
    int k = 0, acc = 0;
    for (int si = 0; si < s->max_slots; ++si) {
        const int t = s->slot_ticket[si];
        if (t == 0) continue;
        const Request &r = s->reqs.at((uint64_t)t);
        if (r.state != 1) continue;
        if (bucket_for(s, kernel_labels(r.L), r.conn, r.sym) != b) continue;
        int nbx, nby;
        grid_tiles(r.H, r.W, &nbx, &nby);
        bk.slots[k] = si;
        bk.prefix[k] = acc;
        acc += nbx * nby;
        ++k;
    }
    bk.count = k;
    bk.prefix[k] = acc;
    s->bucket_dirty[b] = true;
}

crf_status capture_graph(mf_server_t s) {
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    if (s->graph) {
        cudaGraphDestroy(s->graph);
        s->graph = nullptr;
    }
    SCK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    for (size_t b = 0; b < s->bucket_lt.size(); ++b) {
        const int grid = s->bucket_lt[b] >= 24 ? s->grid_large : s->grid_small;
        const cudaError_t e = launch_serve(s->bucket_lt[b], s->bucket_conn[b], s->bucket_sym[b] != 0, s->d_slots,
                                           s->d_buckets + b, s->d_res, grid, s->cap);
        if (e != cudaSuccess) {
            cudaGraph_t g;
            cudaStreamEndCapture(s->cap, &g);
            if (g) cudaGraphDestroy(g);
            return srv_cuda(s, e);
        }
    }
    SCK(cudaStreamEndCapture(s->cap, &s->graph));
    SCK(cudaGraphInstantiate(&s->exec, s->graph, 0));
    s->graph_stale = false;
    return CRF_OK;
}

crf_status ensure_staging(mf_server_t s, size_t floats) {
    if (floats <= s->staging_floats) return CRF_OK;
    if (s->staging) {
        SCK(cudaStreamSynchronize(s->st));
        cudaFree(s->staging);
        s->staging = nullptr;
    }
    SCK(cudaMalloc((void **)&s->staging, floats * sizeof(float)));
    s->staging_floats = floats;
    return CRF_OK;
}

// Upload and prepare one admitted request in its pool block and slot.
crf_status admit(mf_server_t s, Request &r, int si) {
    const SlotLayout l = layout_for(r);
    unsigned char *base = s->pool_base + r.off;
    const size_t N = (size_t)r.H * r.W;
    const int LP = storage_labels(r.L), LT = kernel_labels(r.L), nd = r.conn == 8 ? 4 : 2;
    crf_status rc = ensure_staging(s, std::max(N * r.L, N * nd));
    if (rc != CRF_OK) return rc;
    float *U = (float *)(base + l.U), *s0 = (float *)(base + l.s0), *s1 = (float *)(base + l.s1);
    float *w = (float *)(base + l.w), *mu = (float *)(base + l.mu), *eta = (float *)(base + l.eta);
    float2 *pairs = (float2 *)(base + l.pairs);
    SCK(cudaMemcpyAsync(s->staging, r.U.data(), N * r.L * sizeof(float), cudaMemcpyHostToDevice, s->st));
    SCK(launch_rows_to_padded(s->staging, U, (long long)N, r.L, LP, 0.f, s->st));
    SCK(launch_init_logq(U, s0, (long long)N, r.L, LP, s->st));
    SCK(cudaMemsetAsync(s1, 0, N * LP * sizeof(float), s->st));
    SCK(cudaMemcpyAsync(s->staging, r.w.data(), N * nd * sizeof(float), cudaMemcpyHostToDevice, s->st));
    SCK(launch_weights_to_pixel_major(s->staging, w, 1, nd, r.H, r.W, s->st));
    std::vector<float2> hp((size_t)2 * LT * mu_pair_slots(LT), make_float2(0.f, 0.f));
    build_mu_pairs_host(r.mu.data(), r.L, LT, hp.data());
    SCK(cudaMemcpyAsync(pairs, hp.data(), hp.size() * sizeof(float2), cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemcpyAsync(mu, r.mu.data(), (size_t)r.L * r.L * sizeof(float), cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemsetAsync(base + l.counter, 0, 256, s->st));
    if (r.p.eta > 0) {
        const float e = (float)r.p.eta;
        SCK(cudaMemcpyAsync(eta, &e, sizeof(float), cudaMemcpyHostToDevice, s->st));
    } else {
        SCK(launch_eta_bound(w, r.H, r.W, nd, mu, r.L, eta, s->d_scratch, s->st));
    }
    ServeSlot sl{};
    int nbx, nby;
    grid_tiles(r.H, r.W, &nbx, &nby);
    sl.U = U;
    sl.s[0] = s0;
    sl.s[1] = s1;
    sl.w = w;
    sl.mu_out = pairs;
    sl.mu_in = pairs + (size_t)LT * mu_pair_slots(LT);
    sl.partial = (double *)(base + l.partial);
    sl.counter = (unsigned *)(base + l.counter);
    sl.eta = eta;
    sl.L = r.L;
    sl.H = r.H;
    sl.W = r.W;
    sl.nbx = nbx;
    sl.nblk = nbx * nby;
    sl.max_iters = r.p.max_iters;
    sl.rel_tol = r.p.rel_tol;
    sl.it = 0;
    sl.active = r.p.max_iters > 0 ? 1 : 0;
    sl.F_prev = 0.0;
    s->h_res[si].done = 0;
    s->h_res[si].iters = 0;
    s->h_res[si].F = 0.0;
    SCK(cudaMemcpyAsync(s->d_slots + si, &sl, sizeof(sl), cudaMemcpyHostToDevice, s->st));
    SCK(cudaStreamSynchronize(s->st));   // host staging vectors are pageable
    if (!sl.active) {
        s->h_res[si].done = 1;
    }
    return CRF_OK;
}

// Copy q of a retired slot out, free its slot and pool block.
crf_status retire(mf_server_t s, Request &r, int si) {
    const SlotLayout l = layout_for(r);
    unsigned char *base = s->pool_base + r.off;
    const size_t N = (size_t)r.H * r.W;
    const int LP = storage_labels(r.L);
    const ServeResult res = s->h_res[si];
    const float *final_s = (const float *)(base + ((res.iters & 1) ? l.s1 : l.s0));
    if (r.q_out) {
        crf_status rc = ensure_staging(s, N * r.L);
        if (rc != CRF_OK) return rc;
        SCK(launch_padded_to_rows(final_s, s->staging, (long long)N, r.L, LP, CONV_EXP, s->st));
        SCK(cudaMemcpyAsync(r.q_out, s->staging, N * r.L * sizeof(float), cudaMemcpyDeviceToHost, s->st));
        SCK(cudaStreamSynchronize(s->st));
    }
    r.F = res.F;
    r.iters = res.iters;
    r.state = 2;
    r.U.clear();
    r.U.shrink_to_fit();
    r.w.clear();
    r.w.shrink_to_fit();
    s->pool->release(r.off, r.bytes);
    s->slot_ticket[si] = 0;
    r.slot = -1;
    return CRF_OK;
}

}  // namespace

// ---------------------------------------------------------------- eta bound --

namespace proxmf {

namespace {

// scratch[0] = max over pixels of the weighted degree (edges leaving plus entering)
__global__ void max_degree_kernel(const float *__restrict__ w, int N, int nd, int W, unsigned *out_bits) {
    float best = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int y = p / W, x = p - y * W;
        float d = 0.f;
        for (int k = 0; k < nd; ++k) d += w[(size_t)p * nd + k];
        // entering: right from (y,x-1), down from (y-1,x), dr from (y-1,x-1), dl from (y-1,x+1)
        if (x > 0) d += w[(size_t)(p - 1) * nd + 0];
        if (y > 0) d += w[(size_t)(p - W) * nd + 1];
        if (nd == 4) {
            if (x > 0 && y > 0) d += w[(size_t)(p - W - 1) * nd + 2];
            if (x + 1 < W && y > 0) d += w[(size_t)(p - W + 1) * nd + 3];
        }
        best = fmaxf(best, d);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(best));   // non-negative floats order as uints
}

__global__ void eta_bound_finalize_kernel(const unsigned *deg_bits, const double *nu, float *eta) {
    const double D = (double)__uint_as_float(*deg_bits);
    const double lam = D * fmax(fabs(nu[0]), fabs(nu[1]));
    *eta = (float)(1.0 / (1.0 + lam));
}

}  // namespace

cudaError_t launch_eta_bound(const float *w, int H, int W, int nd, const float *mu, int L, float *eta,
                             double *scratch, cudaStream_t st) {
    // scratch: [0..1] extreme eigenvalues of C mu C, [2] degree bits
    unsigned *deg = reinterpret_cast<unsigned *>(scratch + 2);
    cudaError_t e = cudaMemsetAsync(deg, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int N = H * W;
    max_degree_kernel<<<std::min((N + 255) / 256, 1024), 256, 0, st>>>(w, N, nd, W, deg);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_mu_tilde_extremes(mu, L, scratch, st);
    if (e != cudaSuccess) return e;
    eta_bound_finalize_kernel<<<1, 1, 0, st>>>(deg, scratch, eta);
    return cudaGetLastError();
}

}  // namespace proxmf

// ---------------------------------------------------------------- C ABI --

extern "C" {

crf_status mf_server_create(int64_t budget_bytes, int32_t max_slots, void *stream, mf_server_t *out) {
    PROXMF_RANGE("mf_server_create");
    if (!out) return CRF_E_INVALID;
    *out = nullptr;
    if (budget_bytes <= 0 || max_slots < 1 || max_slots > kMaxServeSlots) return CRF_E_INVALID;
    mf_server_t s = new (std::nothrow) mf_server_s();
    if (!s) return CRF_E_OOM;
    s->st = (cudaStream_t)stream;
    s->budget = (size_t)budget_bytes;
    s->max_slots = max_slots;
    s->slot_ticket.assign(max_slots, 0);
    s->h_buckets.resize(kMaxBuckets);
    for (auto &b : s->h_buckets) {
        b.count = 0;
        b.prefix[0] = 0;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->grid_small = 2 * (sms > 0 ? sms : 148);
    s->grid_large = sms > 0 ? sms : 148;
    bool ok = cudaMalloc((void **)&s->pool_base, s->budget) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->d_slots, sizeof(ServeSlot) * max_slots) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->d_buckets, sizeof(ServeBucket) * kMaxBuckets) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->d_scratch, 8 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&s->h_res, sizeof(ServeResult) * max_slots, cudaHostAllocMapped) == cudaSuccess;
    ok = ok && cudaHostGetDevicePointer((void **)&s->d_res, s->h_res, 0) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(s->d_slots, 0, sizeof(ServeSlot) * max_slots, s->st) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(s->d_buckets, 0, sizeof(ServeBucket) * kMaxBuckets, s->st) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(s->st) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        mf_server_destroy(s);
        return CRF_E_OOM;
    }
    std::memset(s->h_res, 0, sizeof(ServeResult) * max_slots);
    s->pool = new Pool(s->budget);
    *out = s;
    return CRF_OK;
}

crf_status mf_server_destroy(mf_server_t s) {
    PROXMF_RANGE("mf_server_destroy");
    if (!s) return CRF_OK;
    cudaStreamSynchronize(s->st);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->pool_base) cudaFree(s->pool_base);
    if (s->d_slots) cudaFree(s->d_slots);
    if (s->d_buckets) cudaFree(s->d_buckets);
    if (s->d_scratch) cudaFree(s->d_scratch);
    if (s->staging) cudaFree(s->staging);
    if (s->h_res) cudaFreeHost(s->h_res);
    delete s->pool;
    delete s;
    return CRF_OK;
}

crf_status mf_server_submit(mf_server_t s, const crf_desc *d, const float *U, const float *mu, const float *w,
                            const mf_params *p, float *q_out, uint64_t *ticket) {
    PROXMF_RANGE("mf_server_submit");
    if (!s || !d || !U || !mu || !w || !p || !ticket) return CRF_E_INVALID;
    if (s->broken) return CRF_E_STATE;
    if (d->topology != CRF_GRID4 && d->topology != CRF_GRID8) return CRF_E_INVALID;
    if (d->batch != 1 || d->precision != CRF_FP32) return CRF_E_INVALID;
    if (d->n_labels < 1 || d->n_labels > kMaxLabels || d->height < 1 || d->width < 1) return CRF_E_INVALID;
    if (d->height > 65535ll * GY || d->width > (1 << 20)) return CRF_E_INVALID;
    if (p->max_iters < 0 || p->rel_tol < 0 || !(p->eta <= 1.0)) return CRF_E_INVALID;
    if (p->rule != MF_RULE_FIXED) return CRF_E_UNSUPPORTED;   // the server runs the fixed-step rule
    Request r;
    r.ticket = s->next_ticket++;
    r.H = (int)d->height;
    r.W = (int)d->width;
    r.L = d->n_labels;
    r.conn = d->topology == CRF_GRID8 ? 8 : 4;
    const size_t N = (size_t)r.H * r.W, nd = r.conn == 8 ? 4 : 2;
    r.U.assign(U, U + N * r.L);
    r.mu.assign(mu, mu + (size_t)r.L * r.L);
    r.w.assign(w, w + N * nd);
    for (float v : r.mu)
        if (!std::isfinite(v)) return CRF_E_INVALID;
    for (int i = 0; i < r.L; ++i)
        for (int k = i + 1; k < r.L; ++k)
            if (r.mu[i * r.L + k] != r.mu[k * r.L + i]) r.sym = false;
    if (!r.sym && p->eta <= 0) return CRF_E_INVALID;   // the step bound assumes a symmetric mu
    r.p = *p;
    r.q_out = q_out;
    r.bytes = layout_for(r).total;
    if (r.bytes > s->budget) return CRF_E_OOM;
    *ticket = r.ticket;
    s->queue.push_back(r.ticket);
    s->reqs.emplace(r.ticket, std::move(r));
    return CRF_OK;
}

crf_status mf_server_step(mf_server_t s, int32_t iters, int32_t *in_flight, int32_t *queued) {
    PROXMF_RANGE("mf_server_step");
    if (!s || iters < 0) return CRF_E_INVALID;
    if (s->broken) return CRF_E_STATE;
    crf_status rc;
    // 1. retire finished slots
    std::vector<int> touched;
    for (int si = 0; si < s->max_slots; ++si) {
        const uint64_t t = (uint64_t)s->slot_ticket[si];
        if (!t) continue;
        if (*(volatile int *)&s->h_res[si].done) {
            Request &r = s->reqs.at(t);
            touched.push_back(bucket_for(s, kernel_labels(r.L), r.conn, r.sym));
            rc = retire(s, r, si);
            if (rc != CRF_OK) return rc;
        }
    }
    // 2. admit queued requests in arrival order while a slot and memory are free
    while (!s->queue.empty()) {
        Request &r = s->reqs.at(s->queue.front());
        int si = -1;
        for (int k = 0; k < s->max_slots; ++k)
            if (!s->slot_ticket[k]) {
                si = k;
                break;
            }
        size_t off;
        if (si < 0 || !s->pool->alloc(r.bytes, &off)) break;
        r.off = off;
        r.slot = si;
        r.state = 1;
        s->slot_ticket[si] = (int)r.ticket;
        s->queue.pop_front();
        rc = admit(s, r, si);
        if (rc != CRF_OK) return rc;
        touched.push_back(bucket_for(s, kernel_labels(r.L), r.conn, r.sym));
    }
    for (int b : touched)
        if (b >= 0) bucket_rebuild(s, b, {});
    bool uploaded = false;
    for (size_t b = 0; b < s->bucket_lt.size(); ++b)
        if (s->bucket_dirty[b]) {
            SCK(cudaMemcpyAsync(s->d_buckets + b, &s->h_buckets[b], sizeof(ServeBucket), cudaMemcpyHostToDevice,
                                s->st));
            s->bucket_dirty[b] = false;
            uploaded = true;
        }
    if (uploaded) SCK(cudaStreamSynchronize(s->st));   // bucket headers come from pageable host memory
    if (s->graph_stale && !s->bucket_lt.empty()) {
        rc = capture_graph(s);
        if (rc != CRF_OK) return rc;
    }
    // 3. iterate every in-flight request
    int running = 0;
    for (int si = 0; si < s->max_slots; ++si)
        if (s->slot_ticket[si]) ++running;
    if (running && s->exec)
        for (int i = 0; i < iters; ++i) SCK(cudaGraphLaunch(s->exec, s->st));
    if (in_flight) *in_flight = running;
    if (queued) *queued = (int)s->queue.size();
    return CRF_OK;
}

crf_status mf_server_poll(mf_server_t s, uint64_t ticket, int32_t *state, double *F, int32_t *iters) {
    if (!s) return CRF_E_INVALID;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return CRF_E_INVALID;
    const Request &r = it->second;
    if (state) *state = r.state;
    if (F) *F = r.F;
    if (iters) *iters = r.iters;
    return CRF_OK;
}

crf_status mf_server_sync(mf_server_t s) {
    PROXMF_RANGE("mf_server_sync");
    if (!s) return CRF_E_INVALID;
    if (s->broken) return CRF_E_STATE;
    SCK(cudaStreamSynchronize(s->st));
    return CRF_OK;
}

}  // extern "C"
