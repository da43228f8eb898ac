// serve.cu -- host side of the serving loop (continuous batching).
//
// A server owns one device memory pool of a fixed budget.  Requests (single
// grid CRFs of any size, label count and connectivity) are copied on submit
// and queued; each step the server
//   1. retires the slots whose stopping rule fired (flags in host-mapped
//      memory): queues the copy of q out and returns the slot and its pool
//      memory (later work on the stream is ordered after the copy);
//   2. admits queued requests in arrival order while a slot and pool memory
//      (first-fit) are free: uploads and converts the data, builds q^0 and
//      the step size on the device, and enters the slot in the tile table;
//   3. replays a CUDA graph holding one persistent launch over the tiles of
//      every running request (serve.cuh), once per requested iteration.
// Requests therefore join and leave between iterations while the others keep
// running, and every request's arithmetic is that of a solve on its own.
//
// No step waits for the device except to recycle host staging memory: the
// uploads of an admission and the download of a result go through a ring of
// page-locked host memory (cudaMemcpyAsync from pageable memory would
// synchronise the stream, and with it every admission, with the iterations
// already queued); an event per block says when the ring may reuse it and
// when a result has reached its q_out.
#include <algorithm>
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

// Ring of page-locked host memory: blocks are handed out in FIFO order and
// come back when the event recorded after their last copy has completed.
class PinnedRing {
public:
    bool init(size_t size) {
        size_ = size;
        return cudaHostAlloc((void **)&base_, size, cudaHostAllocDefault) == cudaSuccess;
    }
    ~PinnedRing() {
        for (auto &b : live_) cudaEventDestroy(b.ev);
        for (cudaEvent_t e : spare_) cudaEventDestroy(e);
        if (base_) cudaFreeHost(base_);
    }
    size_t size() const { return size_; }
    // A block of `bytes` (256-byte aligned), waiting for the oldest blocks to
    // be released if the ring is full.  nullptr if it can never fit.
    unsigned char *acquire(size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        if (bytes > size_) return nullptr;
        for (;;) {
            reclaim(false);
            size_t off;
            if (fits(bytes, &off)) {
                pending_off_ = off;
                pending_bytes_ = bytes;
                return base_ + off;
            }
            if (live_.empty()) return nullptr;
            cudaEventSynchronize(live_.front().ev);
        }
    }
    // Seal the block handed out last: its copies were issued on st.
    cudaError_t seal(cudaStream_t st) {
        cudaEvent_t e = nullptr;
        if (!spare_.empty()) {
            e = spare_.back();
            spare_.pop_back();
        } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            return cudaErrorMemoryAllocation;
        }
        const cudaError_t r = cudaEventRecord(e, st);
        live_.push_back({pending_off_, pending_bytes_, e});
        return r;
    }
    cudaEvent_t last_event() const { return live_.back().ev; }
    void reclaim(bool all) {
        while (!live_.empty() && (all || cudaEventQuery(live_.front().ev) == cudaSuccess)) {
            if (all) cudaEventSynchronize(live_.front().ev);
            spare_.push_back(live_.front().ev);
            live_.pop_front();
        }
        (void)cudaGetLastError();   // a query of an unfinished event is not an error
    }

private:
    bool fits(size_t bytes, size_t *off) const {
        if (live_.empty()) {
            *off = 0;
            return true;
        }
        const size_t start = live_.front().off, end = live_.back().off + live_.back().bytes;
        if (end > start || (end == start && live_.size() == 0)) {
            if (size_ - end >= bytes) {
                *off = end;
                return true;
            }
            if (start >= bytes) {
                *off = 0;
                return true;
            }
            return false;
        }
        if (start - end >= bytes) {
            *off = end;
            return true;
        }
        return false;
    }
    struct Block {
        size_t off, bytes;
        cudaEvent_t ev;
    };
    unsigned char *base_ = nullptr;
    size_t size_ = 0;
    std::deque<Block> live_;
    std::vector<cudaEvent_t> spare_;
    size_t pending_off_ = 0, pending_bytes_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    int H = 0, W = 0, L = 0, conn = 4;
    std::vector<float> U, mu, w;
    mf_params p{};
    float *q_out = nullptr;
    int state = 0;               // 0 queued, 1 running, 3 result on its way to q_out, 2 done
    int slot = -1;
    size_t off = 0, bytes = 0;
    double F = 0.0;
    int iters = 0;
    bool sym = true;
    const unsigned char *q_host = nullptr;   // pinned copy of q while state 3
    cudaEvent_t q_ready = nullptr;
};

}  // namespace

struct mf_server_s {
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;
    size_t budget = 0;
    int max_slots = 0;
    unsigned char *pool_base = nullptr;
    Pool *pool = nullptr;
    PinnedRing ring;
    ServeSlot *d_slots = nullptr;
    ServeTable *d_table = nullptr;
    ServeTable *h_table[2] = {nullptr, nullptr};   // page-locked, alternating uploads
    cudaEvent_t table_ev[2] = {nullptr, nullptr};
    int table_buf = 0;
    bool table_dirty = false;
    ServeResult *h_res = nullptr, *d_res = nullptr;   // host-mapped
    double *d_scratch = nullptr;
    float *staging = nullptr;
    size_t staging_floats = 0;
    std::vector<int> slot_ticket;
    std::deque<uint64_t> queue;
    std::deque<uint64_t> outgoing;   // results in flight to q_out, in order
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_smem = 0;           // dynamic shared memory the graph's launch was recorded with
    bool broken = false;
    int sms = 0;
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

// Host bytes an admission stages: U and w rows, mu pairs, mu, eta, the slot.
size_t admit_staging_bytes(const Request &r) {
    const size_t N = (size_t)r.H * r.W;
    const int LT = kernel_labels(r.L), nd = r.conn == 8 ? 4 : 2;
    return align256(N * r.L * 4) + align256(N * nd * 4) + align256((size_t)2 * LT * mu_pair_slots(LT) * 8) +
           align256((size_t)r.L * r.L * 4) + 256 + align256(sizeof(ServeSlot));
}

// The tile table over every running slot (slot order), into the next
// page-locked buffer and up to the device.
crf_status upload_table(mf_server_t s) {
    const int k = s->table_buf;
    SCK(cudaEventSynchronize(s->table_ev[k]));   // the previous upload from this buffer is done
    ServeTable &t = *s->h_table[k];
    int n = 0, acc = 0;
    for (int si = 0; si < s->max_slots; ++si) {
        const uint64_t tk = (uint64_t)s->slot_ticket[si];
        if (!tk) continue;
        const Request &r = s->reqs.at(tk);
        if (r.state != 1) continue;
        int nbx, nby;
        grid_tiles(r.H, r.W, &nbx, &nby);
        t.slots[n] = si;
        t.prefix[n] = acc;
        acc += nbx * nby;
        ++n;
    }
    t.count = n;
    t.prefix[n] = acc;
    const size_t bytes = offsetof(ServeTable, prefix) + (size_t)(n + 1) * sizeof(int);
    SCK(cudaMemcpyAsync(s->d_table, &t, bytes, cudaMemcpyHostToDevice, s->st));
    SCK(cudaEventRecord(s->table_ev[k], s->st));
    s->table_buf ^= 1;
    s->table_dirty = false;
    return CRF_OK;
}

// Dynamic shared memory of the serving launch: the largest class running.
size_t needed_smem(mf_server_t s) {
    size_t m = 0;
    for (int si = 0; si < s->max_slots; ++si) {
        const uint64_t tk = (uint64_t)s->slot_ticket[si];
        if (!tk) continue;
        const Request &r = s->reqs.at(tk);
        if (r.state == 1) m = std::max(m, serve_tile_smem(kernel_labels(r.L)));
    }
    return m;
}

crf_status capture_graph(mf_server_t s, size_t smem) {
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    if (s->graph) {
        cudaGraphDestroy(s->graph);
        s->graph = nullptr;
    }
    // persistent grid: every SM, as many blocks as fit with this shared memory
    int per_sm = 0;
    SCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_step_kernel, GT, smem));
    const int grid = s->sms * std::max(per_sm, 1);
    SCK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    serve_step_kernel<<<grid, dim3(GX, GY, 1), smem, s->cap>>>(s->d_slots, s->d_table, s->d_res);
    const cudaError_t e = cudaGetLastError();
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return srv_cuda(s, e != cudaSuccess ? e : e2);
    }
    s->graph = g;
    SCK(cudaGraphInstantiate(&s->exec, s->graph, 0));
    s->graph_smem = smem;
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
    // everything the admission uploads, in one page-locked block
    unsigned char *hb = s->ring.acquire(admit_staging_bytes(r));
    if (!hb) return CRF_E_OOM;
    const size_t npairs = (size_t)2 * LT * mu_pair_slots(LT);
    size_t o = 0;
    float *hU = (float *)(hb + o); o += align256(N * r.L * 4);
    float *hw = (float *)(hb + o); o += align256(N * nd * 4);
    float2 *hp = (float2 *)(hb + o); o += align256(npairs * 8);
    float *hmu = (float *)(hb + o); o += align256((size_t)r.L * r.L * 4);
    float *heta = (float *)(hb + o); o += 256;
    ServeSlot *hsl = (ServeSlot *)(hb + o);
    std::memcpy(hU, r.U.data(), N * r.L * sizeof(float));
    std::memcpy(hw, r.w.data(), N * nd * sizeof(float));
    for (size_t i = 0; i < npairs; ++i) hp[i] = make_float2(0.f, 0.f);
    build_mu_pairs_host(r.mu.data(), r.L, LT, hp);
    std::memcpy(hmu, r.mu.data(), (size_t)r.L * r.L * sizeof(float));
    *heta = (float)r.p.eta;

    SCK(cudaMemcpyAsync(s->staging, hU, N * r.L * sizeof(float), cudaMemcpyHostToDevice, s->st));
    SCK(launch_rows_to_padded(s->staging, U, (long long)N, r.L, LP, 0.f, s->st));
    SCK(launch_init_logq(U, s0, (long long)N, r.L, LP, s->st));
    SCK(cudaMemsetAsync(s1, 0, N * LP * sizeof(float), s->st));
    SCK(cudaMemcpyAsync(s->staging, hw, N * nd * sizeof(float), cudaMemcpyHostToDevice, s->st));
    SCK(launch_weights_to_pixel_major(s->staging, w, 1, nd, r.H, r.W, s->st));
    SCK(cudaMemcpyAsync(pairs, hp, npairs * sizeof(float2), cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemcpyAsync(mu, hmu, (size_t)r.L * r.L * sizeof(float), cudaMemcpyHostToDevice, s->st));
    SCK(cudaMemsetAsync(base + l.counter, 0, 256, s->st));
    if (r.p.eta > 0)
        SCK(cudaMemcpyAsync(eta, heta, sizeof(float), cudaMemcpyHostToDevice, s->st));
    else
        SCK(launch_eta_bound(w, r.H, r.W, nd, mu, r.L, eta, s->d_scratch, s->st));
    int nbx, nby;
    grid_tiles(r.H, r.W, &nbx, &nby);
    ServeSlot &sl = *hsl;
    sl = ServeSlot{};
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
    sl.LT = LT;
    sl.H = r.H;
    sl.W = r.W;
    sl.nbx = nbx;
    sl.nblk = nbx * nby;
    sl.conn = r.conn;
    sl.sym = r.sym ? 1 : 0;
    sl.max_iters = r.p.max_iters;
    sl.rel_tol = r.p.rel_tol;
    sl.it = 0;
    sl.active = r.p.max_iters > 0 ? 1 : 0;
    sl.F_prev = 0.0;
    s->h_res[si].done = sl.active ? 0 : 1;
    s->h_res[si].iters = 0;
    s->h_res[si].F = 0.0;
    SCK(cudaMemcpyAsync(s->d_slots + si, hsl, sizeof(ServeSlot), cudaMemcpyHostToDevice, s->st));
    SCK(s->ring.seal(s->st));
    return CRF_OK;
}

// Queue the copy of q of a retired slot and return its slot and pool block
// (the stream orders every later use of that memory after the copy).
crf_status retire(mf_server_t s, Request &r, int si) {
    const SlotLayout l = layout_for(r);
    unsigned char *base = s->pool_base + r.off;
    const size_t N = (size_t)r.H * r.W;
    const int LP = storage_labels(r.L);
    const ServeResult res = s->h_res[si];
    const float *final_s = (const float *)(base + ((res.iters & 1) ? l.s1 : l.s0));
    r.F = res.F;
    r.iters = res.iters;
    if (r.q_out) {
        crf_status rc = ensure_staging(s, N * r.L);
        if (rc != CRF_OK) return rc;
        unsigned char *hb = s->ring.acquire(N * r.L * sizeof(float));
        if (!hb) return CRF_E_OOM;
        SCK(launch_padded_to_rows(final_s, s->staging, (long long)N, r.L, LP, CONV_EXP, s->st));
        SCK(cudaMemcpyAsync(hb, s->staging, N * r.L * sizeof(float), cudaMemcpyDeviceToHost, s->st));
        SCK(s->ring.seal(s->st));
        r.q_host = hb;
        r.q_ready = s->ring.last_event();
        r.state = 3;
        s->outgoing.push_back(r.ticket);
    } else {
        r.state = 2;
    }
    r.U.clear();
    r.U.shrink_to_fit();
    r.w.clear();
    r.w.shrink_to_fit();
    s->pool->release(r.off, r.bytes);
    s->slot_ticket[si] = 0;
    r.slot = -1;
    s->table_dirty = true;
    return CRF_OK;
}

// Results whose copy has landed reach q_out (in retirement order).
void deliver(mf_server_t s, bool wait) {
    while (!s->outgoing.empty()) {
        Request &r = s->reqs.at(s->outgoing.front());
        if (wait)
            cudaEventSynchronize(r.q_ready);
        else if (cudaEventQuery(r.q_ready) != cudaSuccess)
            break;
        std::memcpy(r.q_out, r.q_host, (size_t)r.H * r.W * r.L * sizeof(float));
        r.q_host = nullptr;
        r.q_ready = nullptr;
        r.state = 2;
        s->outgoing.pop_front();
    }
    (void)cudaGetLastError();
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
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->sms = sms > 0 ? sms : 148;
    bool ok = cudaMalloc((void **)&s->pool_base, s->budget) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->d_slots, sizeof(ServeSlot) * max_slots) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->d_table, sizeof(ServeTable)) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->d_scratch, 8 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&s->h_res, sizeof(ServeResult) * max_slots, cudaHostAllocMapped) == cudaSuccess;
    ok = ok && cudaHostGetDevicePointer((void **)&s->d_res, s->h_res, 0) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) {
        ok = cudaHostAlloc((void **)&s->h_table[k], sizeof(ServeTable), cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&s->table_ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    // page-locked staging: room for the largest requests several times over
    ok = ok && s->ring.init((size_t)256 << 20);
    ok = ok && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) == cudaSuccess;
    static SmemOptIn optin;   // up to the largest class's tile memory, once per device
    ok = ok && smem_optin(optin, serve_step_kernel, serve_tile_smem(kMaxLabels)) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(s->d_slots, 0, sizeof(ServeSlot) * max_slots, s->st) == cudaSuccess;
    if (ok) ok = cudaMemsetAsync(s->d_table, 0, sizeof(ServeTable), s->st) == cudaSuccess;
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
    s->ring.reclaim(true);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->pool_base) cudaFree(s->pool_base);
    if (s->d_slots) cudaFree(s->d_slots);
    if (s->d_table) cudaFree(s->d_table);
    if (s->d_scratch) cudaFree(s->d_scratch);
    if (s->staging) cudaFree(s->staging);
    if (s->h_res) cudaFreeHost(s->h_res);
    for (int k = 0; k < 2; ++k) {
        if (s->h_table[k]) cudaFreeHost(s->h_table[k]);
        if (s->table_ev[k]) cudaEventDestroy(s->table_ev[k]);
    }
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
    if (admit_staging_bytes(r) > s->ring.size() || N * r.L * sizeof(float) > s->ring.size()) return CRF_E_OOM;
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
    deliver(s, false);
    // 1. retire finished slots
    for (int si = 0; si < s->max_slots; ++si) {
        const uint64_t t = (uint64_t)s->slot_ticket[si];
        if (!t) continue;
        Request &r = s->reqs.at(t);
        if (r.state == 1 && *(volatile int *)&s->h_res[si].done) {
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
        s->table_dirty = true;
    }
    if (s->table_dirty) {
        rc = upload_table(s);
        if (rc != CRF_OK) return rc;
    }
    // 3. iterate every in-flight request: one launch per iteration
    const size_t smem = needed_smem(s);
    int running = 0;
    for (int si = 0; si < s->max_slots; ++si)
        if (s->slot_ticket[si] && s->reqs.at((uint64_t)s->slot_ticket[si]).state == 1) ++running;
    if (running) {
        if (!s->exec || smem != s->graph_smem) {
            rc = capture_graph(s, smem);
            if (rc != CRF_OK) return rc;
        }
        for (int i = 0; i < iters; ++i) SCK(cudaGraphLaunch(s->exec, s->st));
    }
    if (in_flight) *in_flight = running;
    if (queued) *queued = (int)s->queue.size();
    return CRF_OK;
}

crf_status mf_server_poll(mf_server_t s, uint64_t ticket, int32_t *state, double *F, int32_t *iters) {
    if (!s) return CRF_E_INVALID;
    deliver(s, false);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return CRF_E_INVALID;
    const Request &r = it->second;
    if (state) *state = r.state == 3 ? 1 : r.state;
    if (F) *F = r.F;
    if (iters) *iters = r.iters;
    return CRF_OK;
}

crf_status mf_server_sync(mf_server_t s) {
    PROXMF_RANGE("mf_server_sync");
    if (!s) return CRF_E_INVALID;
    if (s->broken) return CRF_E_STATE;
    SCK(cudaStreamSynchronize(s->st));
    deliver(s, true);
    return CRF_OK;
}

}  // extern "C"
