// dense_tc.cu -- tensor-core (tcgen05) form of the fully connected step.
//
// The message S = K Q of the dense model is an (N x N) by (N x L) product:
// here K and Q are BF16 and the product runs on the 5th-generation tensor
// cores with FP32 accumulation in tensor memory (TMEM); the proximal update,
// renormalisation and free energy stay in FP32 (dense_common.cuh).
//
// Per CTA: one tile of M = 128 rows of K, all 32 label columns (L padded),
// and half of the k range (split-K 2, so N = 9216 gives 144 CTAs for the 152
// SMs; a four-way split with two CTAs per SM measured slower, its serial
// epilogue tail growing more than the streaming overlap gained).  Warp 0
// lane 0 fills a 10-stage ring guarded by mbarriers: each stage is one
// 16 KiB bulk copy of a 128 x 64 block of K, which the library stores
// pre-tiled and already in the 128-byte-swizzled K-major layout (so a stage
// is one contiguous read from HBM instead of 128 rows of 128 bytes), and a
// TMA load of the 32 x 64 tile of Q^T (128-byte swizzle); warp 1 lane 0
// issues tcgen05.mma (M=128, N=32, K=16, kind::f16) into a 32-column TMEM
// accumulator and releases each stage with tcgen05.commit.  The four warps
// then read the accumulator rows with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31).  The k ranges of a tile
// meet in global memory: the last CTA to finish sums the partials in range
// order (so the result does not depend on which one finishes last) and runs
// the row epilogue for the tile's 128 rows.
//
// Every wait is bounded by a clock budget; on expiry the kernel records
// CRF_E_TIMEOUT, drains its own copies in flight (bounded), frees its TMEM
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>

#include "dense_common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace proxmf {

namespace {

constexpr int kTM = 128;                 // rows per tile (MMA M)
constexpr int kTN = 32;                  // label columns (MMA N)
constexpr int kTK = 64;                  // k per stage (128 bytes of BF16)
constexpr int kStages = 10;
constexpr int kStageA = kTM * kTK * 2;   // 16 KiB
constexpr int kStageB = kTN * kTK * 2;   // 4 KiB
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kThreads = 128;
constexpr int kSplit = 2;                // k ranges per tile

using namespace tc;

// Instruction descriptor: M = 128, N = 32.
constexpr uint32_t kIdesc = idesc_bf16(kTM, kTN);

struct DenseTcArgs {
    const uint8_t *K16;      // [B][nchunk][ntiles] blocks of 128 x 64 BF16, 128-byte swizzled (dense.cu)
    const float *s_in;
    const float *U;
    float *s_out;
    float *q_out;
    __nv_bfloat16 *qt_out;
    const float *eta;
    const float *mu;
    const float *featsT;     // on-the-fly form: [B][nchunk][6][64] (dense_fly_features), else null
    float *split_part;       // [B][ntiles][kSplit][128][32]
    unsigned *tile_count;    // [B][ntiles]
    double *partial;         // [B][ntiles]
    unsigned *counter;       // [B]
    double *f_trace, *f_cur;
    int *done, *status;
    int N, Np, L, ntiles, nchunk;
    int t, trace_cap, update;
    double rel_tol;
    int B, defer, prev_pending;   // deferred free energy (DenseStepLaunch): slots of [B][ntiles]
};

// Sum of the n row-tile partials of one instance by the whole block: thread
// k takes k, k + kThreads, ...; shuffle-down trees; warps in order (the order
// of the ticket form's last-tile sum, so F is the same bit for bit).
template <int NT>
__device__ __forceinline__ double dense_sum_partials(const double *p, int n, double *red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc = 0.0;
    for (int k = tid; k < n; k += NT) acc += __ldcg(p + k);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    double F = 0.0;
    for (int k = 0; k < NT / 32; ++k) F += red[k];
    __syncthreads();   // red is reused
    return F;
}

// F of step t_prev from its deferred partials: trace entry and F_cur (by the
// writer block) and the stopping rule, evaluated identically by every block
// that asks.  True when instance b stops after step t_prev.
template <int NT>
__device__ __forceinline__ bool dense_deferred_f(const DenseTcArgs &a, int b, int t_prev, bool writer,
                                                 double *red) {
    const double F =
        dense_sum_partials<NT>(a.partial + (size_t)(t_prev & 1) * a.B * a.ntiles + (size_t)b * a.ntiles, a.ntiles, red);
    bool stop = false;
    if (a.done != nullptr && a.rel_tol > 0.0 && t_prev > 0 && t_prev - 1 < a.trace_cap) {
        const double Fp = a.f_trace[(size_t)b * a.trace_cap + t_prev - 1];
        stop = fabs(F - Fp) <= a.rel_tol * fabs(F);
    }
    if (writer && threadIdx.x == 0) {
        a.f_cur[b] = F;
        if (!isfinite(F)) atomicExch(a.status, -6);
        if (t_prev < a.trace_cap) a.f_trace[(size_t)b * a.trace_cap + t_prev] = F;
        if (stop) a.done[b] = t_prev + 1;
    }
    return stop;
}

__global__ void __launch_bounds__(kThreads) dense_f_flush_kernel(const __grid_constant__ DenseTcArgs a) {
    __shared__ double red[kThreads / 32];
    const int b = blockIdx.x;
    if (a.done != nullptr && a.done[b] != 0) return;   // the step copied a stopped instance: no partials
    dense_deferred_f<kThreads>(a, b, a.t, true, red);
}

// The tile's rows after the product: the k ranges of a tile meet in global
// memory (the last CTA to finish sums them in range order), then the row
// epilogue of the tile's 128 rows and the tile's free-energy partial (kept for
// the next step, or summed behind a ticket).  NT threads; the first kTM own a
// row, the others only join the block barriers.
template <int LP, int NT>
__device__ __forceinline__ void dense_tc_tail(const DenseTcArgs &a, float (&S)[32], const float *mus, double *red,
                                              int &is_second, int &is_last, int tile, int split, int b,
                                              int nsplit) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = a.N, L = a.L;
    const int row0 = tile * kTM;
    const int r = tid;                // row within the tile (threads >= kTM only join the barriers)
    const bool has_row = tid < kTM;
    const size_t tile_id = (size_t)b * a.ntiles + tile;
    if (nsplit > 1) {
        float *mine = a.split_part + ((tile_id * kSplit + split) * kTM + r) * 32;
#pragma unroll
        for (int i = 0; i < 32 && has_row; i += 4)
            *reinterpret_cast<float4 *>(mine + i) = make_float4(S[i], S[i + 1], S[i + 2], S[i + 3]);
        __threadfence();
        __syncthreads();
        if (tid == 0) is_second = atomicAdd(a.tile_count + tile_id, 1u) == (unsigned)(nsplit - 1);
        __syncthreads();
        if (!is_second) return;
        __threadfence();
        // the last of the k ranges sums all partials in split order
#pragma unroll
        for (int i = 0; i < 32; ++i) S[i] = 0.f;
        for (int sp = 0; sp < nsplit && has_row; ++sp) {
            const float4 *part = reinterpret_cast<const float4 *>(a.split_part + ((tile_id * kSplit + sp) * kTM + r) * 32);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 v = __ldcg(part + i);
                S[4 * i] += v.x;
                S[4 * i + 1] += v.y;
                S[4 * i + 2] += v.z;
                S[4 * i + 3] += v.w;
            }
        }
        if (tid == 0) a.tile_count[tile_id] = 0u;
    }

    // row epilogue on the tile's rows
    float f = 0.f;
    const int i = row0 + r;
    if (has_row && i < N) {
        const size_t o = ((size_t)b * N + i) * LP;
        f = dense_row_update<LP>(S, mus, L, a.eta[b], a.s_in + o, a.U + o, a.s_out + o, a.q_out + o,
                                 a.qt_out ? a.qt_out + (size_t)b * 32 * a.Np + i : nullptr, (size_t)a.Np,
                                 a.update != 0);
    }
    double fd = (double)f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) fd += __shfl_down_sync(0xffffffffu, fd, off);
    if (lane == 0) red[warp] = fd;
    __syncthreads();
    if (a.defer) {
        // the next step (or the flush kernel) sums this slot
        if (tid == 0) {
            double bs = 0.0;
            for (int k = 0; k < NT / 32; ++k) bs += red[k];
            a.partial[(size_t)(a.t & 1) * a.B * a.ntiles + (size_t)b * a.ntiles + tile] = bs;
        }
        return;
    }
    if (tid == 0) {
        double bs = 0.0;
        for (int k = 0; k < NT / 32; ++k) bs += red[k];
        a.partial[(size_t)b * a.ntiles + tile] = bs;
        __threadfence();
        is_last = atomicAdd(a.counter + b, 1u) == (unsigned)(a.ntiles - 1);
    }
    __syncthreads();
    if (!is_last) return;
    // last tile of the instance: all threads sum fixed strided subsets of the
    // partials, then a fixed-shape tree (deterministic)
    __threadfence();
    double acc = 0.0;
    for (int k = tid; k < a.ntiles; k += NT) acc += __ldcg(a.partial + (size_t)b * a.ntiles + k);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    __syncthreads();   // red is reused
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid != 0) return;
    double F = 0.0;
    for (int k = 0; k < NT / 32; ++k) F += red[k];
    a.f_cur[b] = F;
    if (!isfinite(F)) atomicExch(a.status, -6);
    if (a.update) {
        if (a.t < a.trace_cap) a.f_trace[(size_t)b * a.trace_cap + a.t] = F;
        if (a.rel_tol > 0.0 && a.t > 0 && a.t - 1 < a.trace_cap && a.done != nullptr) {
            const double Fp = a.f_trace[(size_t)b * a.trace_cap + a.t - 1];
            if (fabs(F - Fp) <= a.rel_tol * fabs(F)) a.done[b] = a.t + 1;
        }
    }
    a.counter[b] = 0u;
}

template <int LP>
__global__ void __launch_bounds__(kThreads, 1)
dense_step_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ DenseTcArgs a) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], tmem_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float mus[kMaxLabels * kMaxLabels];   // mu^T, zero-padded
    __shared__ double red[kThreads / 32];
    __shared__ int is_second, is_last, abort_flag;

    const int tile = blockIdx.x, split = blockIdx.y, b = blockIdx.z;
    const int nsplit = gridDim.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int N = a.N, L = a.L;
    const int row0 = tile * kTM;
    // k range of this CTA
    const int c_begin = (a.nchunk * split) / nsplit, c_end = (a.nchunk * (split + 1)) / nsplit;
    const int nc = c_end - c_begin;

    // aligned by pointer arithmetic on the shared base, so that accesses
    // through it stay shared-memory instructions
    uint8_t *ring = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
    // The next step may be launched now (programmatic dependent launch); it
    // takes the SMs this launch frees.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    load_mu_transposed(mus, a.mu, L, tid, kThreads);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tmem_bar, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, kTN);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    auto kblock = [&](int c) {
        return a.K16 + (((size_t)b * a.nchunk + (c_begin + c)) * a.ntiles + tile) * kStageA;
    };
    // K does not change between steps: the first ring's worth of its blocks
    // is requested before waiting for the previous step (which writes Q, the
    // state and the stopping flags).  Their barriers only count the bytes
    // here; the arrival comes with the Q tile below.
    const int npre = nc < kStages ? nc : kStages;
    if (warp == 0 && lane == 0)
        for (int c = 0; c < npre; ++c) {
            mbar_expect_tx_only(&full_bar[c], kStageA);
            bulk_load(ring + c * kStageBytes, kblock(c), kStageA, &full_bar[c]);
        }
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // stopped before, or the pending F of the previous step meets the rule:
    // read once per block (the writer block of this launch may set done[b])
    if (tid == 0) is_second = a.done != nullptr ? a.done[b] : 0;
    __syncthreads();
    bool stopped = is_second != 0;
    __syncthreads();   // is_second is reused below
    if (!stopped && a.prev_pending) {
        const bool writer = tile == 0 && split == 0;
        if (writer || (a.done != nullptr && a.rel_tol > 0.0)) stopped = dense_deferred_f<kThreads>(a, b, a.t - 1, writer, red);
    }
    if (stopped) {
        // stopping rule met: carry the state through (split 0 copies)
        if (a.update && split == 0)
            for (int idx = tid; idx < kTM * LP; idx += kThreads) {
                const int r = row0 + idx / LP;
                if (r < N) {
                    const size_t o = ((size_t)b * N + r) * LP + idx % LP;
                    a.s_out[o] = a.s_in[o];
                    const float q = idx % LP < L ? __expf(a.s_in[o]) : 0.f;
                    a.q_out[o] = q;
                    if (a.qt_out) a.qt_out[((size_t)b * 32 + idx % LP) * a.Np + r] = __float2bfloat16_rn(q);
                }
            }
        if (warp == 0 && lane == 0)
            for (int c = 0; c < npre; ++c) {   // no copy into this CTA's memory outlives it
                mbar_arrive(&full_bar[c]);
                mbar_wait(&full_bar[c], 0, a.status);
            }
        __syncthreads();
        if (warp == 0) tmem_dealloc(tmem, kTN);
        return;
    }

    if (warp == 0 && lane == 0 && nc > 0) {
        // producer: TMA loads into the ring
        int issued = 0;
        for (int c = 0; c < nc; ++c) {
            const int s = c % kStages;
            if (c >= kStages && !mbar_wait(&empty_bar[s], ((c / kStages) - 1) & 1, a.status)) break;
            if (abort_flag) break;
            uint8_t *sa = ring + s * kStageBytes;
            const int kc = (c_begin + c) * kTK;
            if (c < npre) {
                mbar_expect_tx(&full_bar[s], kStageB);   // K already requested
            } else {
                mbar_expect_tx(&full_bar[s], kStageBytes);
                bulk_load(sa, kblock(c), kStageA, &full_bar[s]);
            }
            tma_load_2d(sa + kStageA, &tmQ, &full_bar[s], kc, b * 32);
            ++issued;
        }
        if (issued < nc) {
            abort_flag = 1;
            // complete the prefetched stages never armed, then drain (bounded)
            // the copies already issued
            for (int c = issued; c < npre; ++c) mbar_arrive(&full_bar[c]);
            const int last = issued > npre ? issued : npre;
            for (int c = (last > kStages ? last - kStages : 0); c < last; ++c)
                mbar_wait(&full_bar[c % kStages], (c / kStages) & 1, a.status);
        }
    } else if (warp == 1 && lane == 0 && nc > 0) {
        // MMA issuer
        int c = 0;
        for (; c < nc; ++c) {
            const int s = c % kStages;
            if (!mbar_wait(&full_bar[s], (c / kStages) & 1, a.status)) break;
            fence_after_sync();
            const uint32_t sa = smem_u32(ring + s * kStageBytes);
            const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + kStageA);
#pragma unroll
            for (int kk = 0; kk < kTK / 16; ++kk)
                mma_bf16(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), kIdesc,
                         (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&empty_bar[s]);
        }
        if (c < nc) abort_flag = 1;
        mma_commit(&tmem_bar);
    }
    __syncwarp();

    // epilogue: this thread's row of the partial sum
    float S[32];
    bool ok = true;
    if (nc > 0) {
        ok = mbar_wait(&tmem_bar, 0, a.status) && !abort_flag;
        fence_after_sync();
        if (ok) tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), S);
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) S[i] = 0.f;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTN);
    if (!ok || abort_flag) return;

    dense_tc_tail<LP, kThreads>(a, S, mus, red, is_second, is_last, tile, split, b, nsplit);
}

// ---------------------------------------------------------------------------
// On-the-fly form: K is not read from memory but computed in the kernel.
//
// With features prescaled by s = sqrt(log2 e / (2 theta^2)) per group, the
// Gaussian weight is K_ij = 2^(-|f_i - f_j|^2) = 2^(2 f_i.f_j - |f_i|^2 -
// |f_j|^2) (zero on the diagonal).  Per chunk of 64 columns the library keeps
// sqrt(2) f_j (5 rows of 64) and -|f_j|^2 (one row) side by side
// (dense_fly_features), 1.5 KiB that one bulk copy brings into a stage with
// the Q^T tile.  Eight builder warps make the 128 x 64 BF16 block of K in
// the stage -- thread t takes rows t mod 64 and t mod 64 + 64 and part t / 64
// of the columns, so each column's features serve two rows: three packed FMAs
// and one exponential per weight -- in the 128-byte-swizzled
// K-major layout of the materialised form, and one more warp issues the same
// tcgen05.mma chain and the copies of the stages ahead.  No K bytes cross
// HBM; the step is bound by the builders' instruction stream (loads of the
// column features, packed FMAs, exponentials, conversions and the per-chunk
// barriers), not by the special-function unit alone.  Split-K, combine, row
// epilogue and free energy are those of the materialised form (dense_tc_tail).
constexpr int kFlyBuilders = 256;                // eight warps build the blocks of K (sixteen measured slower)
constexpr int kFlyParts = kFlyBuilders / (kTM / 2);   // column parts of a chunk; a builder takes two rows
constexpr int kFlyCols = kTK / kFlyParts;              // columns per builder and chunk
constexpr int kFlyThreads = kFlyBuilders + 32;   // and one more issues the MMAs and copies
constexpr int kFlyStages = 8;   // the copies of a stage take about two chunks' work to land
constexpr int kStageF = 6 * kTK * 4;                                       // 1.5 KiB
constexpr int kFlyStageBytes = (kStageA + kStageB + kStageF + 1023) / 1024 * 1024;

template <int LP>
__global__ void __launch_bounds__(kFlyThreads, 1)
dense_fly_tc_kernel(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ DenseTcArgs a) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ __align__(8) uint64_t ld_bar[kFlyStages], a_bar[kFlyStages], empty_bar[kFlyStages], tmem_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float mus[kMaxLabels * kMaxLabels];   // mu^T, zero-padded
    __shared__ double red[kFlyThreads / 32];
    __shared__ int is_second, is_last, abort_flag;

    const int tile = blockIdx.x, split = blockIdx.y, b = blockIdx.z;
    const int nsplit = gridDim.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int N = a.N, L = a.L;
    const int row0 = tile * kTM;
    const int c_begin = (a.nchunk * split) / nsplit, c_end = (a.nchunk * (split + 1)) / nsplit;
    const int nc = c_end - c_begin;
    // builders: rows rr and rr + 64 of the tile, part `half` of a chunk's columns
    const int rr = tid & (kTM / 2 - 1), half = tid / (kTM / 2);
    const int i = tid < kFlyBuilders ? row0 + rr : N, i2 = tid < kFlyBuilders ? i + kTM / 2 : N;

    // aligned by pointer arithmetic on the shared base, so that accesses
    // through it stay shared-memory instructions
    uint8_t *ring = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    load_mu_transposed(mus, a.mu, L, tid, kFlyThreads);
    if (tid == 0) {
        for (int s = 0; s < kFlyStages; ++s) {
            mbar_init(&ld_bar[s], 1);
            mbar_init(&a_bar[s], kFlyBuilders / 32);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tmem_bar, 1);
        abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, kTN);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    auto fblock = [&](int c) { return a.featsT + ((size_t)b * a.nchunk + (c_begin + c)) * (kStageF / 4); };
    // this thread's rows: sqrt(2) f_i and -|f_i|^2 (rows past N get zeros; their results are not used)
    float fi[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, ni = 0.f, fi2[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, ni2 = 0.f;
    if (i < N) {
        const float *fr = a.featsT + ((size_t)b * a.nchunk + i / kTK) * (kStageF / 4) + (i % kTK);
#pragma unroll
        for (int k = 0; k < 5; ++k) fi[k] = __ldg(fr + k * kTK);
        ni = __ldg(fr + 5 * kTK);
    }
    if (i2 < N) {
        const float *fr = a.featsT + ((size_t)b * a.nchunk + i2 / kTK) * (kStageF / 4) + (i2 % kTK);
#pragma unroll
        for (int k = 0; k < 5; ++k) fi2[k] = __ldg(fr + k * kTK);
        ni2 = __ldg(fr + 5 * kTK);
    }
    // the features do not change between steps: the first stages' blocks are
    // requested before waiting for the previous step (which writes Q^T)
    const int npre = nc < kFlyStages ? nc : kFlyStages;
    if (tid == 0)
        for (int c = 0; c < npre; ++c) {
            mbar_expect_tx_only(&ld_bar[c], kStageF);
            bulk_load(ring + c * kFlyStageBytes + kStageA + kStageB, fblock(c), kStageF, &ld_bar[c]);
        }
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (tid == 0) is_second = a.done != nullptr ? a.done[b] : 0;
    __syncthreads();
    bool stopped = is_second != 0;
    __syncthreads();   // is_second is reused below
    if (!stopped && a.prev_pending) {
        const bool writer = tile == 0 && split == 0;
        if (writer || (a.done != nullptr && a.rel_tol > 0.0))
            stopped = dense_deferred_f<kFlyThreads>(a, b, a.t - 1, writer, red);
    }
    if (stopped) {
        // stopping rule met: carry the state through (split 0 copies)
        if (a.update && split == 0)
            for (int idx = tid; idx < kTM * LP; idx += kFlyThreads) {
                const int r = row0 + idx / LP;
                if (r < N) {
                    const size_t o = ((size_t)b * N + r) * LP + idx % LP;
                    a.s_out[o] = a.s_in[o];
                    const float q = idx % LP < L ? __expf(a.s_in[o]) : 0.f;
                    a.q_out[o] = q;
                    if (a.qt_out) a.qt_out[((size_t)b * 32 + idx % LP) * a.Np + r] = __float2bfloat16_rn(q);
                }
            }
        if (tid == 0)
            for (int c = 0; c < npre; ++c) {   // no copy into this CTA's memory outlives it
                mbar_arrive(&ld_bar[c]);
                mbar_wait(&ld_bar[c], 0, a.status);
            }
        __syncthreads();
        if (warp == 0) tmem_dealloc(tmem, kTN);
        return;
    }

    volatile int *abort_v = &abort_flag;
    if (warp < kFlyBuilders / 32) {
        // builders: the 128 x 64 block of K of each chunk
        for (int c = 0; c < nc; ++c) {
            const int s = c % kFlyStages;
            const uint32_t ph = (uint32_t)(c / kFlyStages) & 1u;
            uint8_t *st = ring + s * kFlyStageBytes;
            if (!mbar_wait(&ld_bar[s], ph, a.status)) *abort_v = 1;
            if (!*abort_v) {
                // K[i][j] for this thread's two rows and kFlyCols columns of the chunk
                const float *F = reinterpret_cast<const float *>(st + kStageA + kStageB);
                const int dj = i - (c_begin + c) * kTK, dj2 = dj + kTM / 2;   // the diagonal's columns
                const bool diag = (unsigned)(dj - half * kFlyCols) < (unsigned)kFlyCols;
                const bool diag2 = (unsigned)(dj2 - half * kFlyCols) < (unsigned)kFlyCols;
                uint32_t w[kFlyCols / 2], w2[kFlyCols / 2];
#pragma unroll
                for (int q4 = 0; q4 < kFlyCols / 4; ++q4) {
                    const int j = half * kFlyCols + q4 * 4;
                    const float4 nj = *reinterpret_cast<const float4 *>(F + 5 * kTK + j);
                    float2 e01 = add2(make_float2(nj.x, nj.y), splat2(ni));
                    float2 e23 = add2(make_float2(nj.z, nj.w), splat2(ni));
                    float2 g01 = add2(make_float2(nj.x, nj.y), splat2(ni2));
                    float2 g23 = add2(make_float2(nj.z, nj.w), splat2(ni2));
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const float4 fj = *reinterpret_cast<const float4 *>(F + k * kTK + j);
                        const float2 f01 = make_float2(fj.x, fj.y), f23 = make_float2(fj.z, fj.w);
                        e01 = fma2(splat2(fi[k]), f01, e01);
                        e23 = fma2(splat2(fi[k]), f23, e23);
                        g01 = fma2(splat2(fi2[k]), f01, g01);
                        g23 = fma2(splat2(fi2[k]), f23, g23);
                    }
                    float v0 = ex2_ftz(e01.x), v1 = ex2_ftz(e01.y), v2 = ex2_ftz(e23.x), v3 = ex2_ftz(e23.y);
                    float u0 = ex2_ftz(g01.x), u1 = ex2_ftz(g01.y), u2 = ex2_ftz(g23.x), u3 = ex2_ftz(g23.y);
                    if (diag) {
                        if (j == dj) v0 = 0.f;
                        if (j + 1 == dj) v1 = 0.f;
                        if (j + 2 == dj) v2 = 0.f;
                        if (j + 3 == dj) v3 = 0.f;
                    }
                    if (diag2) {
                        if (j == dj2) u0 = 0.f;
                        if (j + 1 == dj2) u1 = 0.f;
                        if (j + 2 == dj2) u2 = 0.f;
                        if (j + 3 == dj2) u3 = 0.f;
                    }
                    const __nv_bfloat162 p01 = __floats2bfloat162_rn(v0, v1), p23 = __floats2bfloat162_rn(v2, v3);
                    const __nv_bfloat162 r01 = __floats2bfloat162_rn(u0, u1), r23 = __floats2bfloat162_rn(u2, u3);
                    w[2 * q4] = *reinterpret_cast<const uint32_t *>(&p01);
                    w[2 * q4 + 1] = *reinterpret_cast<const uint32_t *>(&p23);
                    w2[2 * q4] = *reinterpret_cast<const uint32_t *>(&r01);
                    w2[2 * q4 + 1] = *reinterpret_cast<const uint32_t *>(&r23);
                }
                // the rows' 16-byte groups in the 128-byte-swizzled K-major layout
                const int rr2 = rr + kTM / 2;
                uint8_t *arow = st + rr * 128, *arow2 = st + rr2 * 128;
#pragma unroll
                for (int g = 0; g < kFlyCols / 8; ++g) {
                    const int gg = half * (kFlyCols / 8) + g;
                    *reinterpret_cast<uint4 *>(arow + ((gg ^ (rr & 7)) << 4)) =
                        make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
                    *reinterpret_cast<uint4 *>(arow2 + ((gg ^ (rr2 & 7)) << 4)) =
                        make_uint4(w2[4 * g], w2[4 * g + 1], w2[4 * g + 2], w2[4 * g + 3]);
                }
            }
            fence_async_smem();   // the tensor cores read the block
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_bar[s]);
            if (*abort_v) break;
        }
    } else if (lane == 0) {
        // the issuer: Q^T of the first stages, then per chunk the MMAs and the
        // copies of the chunk kFlyStages - 1 ahead
        for (int c = 0; c < npre; ++c) {
            mbar_expect_tx(&ld_bar[c], kStageB);   // arrives; the features were counted above
            tma_load_2d(ring + c * kFlyStageBytes + kStageA, &tmQ, &ld_bar[c], (c_begin + c) * kTK, b * 32);
        }
        int issued = npre;   // chunks whose stage copies have been requested
        int c = 0;
        for (; c < nc; ++c) {
            const int s = c % kFlyStages;
            const uint32_t ph = (uint32_t)(c / kFlyStages) & 1u;
            if (!mbar_wait(&a_bar[s], ph, a.status)) *abort_v = 1;
            if (!*abort_v) {
                fence_after_sync();
                const uint32_t sa = smem_u32(ring + s * kFlyStageBytes);
                const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + kStageA);
#pragma unroll
                for (int kk = 0; kk < kTK / 16; ++kk)
                    mma_bf16(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), kIdesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty_bar[s]);
            // refill the stage of chunk c - 1, whose MMAs were issued an iteration ago
            const int cn = c - 1 + kFlyStages;
            if (c >= 1 && cn < nc && !*abort_v) {
                const int sp = (c - 1) % kFlyStages;
                if (mbar_wait(&empty_bar[sp], (uint32_t)((c - 1) / kFlyStages) & 1u, a.status)) {
                    uint8_t *sn = ring + sp * kFlyStageBytes;
                    mbar_expect_tx(&ld_bar[sp], kStageB + kStageF);
                    tma_load_2d(sn + kStageA, &tmQ, &ld_bar[sp], (c_begin + cn) * kTK, b * 32);
                    bulk_load(sn + kStageA + kStageB, fblock(cn), kStageF, &ld_bar[sp]);
                    ++issued;
                } else {
                    *abort_v = 1;
                }
            }
            if (*abort_v) break;
        }
        mma_commit(&tmem_bar);
        // after an abort: the copies already requested land before the CTA leaves (bounded)
        for (int cc = c; cc < issued; ++cc)
            mbar_wait(&ld_bar[cc % kFlyStages], (uint32_t)(cc / kFlyStages) & 1u, a.status);
    }
    __syncwarp();

    float S[32];
    bool ok = true;
    if (nc > 0) {
        ok = mbar_wait(&tmem_bar, 0, a.status) && !*abort_v;
        fence_after_sync();
        if (ok && warp < kTM / 32) {
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), S);
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) S[k] = 0.f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) S[k] = 0.f;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTN);
    if (!ok || *abort_v) return;
    dense_tc_tail<LP, kFlyThreads>(a, S, mus, red, is_second, is_last, tile, split, b, nsplit);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encoder() {
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return cudaSuccess;
}

// 2-D BF16 view [rows][Np] with a box of box_rows x 64 and 128-byte swizzle.
cudaError_t encode_2d(CUtensorMap *map, const void *base, long long rows, int Np, int box_rows) {
    cudaError_t e = get_encoder();
    if (e != cudaSuccess) return e;
    cuuint64_t dims[2] = {(cuuint64_t)Np, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Np * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int dense_tc_tiles(int N) { return (N + kTM - 1) / kTM; }
int dense_tc_pitch(int N) { return (N + kTK - 1) / kTK * kTK; }

cudaError_t launch_dense_f_flush(const DenseStepLaunch &l, int t, cudaStream_t st) {
    DenseTcArgs a{};
    a.partial = l.partial;
    a.f_trace = l.f_trace;
    a.f_cur = l.f_cur;
    a.done = l.done;
    a.status = l.status;
    a.N = l.N;
    a.L = l.L;
    a.ntiles = dense_tc_tiles(l.N);
    a.t = t;
    a.trace_cap = l.trace_cap;
    a.update = 1;
    a.rel_tol = l.rel_tol;
    a.B = l.B;
    dense_f_flush_kernel<<<l.B, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dense_step_tc(const DenseStepLaunch &l, const DenseTcBuffers &tb, cudaStream_t st) {
    CUtensorMap tmQ;
    const int Np = dense_tc_pitch(l.N);
    cudaError_t e = encode_2d(&tmQ, l.qt_in, (long long)l.B * 32, Np, kTN);
    if (e != cudaSuccess) return e;
    DenseTcArgs a;
    a.K16 = reinterpret_cast<const uint8_t *>(l.K16);
    a.s_in = l.s_in;
    a.U = l.U;
    a.s_out = l.s_out;
    a.q_out = l.q_out;
    a.qt_out = l.qt_out;
    a.eta = l.eta;
    a.mu = l.mu;
    a.featsT = l.featsT;
    const bool fly = l.featsT != nullptr;   // K computed in the kernel
    a.split_part = tb.split_part;
    a.tile_count = tb.tile_count;
    a.partial = l.partial;
    a.counter = l.counter;
    a.f_trace = l.f_trace;
    a.f_cur = l.f_cur;
    a.done = l.done;
    a.status = l.status;
    a.N = l.N;
    a.Np = Np;
    a.L = l.L;
    a.ntiles = dense_tc_tiles(l.N);
    a.nchunk = Np / kTK;
    a.t = l.t;
    a.trace_cap = l.trace_cap;
    a.update = l.update;
    a.rel_tol = l.rel_tol;
    a.B = l.B;
    a.defer = l.defer;
    a.prev_pending = l.prev_pending;
    const int nsplit = a.nchunk >= 2 * kSplit ? kSplit : 1;
    dim3 grid(a.ntiles, nsplit, l.B);
    const size_t smem = fly ? (size_t)kFlyStages * kFlyStageBytes + 1024 : (size_t)kStages * kStageBytes + 1024;
    // programmatic dependent launch: the step may start while the previous
    // one drains (the kernel waits before it reads anything a step writes)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(fly ? kFlyThreads : kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    switch (storage_labels(l.L)) {
#define PROXMF_TC_CASE(LPV)                                                                                   \
    case LPV: {                                                                                               \
        auto kern = fly ? dense_fly_tc_kernel<LPV> : dense_step_tc_kernel<LPV>;                               \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);               \
        if (e != cudaSuccess) return e;                                                                       \
        e = cudaLaunchKernelEx(&cfg, kern, tmQ, a);                                                           \
        if (e != cudaSuccess) return e;                                                                       \
        break;                                                                                                \
    }
        PROXMF_TC_CASE(2)
        PROXMF_TC_CASE(4)
        PROXMF_TC_CASE(8)
        PROXMF_TC_CASE(12)
        PROXMF_TC_CASE(16)
        PROXMF_TC_CASE(20)
        PROXMF_TC_CASE(24)
#undef PROXMF_TC_CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace proxmf
