// lanczos.cu -- the step-size constant Lambda of Sec. 3.2, on the device.
//
// For a pairwise model E(q) is quadratic, so its Hessian H (the paper's
// "potential matrix") is constant, and the paper takes its largest eigenvalue
// as the Lipschitz constant of grad E (Sec. 3.2), computed by an iterative
// eigen-solver (the power method, Sec. 4.3).  The update only moves q inside
// the tangent space T = {v : sum_l v_il = 0 for all i} of the simplex product,
// so the constant that governs descent is the top eigenvalue of H restricted
// to T, H_T = C H C with (C v)_il = v_il - mean_l v_il.  It is never larger
// than the unrestricted one, is invariant to constant shifts of mu (which do
// not change the iteration), and is <= 0 exactly when the restricted potential
// matrix is negative semi-definite, where the full parallel update (eta = 1)
// is safe (Sec. 3.2).
//
// Two forms:
//  - symmetric mu: H = W (x) mu with W the symmetric weighted adjacency, so
//    H_T = W (x) (C mu C) and its spectrum is {lambda(W) nu} with nu the
//    eigenvalues of C mu C.  Lanczos runs on the scalar field W (N unknowns)
//    and a one-thread Jacobi solve gives nu; Lambda is the largest product of
//    the extreme values.
//  - otherwise: Lanczos on H_T itself (N*L unknowns), the matrix-vector
//    product being the message computation of the step kernel in FP64.
// Lanczos runs without re-orthogonalisation; its extreme Ritz values converge
// to the extreme eigenvalues from inside.  Every instance of a batch gets its
// own constant.  All arithmetic is on the device; the host only sequences
// launches and reads back convergence flags.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"

namespace proxmf {

namespace {

constexpr int kLzThreads = 256;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    // SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-level sum, then last-block-of-instance finalisation in fixed order.
// Returns true in the (single) thread that holds the instance total in *tot.
__device__ bool instance_reduce(double v, double *partial, unsigned *counter, int b, int nblk,
                                double *tot) {
    __shared__ double red[kLzThreads / 32];
    __shared__ int last;
    const int tid = threadIdx.x;
    v = warp_sum(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int k = 0; k < kLzThreads / 32; ++k) s += red[k];
        partial[(size_t)b * nblk + blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(counter + b, 1u) == (unsigned)(nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc = 0.0;
    for (int k = tid; k < nblk; k += kLzThreads) acc += __ldcg(partial + (size_t)b * nblk + k);
    acc = warp_sum(acc);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid != 0) return false;
    double s = 0.0;
    for (int k = 0; k < kLzThreads / 32; ++k) s += red[k];
    *tot = s;
    counter[b] = 0u;
    return true;
}

struct LzGeom {
    int B, Lv, L, H, W, P, conn;   // Lv = 1 (scalar W) or L (full H_T)
    int nblk;                      // blocks per instance over H*W pixels
};

__device__ __forceinline__ void dir_off(int k, int *dy, int *dx) {
    *dy = k == 0 ? 0 : 1;
    *dx = k == 0 ? 1 : (k == 1 ? 0 : (k == 2 ? 1 : -1));
}

// v = random start vector (uniform in [-1, 1] from SplitMix64), centred over
// labels in the full form; padding columns are 0.
__global__ void lz_init_kernel(double *v, LzGeom g, unsigned long long seed) {
    const int b = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.H * g.W) return;
    const int y = p / g.W, x = p - y * g.W;
    const size_t plane = (size_t)g.H * g.P;
    double *vb = v + (size_t)b * g.Lv * plane + (size_t)y * g.P + x;
    double mean = 0.0;
    for (int l = 0; l < g.Lv; ++l) {
        const unsigned long long h =
            splitmix64(seed ^ splitmix64(((unsigned long long)b * g.Lv + l) * 0x100000000ull + (unsigned)p));
        const double r = (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        vb[l * plane] = r;
        mean += r;
    }
    if (g.Lv > 1) {
        mean /= g.Lv;
        for (int l = 0; l < g.Lv; ++l) vb[l * plane] -= mean;
    }
}

// Lanczos state.  Raw vectors u_k live in R[k % 3]; v_k = u_k / nrm[k] is
// never written out (normalisation is applied on the fly).  The step index k
// is read from *kdev, so that a CUDA graph of many steps can be replayed.
struct LzState {
    double *R0, *R1, *R2;
    double *alpha, *nrm;   // [B][ld]: alpha_k, nrm[k] = |u_k| (nrm[k+1] = beta_k)
    int *kdev;
    int *stop;
    double *partial;
    unsigned *counter;
    int ld;
};

__device__ __forceinline__ double *lz_buf(const LzState &s, int i) {
    return i == 0 ? s.R0 : (i == 1 ? s.R1 : s.R2);
}

// FP64 copy of the pixel-major edge weights for the scalar form (FP64 is the
// slow pipe on this part: converting once instead of every step halves the
// FP64 work of a Lanczos step).
// max |w| as float bits (non-negative floats order as unsigned integers)
__global__ void lz_absmax_kernel(const float *__restrict__ w, size_t n, unsigned *out_bits) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(w[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
}

__global__ void lz_weights_f64_kernel(const float *__restrict__ w, double *__restrict__ wd, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        wd[i] = (double)w[i];
}

// Step part A: t = A v_k into R[(k+1) % 3] and alpha_k = v_k . t, with
// A = W (scalar form) or C H C (full form).
// Scalar form (symmetric mu): t = W v_k, one value per pixel.
__global__ void __launch_bounds__(kLzThreads)
lz_step_a_scalar_kernel(LzState st, const double *__restrict__ w, LzGeom g) {
    const int b = blockIdx.y;
    const int k = *st.kdev;
    if (st.stop[b] || k >= st.ld - 1) return;
    const double *v = lz_buf(st, k % 3) + (size_t)b * g.H * g.P;
    double *out = lz_buf(st, (k + 1) % 3) + (size_t)b * g.H * g.P;
    const double inv = 1.0 / st.nrm[(size_t)b * st.ld + k];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int nd = g.conn == 8 ? 4 : 2;
    double dot = 0.0;
    if (p < g.H * g.W) {
        const int y = p / g.W, x = p - y * g.W;
        const double *wb = w + (size_t)b * g.H * g.W * nd;
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            if (d >= nd) break;
            const int dy = d == 0 ? 0 : 1, dx = d == 0 ? 1 : (d == 1 ? 0 : (d == 2 ? 1 : -1));
            const int yo = y + dy, xo = x + dx;
            if (yo < g.H && xo >= 0 && xo < g.W) acc = fma(wb[((size_t)y * g.W + x) * nd + d], v[(size_t)yo * g.P + xo], acc);
            const int yi = y - dy, xi = x - dx;
            if (yi >= 0 && xi >= 0 && xi < g.W) acc = fma(wb[((size_t)yi * g.W + xi) * nd + d], v[(size_t)yi * g.P + xi], acc);
        }
        const double r = acc * inv;
        out[(size_t)y * g.P + x] = r;
        dot = r * v[(size_t)y * g.P + x] * inv;
    }
    double tot;
    if (instance_reduce(dot, st.partial, st.counter, b, g.nblk, &tot)) st.alpha[(size_t)b * st.ld + k] = tot;
}

// Dense scalar form: t = K v_k, one warp per row of the FP32 weight matrix
// (FP64 accumulation); alpha_k from one partial per block.
__global__ void __launch_bounds__(kLzThreads)
lz_step_a_dense_kernel(LzState st, const float *__restrict__ K, LzGeom g, int nblk_a) {
    const int b = blockIdx.y;
    const int k = *st.kdev;
    if (st.stop[b] || k >= st.ld - 1) return;
    const int N = g.W;
    const double *v = lz_buf(st, k % 3) + (size_t)b * N;
    double *out = lz_buf(st, (k + 1) % 3) + (size_t)b * N;
    const double inv = 1.0 / st.nrm[(size_t)b * st.ld + k];
    const int row = blockIdx.x * (kLzThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    double dot = 0.0;
    if (row < N) {
        const float *kr = K + ((size_t)b * N + row) * N;
        double acc = 0.0;
        for (int j = lane; j < N; j += 32) acc += (double)kr[j] * v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double r = acc * inv;
        if (lane == 0) {
            out[row] = r;
            dot = r * v[row] * inv;
        }
    }
    double tot;
    if (instance_reduce(dot, st.partial, st.counter, b, nblk_a, &tot)) st.alpha[(size_t)b * st.ld + k] = tot;
}

// Full form (any mu): t = C H C v_k over N*L unknowns.
__global__ void __launch_bounds__(kLzThreads)
lz_step_a_kernel(LzState st, const float *__restrict__ w, const float *__restrict__ mu, LzGeom g) {
    const int b = blockIdx.y;
    const int k = *st.kdev;
    if (st.stop[b] || k >= st.ld - 1) return;
    __shared__ double mus[kMaxLabels * kMaxLabels];
    if (g.Lv > 1)
        for (int i = threadIdx.x; i < g.L * g.L; i += blockDim.x) mus[i] = (double)mu[i];
    __syncthreads();
    const double *v = lz_buf(st, k % 3);
    double *out = lz_buf(st, (k + 1) % 3);
    const double inv = 1.0 / st.nrm[(size_t)b * st.ld + k];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int nd = g.conn == 8 ? 4 : 2;
    const size_t plane = (size_t)g.H * g.P;
    double dot = 0.0;
    if (p < g.H * g.W) {
        const int y = p / g.W, x = p - y * g.W;
        const double *vb = v + (size_t)b * g.Lv * plane;
        const float *wb = w + (size_t)b * g.H * g.W * nd;   // pixel-major [N][nd]
        const size_t pix = (size_t)y * g.P + x;
        double So[kMaxLabels], Si[kMaxLabels];
        for (int l = 0; l < g.Lv; ++l) So[l] = Si[l] = 0.0;
        for (int d = 0; d < nd; ++d) {
            int dy, dx;
            dir_off(d, &dy, &dx);
            const int yo = y + dy, xo = x + dx;           // out-going edge to (yo, xo)
            if (yo >= 0 && yo < g.H && xo >= 0 && xo < g.W) {
                const double wo = (double)wb[((size_t)y * g.W + x) * nd + d];
                const size_t po = (size_t)yo * g.P + xo;
                for (int l = 0; l < g.Lv; ++l) So[l] += wo * vb[l * plane + po];
            }
            const int yi = y - dy, xi = x - dx;           // in-coming edge from (yi, xi)
            if (yi >= 0 && yi < g.H && xi >= 0 && xi < g.W) {
                const size_t pi = (size_t)yi * g.P + xi;
                const double wi = (double)wb[((size_t)yi * g.W + xi) * nd + d];
                for (int l = 0; l < g.Lv; ++l) Si[l] += wi * vb[l * plane + pi];
            }
        }
        double *ob = out + (size_t)b * g.Lv * plane;
        if (g.Lv == 1) {
            const double r = (So[0] + Si[0]) * inv;
            ob[pix] = r;
            dot = r * vb[pix] * inv;
        } else {
            double m[kMaxLabels];
            double mean = 0.0;
            for (int l = 0; l < g.L; ++l) {
                double t = 0.0;
                for (int q = 0; q < g.L; ++q) t += mus[l * g.L + q] * So[q] + mus[q * g.L + l] * Si[q];
                m[l] = t * inv;
                mean += m[l];
            }
            mean /= g.L;
            for (int l = 0; l < g.L; ++l) {
                const double r = m[l] - mean;
                ob[l * plane + pix] = r;
                dot += r * vb[l * plane + pix] * inv;
            }
        }
    }
    double tot;
    if (instance_reduce(dot, st.partial, st.counter, b, g.nblk, &tot)) st.alpha[(size_t)b * st.ld + k] = tot;
}

// Step part B: u_{k+1} = t - alpha_k v_k - nrm[k] v_{k-1} in place of t, and
// nrm[k+1] = |u_{k+1}|; the last block of the last instance advances k.
// An instance whose new norm collapses (an invariant subspace) stops.
__global__ void __launch_bounds__(kLzThreads)
lz_step_b_kernel(LzState st, LzGeom g) {
    const int b = blockIdx.y;
    const int k = *st.kdev;
    const bool active = !st.stop[b] && k < st.ld - 1;
    double nrm2 = 0.0;
    if (active) {
        const size_t plane = (size_t)g.H * g.P;
        double *t = lz_buf(st, (k + 1) % 3);
        const double *uk = lz_buf(st, k % 3);
        const double *um = lz_buf(st, (k + 2) % 3);
        const double a = st.alpha[(size_t)b * st.ld + k];
        const double nk = st.nrm[(size_t)b * st.ld + k];
        const double ik = 1.0 / nk;
        const double im = k > 0 ? 1.0 / st.nrm[(size_t)b * st.ld + k - 1] : 0.0;
        const double ca = a * ik, cm = nk * im;   // coefficients of u_k and u_{k-1}
        const int p = blockIdx.x * blockDim.x + threadIdx.x;
        if (p < g.H * g.W) {
            const int y = p / g.W, x = p - y * g.W;
            const size_t off = (size_t)b * g.Lv * plane + (size_t)y * g.P + x;
            for (int l = 0; l < g.Lv; ++l) {
                const size_t i = off + l * plane;
                double r = fma(-ca, uk[i], t[i]);
                if (k > 0) r = fma(-cm, um[i], r);
                t[i] = r;
                nrm2 = fma(r, r, nrm2);
            }
        }
    }
    // every block takes part in the counter so that the last one can advance k
    __shared__ double red[kLzThreads / 32];
    __shared__ int last_inst;
    double v = warp_sum(nrm2);
    const int tid = threadIdx.x;
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < kLzThreads / 32; ++i) s += red[i];
        st.partial[(size_t)b * g.nblk + blockIdx.x] = s;
        __threadfence();
        last_inst = atomicAdd(st.counter + b, 1u) == (unsigned)(g.nblk - 1);
    }
    __syncthreads();
    if (!last_inst) return;
    __threadfence();
    double acc = 0.0;
    for (int i = tid; i < g.nblk; i += kLzThreads) acc += __ldcg(st.partial + (size_t)b * g.nblk + i);
    acc = warp_sum(acc);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid != 0) return;
    double s = 0.0;
    for (int i = 0; i < kLzThreads / 32; ++i) s += red[i];
    st.counter[b] = 0u;
    if (active) {
        const double bk = sqrt(s);
        // breakdown scale |alpha_k| + beta_{k-1}; at k = 0, |alpha_0| + beta_0
        // (nrm[0] is the start vector's norm, unrelated to the matrix scale)
        const double ref = fabs(st.alpha[(size_t)b * st.ld + k]) + (k > 0 ? st.nrm[(size_t)b * st.ld + k] : bk);
        st.nrm[(size_t)b * st.ld + k + 1] = bk;
        if (!(bk > 1e-13 * ref) || !(bk > 1e-300)) st.stop[b] = k + 1;
    }
    // the instances finish in any order: the last one advances the step
    __threadfence();
    if (atomicAdd(st.counter + g.B, 1u) == (unsigned)(g.B - 1)) {
        st.counter[g.B] = 0u;
        *st.kdev = k + 1;
    }
}

// ---- cooperative form: a whole chunk of scalar-form steps in one launch ----
//
// One block per SM (or fewer), every block of an instance owning a fixed
// strided set of pixels; the two reductions of a step (alpha_k and |u_{k+1}|)
// are block partials summed in a fixed order after a grid barrier by every
// block, so all blocks hold the same alpha_k and beta_k and no launch or
// last-block tail separates the steps.  The vectors u_k are stored as
// double-float pairs (same 8 bytes as an FP64 value); the step's scalars are
// FP64, formed once per block (FP64 division is a long sequence on the
// narrow FP64 pipe).

constexpr int kCoopThreads = 512;
constexpr long long kLzWaitCycles = 4000000000ll;   // ~2 s at 2 GHz per barrier wait

struct LzCoop {
    unsigned *bar;   // [0] arrivals, [1] generation
    int *abort;      // set once a barrier wait ran out; every later barrier fails
    double *part;    // [2][B][gx] block partials of alpha_k and |u_{k+1}|^2
    int gx;          // blocks per instance
};

// Grid-wide barrier of a cooperative launch with a bounded wait, run by one
// thread per block.  The thread arrives on the counter with an acquire-
// release atomic (its block's earlier writes, ordered before it by the
// block barrier, are released with it); the last arrival resets the counter
// and advances the generation word with a release, which the others poll
// with acquire loads.  Returns false when this or another block's wait ran
// out of its clock budget (the abort word is then set for everyone).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool grid_arrive_wait(const LzCoop &c, unsigned nblocks) {
    volatile int *ab = c.abort;
    if (*ab != 0) return false;
    const unsigned g0 = ld_acquire(c.bar + 1);
    if (atom_add_acq_rel(c.bar, 1u) == nblocks - 1) {
        atomicExch(c.bar, 0u);
        red_add_release(c.bar + 1, 1u);
        return true;
    }
    const long long t0 = clock64();
    while (ld_acquire(c.bar + 1) == g0) {
        if (*ab != 0) return false;
        if (clock64() - t0 > kLzWaitCycles) {
            atomicExch(c.abort, 1);
            return false;
        }
    }
    return true;
}

// The same as a block-level call: every thread returns the outcome.
__device__ bool coop_barrier(const LzCoop &c, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) ok = grid_arrive_wait(c, nblocks) ? 1 : 0;
    __syncthreads();
    return ok != 0;
}

// Sum of the n partials of an instance in a fixed order by warp 0 (strided
// per lane, fixed-shape tree); the value is returned in thread 0.
__device__ double coop_sum(const double *p, int n) {
    if (threadIdx.x >= 32) return 0.0;
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) a += __ldcg(p + i);
    return warp_sum(a);
}

// Block total of the threads' double-float values into *part (thread 0):
// double-float warp trees, then the warps' FP64 values in index order.
__device__ void coop_partial(df v, double *red, double *part) {
    v = warp_sum_df(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = df_to(v);
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kCoopThreads / 32; ++k) s += red[k];
        __stcg(part, s);
    }
}

// (W u)_p of the scalar form: the weighted neighbour sum over the grid's
// edges at pixel p, compensated, from the FP32 pixel-major weights (read
// only, through L1) and the double-float vector u (read through L2: it is
// written inside the launch and L1 is not coherent across blocks).
__device__ __forceinline__ df w_times(const float *__restrict__ wb, const float2 *u, const LzGeom &g, int nd,
                                      int p) {
    const int y = p / g.W, x = p - y * g.W;
    float ah = 0.f, al = 0.f;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        if (d >= nd) break;
        const int dy = d == 0 ? 0 : 1, dx = d == 0 ? 1 : (d == 1 ? 0 : (d == 2 ? 1 : -1));
        const int yo = y + dy, xo = x + dx;
        if (yo < g.H && xo >= 0 && xo < g.W) {
            const int q = yo * g.W + xo;
            const float2 v = __ldcg(u + q);
            acc_prod_f(ah, al, __ldg(wb + (size_t)p * nd + d), df{v.x, v.y});
        }
        const int yi = y - dy, xi = x - dx;
        if (yi >= 0 && xi >= 0 && xi < g.W) {
            const int q = yi * g.W + xi;
            const float2 v = __ldcg(u + q);
            acc_prod_f(ah, al, __ldg(wb + (size_t)q * nd + d), df{v.x, v.y});
        }
    }
    return df_fast_two_sum(ah, al);
}

// The step's scalars, formed in FP64 by thread 0 of every block (all blocks
// hold the same sums, so they agree) and handed to the block as double-float
// pairs in shared memory; no other thread touches the FP64 pipe.
struct CoopScalars {
    float inv_h, inv_l;   // 1 / |u_k|
    float cm_h, cm_l;     // -|u_k| / |u_{k-1}|
    float ca_h, ca_l;     // -alpha_k / |u_k|
    int brk;              // the instance stopped at this step
};

struct CoopThread0 {      // FP64 state, meaningful in thread 0
    double nk, inv, alpha;
};

__device__ __forceinline__ void coop_scalars_init(const LzState &st, int b, int k0, bool active, CoopScalars &cs,
                                                  CoopThread0 &t0) {
    const size_t ld = (size_t)st.ld;
    t0.nk = st.nrm[b * ld + k0];
    t0.inv = active ? 1.0 / t0.nk : 0.0;
    t0.alpha = 0.0;
    const df a = df_from(t0.inv), m = df_from(active && k0 > 0 ? -t0.nk / st.nrm[b * ld + k0 - 1] : 0.0);
    cs.inv_h = a.h;
    cs.inv_l = a.l;
    cs.cm_h = m.h;
    cs.cm_l = m.l;
    cs.ca_h = cs.ca_l = 0.f;
    cs.brk = 0;
}

// after the alpha reduction (s = sum of t . u_k over the instance)
__device__ __forceinline__ void coop_scalars_alpha(double s, CoopScalars &cs, CoopThread0 &t0) {
    t0.alpha = s * t0.inv;
    const df ca = df_from(-t0.alpha * t0.inv);
    cs.ca_h = ca.h;
    cs.ca_l = ca.l;
}

// after the norm reduction (s = |u_{k+1}|^2): record alpha_k and beta_k,
// apply the stopping rule, form the next step's scalars
__device__ __forceinline__ void coop_scalars_beta(double s, const LzState &st, int b, int bx, int k, CoopScalars &cs,
                                                  CoopThread0 &t0) {
    const size_t ld = (size_t)st.ld;
    const double bk = sqrt(s);
    const double ref = fabs(t0.alpha) + (k > 0 ? t0.nk : bk);   // as in the two-kernel form
    const bool brk = !(bk > 1e-13 * ref) || !(bk > 1e-300);
    if (bx == 0) {
        st.alpha[b * ld + k] = t0.alpha;
        st.nrm[b * ld + k + 1] = bk;
        if (brk) st.stop[b] = k + 1;
    }
    t0.inv = brk ? 0.0 : 1.0 / bk;
    const df a = df_from(t0.inv), m = df_from(-bk / t0.nk);
    cs.inv_h = a.h;
    cs.inv_l = a.l;
    cs.cm_h = m.h;
    cs.cm_l = m.l;
    cs.brk = brk ? 1 : 0;
    t0.nk = bk;
}

// Steps k0 .. k1-1 of the scalar form (t = W v_k, W the symmetric weighted
// adjacency of the grid), any size: each thread strides over the pixels of
// its instance and every vector travels through L2 (t in the u_{k+1}
// buffer).  The recurrence and stopping rule are those of the two-kernel
// FP64 form above.
__global__ void __launch_bounds__(kCoopThreads, 1)
lz_chunk_strided_kernel(LzState st, const float *__restrict__ w, LzGeom g, LzCoop c, int k0, int k1, int) {
    __shared__ double red[kCoopThreads / 32];
    __shared__ CoopScalars cs;
    const int b = blockIdx.y, bx = blockIdx.x, tid = threadIdx.x;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const int N = g.H * g.W;
    const int nd = g.conn == 8 ? 4 : 2;
    const size_t base = (size_t)b * N;
    const float *wb = w + base * nd;
    double *pa = c.part + (size_t)b * c.gx;
    double *pb = c.part + ((size_t)g.B + b) * c.gx;
    const int p0 = bx * kCoopThreads + tid, stride = c.gx * kCoopThreads;
    bool active = st.stop[b] == 0;
    CoopThread0 t0{};
    if (tid == 0) coop_scalars_init(st, b, k0, active, cs, t0);
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const df inv = {cs.inv_h, cs.inv_l}, cm = {cs.cm_h, cs.cm_l};
        const float2 *v = reinterpret_cast<const float2 *>(lz_buf(st, k % 3)) + base;
        float2 *t = reinterpret_cast<float2 *>(lz_buf(st, (k + 1) % 3)) + base;
        const float2 *vm = reinterpret_cast<const float2 *>(lz_buf(st, (k + 2) % 3)) + base;
        // t = W v_k = (W u_k) / |u_k| and the partial of alpha_k |u_k| = t . u_k
        float dh = 0.f, dl = 0.f;
        if (active) {
            for (int p = p0; p < N; p += stride) {
                const df r = df_mul(w_times(wb, v, g, nd, p), inv);
                __stcg(t + p, make_float2(r.h, r.l));
                const float2 u = __ldcg(v + p);
                acc_prod(dh, dl, r, df{u.x, u.y});
            }
        }
        coop_partial(df_fast_two_sum(dh, dl), red, pa + bx);
        if (!coop_barrier(c, nblocks)) return;
        const double sa = coop_sum(pa, c.gx);
        if (tid == 0 && active) coop_scalars_alpha(sa, cs, t0);
        __syncthreads();
        // u_{k+1} = t - alpha_k v_k - |u_k| v_{k-1} and its squared norm
        float nh = 0.f, nl = 0.f;
        if (active) {
            const df ca = {cs.ca_h, cs.ca_l};
            for (int p = p0; p < N; p += stride) {
                const float2 tp = __ldcg(t + p), u = __ldcg(v + p);
                float rh = tp.x, rl = tp.y;
                acc_prod(rh, rl, ca, df{u.x, u.y});
                if (k > 0) {
                    const float2 m2 = __ldcg(vm + p);
                    acc_prod(rh, rl, cm, df{m2.x, m2.y});
                }
                const df r = df_fast_two_sum(rh, rl);
                __stcg(t + p, make_float2(r.h, r.l));
                acc_prod(nh, nl, r, r);
            }
        }
        coop_partial(df_fast_two_sum(nh, nl), red, pb + bx);
        if (!coop_barrier(c, nblocks)) return;
        const double sb = coop_sum(pb, c.gx);
        if (tid == 0 && active) coop_scalars_beta(sb, st, b, bx, k, cs, t0);
        __syncthreads();
        if (cs.brk != 0) active = false;
    }
}

// (W u) at stage index i with weights and vector staged in shared memory:
// ws holds the pixel-major weights of the edges leaving each pixel (right,
// down, down-right, down-left; zero for edges that leave the image) and u the
// double-float vector, both zero outside the instance.  On the linear pixel
// index the neighbour in direction d is i + off_d and the edge entering from
// the opposite side comes from i - off_d; a pair that is not a grid edge
// (a row wrap) always carries a zero weight, so no bounds tests are needed.
template <int ND>
__device__ __forceinline__ df w_times_staged(const float *__restrict__ ws, const float2 *__restrict__ u, int i,
                                             int W) {
    float ah = 0.f, al = 0.f;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const int off = d == 0 ? 1 : (d == 1 ? W : (d == 2 ? W + 1 : W - 1));
        const float2 vo = u[i + off], vi = u[i - off];
        acc_prod_f(ah, al, ws[i * 4 + d], df{vo.x, vo.y});
        acc_prod_f(ah, al, ws[(i - off) * 4 + d], df{vi.x, vi.y});
    }
    return df_fast_two_sum(ah, al);
}

// Steps k0 .. k1-1 of the scalar form with one grid barrier per step.
// Block bx of an instance owns the contiguous pixels [ps, pe); with
// R1 = W + 1 every neighbour of a pixel p lies in [p - R1, p + R1].  The
// block keeps u_k, u_{k-1} and the edge weights in shared memory over
// [ps - 2 R1, pe + 2 R1) and advances u redundantly on the ring
// [ps - R1, pe + R1) too, with the same arithmetic as the owning blocks (so
// the copies agree bit for bit): the next product then needs no other
// block's new values, and the one barrier of a step serves both the
// reductions and the visibility of the vectors written one step earlier,
// from which the outer ring is reloaded.  With the unnormalised u_k,
// t' = W u_k, one reduction gives alpha_k = t'.u_k / |u_k|^2 and
// |u_k| = beta_{k-1} together, and
//   u_{k+1} = (t' - alpha_k u_k) / |u_k| - (|u_k| / |u_{k-1}|) u_{k-1}.
// nrm[k] = |u_k| is recorded at step k; a collapsed |u_k| stops the
// instance with k rows, as in the other forms.  Warp 0 runs the control
// path (barrier, fixed-order sums, FP64 scalars); warps 1.. own at most PPT
// pixels per thread.
constexpr int kCoopWorkers = kCoopThreads - 32;

template <int PPT, int ND>
__global__ void __launch_bounds__(kCoopThreads, 1)
lz_chunk_halo_kernel(LzState st, const float *__restrict__ w, LzGeom g, LzCoop c, int k0, int k1, int chunk) {
    extern __shared__ float4 smem4[];
    __shared__ double red[2 * (kCoopThreads / 32)];
    __shared__ float fs[6];   // c1 = 1/|u_k|, c2 = -alpha_k/|u_k|, c3 = -|u_k|/|u_{k-1}| (h, l)
    __shared__ int flags[2];  // [0] grid barrier outcome, [1] the instance stopped
    const int b = blockIdx.y, bx = blockIdx.x, tid = threadIdx.x, warp = tid >> 5;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const int N = g.H * g.W, W = g.W, R1 = g.W + 1;
    const size_t base = (size_t)b * N;
    const float *wb = w + base * ND;
    double *pa = c.part + (size_t)b * c.gx;
    double *pb = c.part + ((size_t)g.B + b) * c.gx;
    const size_t ld = (size_t)st.ld;
    const int ps = min(N, bx * chunk), pe = min(N, ps + chunk);
    const int o2 = ps - 2 * R1;                 // pixel of stage index 0 (may be negative)
    const int S = chunk + 4 * R1;               // stage entries
    const int lo1 = max(0, ps - R1), hi1 = min(N, pe + R1);
    const int lo2 = max(0, ps - 2 * R1), hi2 = min(N, pe + 2 * R1);
    const int nl1 = ps - lo1, nring = nl1 + (hi1 - pe);
    const int wt = tid - 32;
    float *ws = reinterpret_cast<float *>(smem4);                               // [S][4] weights
    float2 *su = reinterpret_cast<float2 *>(smem4 + S), *sm = su + S;          // u_k, u_{k-1}
    bool active = st.stop[b] == 0;
    // thread 0: |u_{k-1}|, its reciprocal and alpha_{k-1}
    double n_prev = 0.0, a_prev = 0.0, inv_prev = 0.0;
    if (tid == 0) {
        n_prev = k0 > 0 ? st.nrm[b * ld + k0 - 1] : 0.0;
        a_prev = k0 > 0 ? st.alpha[b * ld + k0 - 1] : 0.0;
        inv_prev = k0 > 0 ? 1.0 / n_prev : 0.0;
        flags[1] = 0;
    }
    {
        const float2 *v0 = reinterpret_cast<const float2 *>(lz_buf(st, k0 % 3)) + base;
        const float2 *v1 = reinterpret_cast<const float2 *>(lz_buf(st, (k0 + 2) % 3)) + base;
        const float2 z = make_float2(0.f, 0.f);
        for (int i = tid; i < S; i += kCoopThreads) {
            const int q = o2 + i;
            const bool in = q >= 0 && q < N;
            su[i] = in && q < hi2 ? __ldcg(v0 + q) : z;
            sm[i] = in && q >= lo1 && q < hi1 ? __ldcg(v1 + q) : z;
#pragma unroll
            for (int d = 0; d < 4; ++d) ws[i * 4 + d] = in && d < ND ? __ldg(wb + (size_t)q * ND + d) : 0.f;
        }
    }
    df tt[PPT];
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const float2 *ucur = reinterpret_cast<const float2 *>(lz_buf(st, k % 3)) + base;
        float2 *unext = reinterpret_cast<float2 *>(lz_buf(st, (k + 1) % 3)) + base;
        // t' = W u_k on the own pixels, partials of t'.u_k and |u_k|^2 (workers)
        if (wt >= 0) {
            float dh = 0.f, dl = 0.f, nh = 0.f, nl = 0.f;
            if (active) {
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const int p = ps + wt + j * kCoopWorkers;
                    if (p < pe) {
                        tt[j] = w_times_staged<ND>(ws, su, p - o2, W);
                        const float2 u2 = su[p - o2];
                        const df u = {u2.x, u2.y};
                        acc_prod(dh, dl, tt[j], u);
                        acc_prod(nh, nl, u, u);
                    }
                }
            }
            const df d = warp_sum_df(df_fast_two_sum(dh, dl));
            const df n = warp_sum_df(df_fast_two_sum(nh, nl));
            if ((tid & 31) == 0) {
                red[warp] = df_to(d);
                red[16 + warp] = df_to(n);
            }
        }
        __syncthreads();
        if (warp == 0) {
            // block partials: the warps' values by a fixed-shape tree
            const int lane = tid;
            double sd = lane >= 1 && lane < kCoopThreads / 32 ? red[lane] : 0.0;
            double sn = lane >= 1 && lane < kCoopThreads / 32 ? red[16 + lane] : 0.0;
            sd = warp_sum(sd);
            sn = warp_sum(sn);
            if (lane == 0) {
                __stcg(pa + bx, sd);
                __stcg(pb + bx, sn);
                flags[0] = grid_arrive_wait(c, nblocks) ? 1 : 0;
            }
        }
        __syncthreads();
        if (flags[0] == 0) return;
        if (warp == 0) {
            // both sums of the instance in one pass over the partials
            double sd = 0.0, sn = 0.0;
            for (int i = tid; i < c.gx; i += 32) {
                sd += __ldcg(pa + i);
                sn += __ldcg(pb + i);
            }
            sd = warp_sum(sd);
            sn = warp_sum(sn);
            if (tid == 0 && active) {
                // one reciprocal square root; the rest are products
                const double inv = rsqrt(sn);
                const double nk = sn * inv;
                // beta_{k-1} against |alpha_{k-1}| + beta_{k-2} (beta_0 itself at k = 1)
                const bool brk =
                    !(nk > 1e-300) || (k > 0 && !(nk > 1e-13 * (fabs(a_prev) + (k > 1 ? n_prev : nk))));
                const double alpha = sd * inv * inv;
                if (bx == 0) {
                    if (k > 0) st.nrm[b * ld + k] = nk;
                    if (brk)
                        st.stop[b] = k;
                    else
                        st.alpha[b * ld + k] = alpha;
                }
                const df c1 = df_from(inv), c2 = df_from(-alpha * inv), c3 = df_from(k > 0 ? -nk * inv_prev : 0.0);
                fs[0] = c1.h;
                fs[1] = c1.l;
                fs[2] = c2.h;
                fs[3] = c2.l;
                fs[4] = c3.h;
                fs[5] = c3.l;
                flags[1] = brk ? 1 : 0;
                a_prev = alpha;
                n_prev = nk;
                inv_prev = inv;
            }
        } else if (active) {
            // outer ring of u_k from L2: written by its owners at step k - 1,
            // visible since this step's barrier
            for (int q = lo2 + wt; q < lo1; q += kCoopWorkers) su[q - o2] = __ldcg(ucur + q);
            for (int q = hi1 + wt; q < hi2; q += kCoopWorkers) su[q - o2] = __ldcg(ucur + q);
        }
        __syncthreads();
        if (flags[1] != 0) active = false;
        // u_{k+1} on the own pixels (also to L2) and on the inner ring, into sm
        if (wt >= 0 && active) {
            const df c1 = {fs[0], fs[1]}, c2 = {fs[2], fs[3]}, c3 = {fs[4], fs[5]};
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int p = ps + wt + j * kCoopWorkers;
                if (p < pe) {
                    const float2 u = su[p - o2], m = sm[p - o2];
                    float rh = 0.f, rl = 0.f;
                    acc_prod(rh, rl, c1, tt[j]);
                    acc_prod(rh, rl, c2, df{u.x, u.y});
                    acc_prod(rh, rl, c3, df{m.x, m.y});
                    const df r = df_fast_two_sum(rh, rl);
                    const float2 r2 = make_float2(r.h, r.l);
                    sm[p - o2] = r2;
                    __stcg(unext + p, r2);
                }
            }
            for (int i = wt; i < nring; i += kCoopWorkers) {
                const int q = i < nl1 ? lo1 + i : pe + (i - nl1);
                const df t = w_times_staged<ND>(ws, su, q - o2, W);
                const float2 u = su[q - o2], m = sm[q - o2];
                float rh = 0.f, rl = 0.f;
                acc_prod(rh, rl, c1, t);
                acc_prod(rh, rl, c2, df{u.x, u.y});
                acc_prod(rh, rl, c3, df{m.x, m.y});
                const df r = df_fast_two_sum(rh, rl);
                sm[q - o2] = make_float2(r.h, r.l);
            }
        }
        __syncthreads();
        float2 *tmp = su;
        su = sm;
        sm = tmp;
    }
}

// In-place FP64 -> double-float conversion of the start vector (same 8 bytes).
__global__ void lz_split_kernel(double *v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const df x = df_from(v[i]);
        reinterpret_cast<float2 *>(v)[i] = make_float2(x.h, x.l);
    }
}

// nrm[0] = |u_0| (start vector).
__global__ void __launch_bounds__(kLzThreads) lz_norm0_kernel(LzState st, LzGeom g) {
    const int b = blockIdx.y;
    const size_t plane = (size_t)g.H * g.P;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double n2 = 0.0;
    if (p < g.H * g.W) {
        const int y = p / g.W, x = p - y * g.W;
        const size_t off = (size_t)b * g.Lv * plane + (size_t)y * g.P + x;
        for (int l = 0; l < g.Lv; ++l) n2 += st.R0[off + l * plane] * st.R0[off + l * plane];
    }
    double tot;
    if (instance_reduce(n2, st.partial, st.counter, b, g.nblk, &tot)) st.nrm[(size_t)b * st.ld] = sqrt(tot);
}

// ---- extreme eigenvalues of symmetric tridiagonal matrices ----

constexpr int kRitzThreads = 128;

// Number of eigenvalues below x of the symmetric tridiagonal T with diagonal
// a[0..n) and squared off-diagonals c2 (c2[i] couples rows i-1 and i;
// c2[0] = 0), scaled so that its entries are at most 1 in magnitude, in
// double-float.  It is the number of negative pivots of T - x I = L D L^T,
// read off as the sign changes along the leading principal minors
// p_i = det(T_{0..i} - x I) = (a_i - x) p_{i-1} - c2_i p_{i-2} (no
// divisions).  A zero minor stands for the tiny pivot -2^-60 (a zero pivot
// counted negative, as in bisection with a minimum pivot), and the latest
// pair of minors is rescaled by 2^-+40 whenever both leave [2^-40, 2^40].
__device__ int sturm_count_df(const float2 *a, const float2 *c2, int n, df x) {
    int cnt = 0;
    bool neg_prev = false;
    df pm2 = {0.f, 0.f}, pm1 = {1.f, 0.f};
    for (int i = 0; i < n; ++i) {
        const float2 ai = a[i], ci = c2[i];
        const df d = df_add(df{ai.x, ai.y}, df{-x.h, -x.l});
        float ph = 0.f, pl = 0.f;
        acc_prod(ph, pl, d, pm1);
        acc_prod(ph, pl, df{-ci.x, -ci.y}, pm2);
        df pi = df_fast_two_sum(ph, pl);
        if (pi.h == 0.f) pi = df{-0x1p-60f * pm1.h, -0x1p-60f * pm1.l};
        const bool neg = pi.h < 0.f;
        cnt += neg != neg_prev;
        neg_prev = neg;
        const float m = fmaxf(fabsf(pi.h), fabsf(pm1.h));
        pm2 = pm1;
        pm1 = pi;
        if (m > 0x1p40f) {
            pm1 = df{pm1.h * 0x1p-40f, pm1.l * 0x1p-40f};
            pm2 = df{pm2.h * 0x1p-40f, pm2.l * 0x1p-40f};
        } else if (m < 0x1p-40f) {
            pm1 = df{pm1.h * 0x1p40f, pm1.l * 0x1p40f};
            pm2 = df{pm2.h * 0x1p40f, pm2.l * 0x1p40f};
        }
    }
    return cnt;
}

// Largest (want_max) or smallest eigenvalue of the symmetric tridiagonal
// (a, c2) in shared memory (FP64, overwritten by a scaled double-float copy),
// by multisection: each round the kRitzThreads threads of the block test as
// many interior points of the bracket.  Every thread of the block calls it
// and gets the same value.  A finite prev inside the Gershgorin interval
// bounds the wanted extreme from inside (by interlacing, the Ritz value of a
// shorter Lanczos run): the first round then tests points at growing
// distances beyond it, which brackets the extreme to about its change since
// prev and saves most of the rounds.
__device__ double tridiag_extreme(double *a, double *c2, int n, bool want_max, double prev, double *red) {
    const int tid = threadIdx.x;
    // Gershgorin interval
    double lo = INFINITY, hi = -INFINITY, amax = 0.0;
    for (int i = tid; i < n; i += kRitzThreads) {
        const double r = sqrt(c2[i]) + (i + 1 < n ? sqrt(c2[i + 1]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
        amax = fmax(amax, fabs(a[i]) + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if ((tid & 31) == 0) {
        red[tid >> 5] = lo;
        red[4 + (tid >> 5)] = hi;
        red[8 + (tid >> 5)] = amax;
    }
    __syncthreads();
    lo = fmin(fmin(red[0], red[1]), fmin(red[2], red[3]));
    hi = fmax(fmax(red[4], red[5]), fmax(red[6], red[7]));
    amax = fmax(fmax(red[8], red[9]), fmax(red[10], red[11]));
    // scale by a power of two sigma >= amax (exact), then to double-float in place
    int e = 0;
    frexp(amax, &e);
    const double sigma = amax > 0.0 && isfinite(amax) ? ldexp(1.0, e) : 1.0;
    const double is = 1.0 / sigma, is2 = is * is;
    float2 *af = reinterpret_cast<float2 *>(a), *cf = reinterpret_cast<float2 *>(c2);
    for (int i = tid; i < n; i += kRitzThreads) {
        const df x = df_from(a[i] * is), y = df_from(c2[i] * is2);
        af[i] = make_float2(x.h, x.l);
        cf[i] = make_float2(y.h, y.l);
    }
    __syncthreads();
    if (isfinite(prev) && prev > lo && prev < hi) {
        const double delta = fmax(fabs(prev), 1e-300) * 1e-14;
        const double sc = exp2(0.5 * tid);
        const double x = want_max ? prev + delta * sc : prev - delta * sc;
        const int cnt = sturm_count_df(af, cf, n, df_from(x * is));
        // the extreme lies beyond x: max <=> fewer than n below x; min <=> at least one below x
        const int nb = __syncthreads_count(want_max ? (cnt < n) : (cnt >= 1));
        const double inner = nb == 0 ? prev : prev + (want_max ? 1.0 : -1.0) * delta * exp2(0.5 * (nb - 1));
        const double outer = nb == kRitzThreads ? (want_max ? hi : lo)
                                                : prev + (want_max ? 1.0 : -1.0) * delta * exp2(0.5 * nb);
        if (want_max) {
            lo = inner;
            hi = fmin(outer, hi);
        } else {
            hi = inner;
            lo = fmax(outer, lo);
        }
    }
    for (int round = 0; round < 64; ++round) {
        if (!(hi - lo > 1e-13 * fmax(fabs(lo), fabs(hi)) + 1e-300)) break;
        const double step = (hi - lo) / (double)(kRitzThreads + 1);
        const double x = lo + step * (double)(tid + 1);
        const int cnt = sturm_count_df(af, cf, n, df_from(x * is));
        // "below the extreme" holds for a prefix of the points
        const int nb = __syncthreads_count(want_max ? (cnt < n) : (cnt < 1));
        const double nlo = nb > 0 ? lo + step * nb : lo;
        const double nhi = nb < kRitzThreads ? lo + step * (nb + 1) : hi;
        lo = nlo;
        hi = nhi;
    }
    return 0.5 * (lo + hi);
}

// Extreme eigenvalues of the Lanczos tridiagonal of each instance: block
// (b, 0) the largest, block (b, 1) the smallest.  With have_prev, rmin /
// rmax hold the values of a shorter run of the same instance.
__global__ void __launch_bounds__(kRitzThreads)
lz_ritz_kernel(const double *alpha, const double *beta, int ld, int kcur, const int *stop, int have_prev,
               double *rmin, double *rmax) {
    extern __shared__ double tri[];   // a[n], c2[n]
    __shared__ double red[12];
    const int b = blockIdx.x;
    const bool want_max = blockIdx.y == 0;
    int n = kcur;
    if (stop[b] && stop[b] < n) n = stop[b];
    if (n <= 0) return;
    double *a = tri, *c2 = tri + n;
    for (int i = threadIdx.x; i < n; i += kRitzThreads) {
        a[i] = alpha[(size_t)b * ld + i];
        const double c = i > 0 ? beta[(size_t)b * ld + i] : 0.0;   // beta_{i-1} = nrm[i]
        c2[i] = c * c;
    }
    __syncthreads();
    double *slot = want_max ? rmax + b : rmin + b;
    const double r = tridiag_extreme(a, c2, n, want_max, have_prev ? *slot : NAN, red);
    if (threadIdx.x == 0) *slot = r;
}

// Extreme eigenvalues nu_min, nu_max of C mu_s C (mu_s the symmetric part of
// mu, C the centring projector over labels), FP64.  Block 0 returns the
// largest, block 1 the smallest.  Warp 0 reduces the matrix to tridiagonal
// form by Householder reflections (lane i owns row i; reductions are
// shuffle-down trees broadcast from lane 0, so every lane uses the same
// values), then the block bisects.
__global__ void __launch_bounds__(kRitzThreads) mu_tilde_extremes_kernel(const float *mu, int L, double *nu) {
    __shared__ double A[kMaxLabels][kMaxLabels + 1];
    __shared__ double v[kMaxLabels], q[kMaxLabels], rm[kMaxLabels];
    __shared__ double a[kMaxLabels], c2[kMaxLabels];
    __shared__ double red[12];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        if (lane < L) {
            double r = 0.0;
            for (int j = 0; j < L; ++j) r += 0.5 * ((double)mu[lane * L + j] + (double)mu[j * L + lane]);
            rm[lane] = r / L;   // row mean of mu_s (= column mean: mu_s is symmetric)
        }
        __syncwarp();
        double tm = 0.0;
        for (int j = 0; j < L; ++j) tm += rm[j];
        tm /= L;
        if (lane < L)
            for (int j = 0; j < L; ++j)
                A[lane][j] = 0.5 * ((double)mu[lane * L + j] + (double)mu[j * L + lane]) - rm[lane] - rm[j] + tm;
        __syncwarp();
        for (int k = 0; k + 2 < L; ++k) {
            const double xi = (lane > k + 1 && lane < L) ? A[lane][k] : 0.0;
            const double tail = __shfl_sync(0xffffffffu, warp_sum(xi * xi), 0);
            if (tail == 0.0) continue;   // column k is already reduced
            const double x1 = A[k + 1][k];
            const double nrm = sqrt(x1 * x1 + tail);
            const double alpha = x1 > 0.0 ? -nrm : nrm;
            const double h = nrm * nrm - x1 * alpha;   // v^T v / 2
            const double vi = lane == k + 1 ? x1 - alpha : xi;
            v[lane] = vi;
            __syncwarp();
            double pi = 0.0;
            if (lane > k && lane < L) {
                for (int j = k + 1; j < L; ++j) pi = fma(A[lane][j], v[j], pi);
                pi /= h;
            }
            const double K = __shfl_sync(0xffffffffu, warp_sum(vi * pi), 0) / (2.0 * h);
            const double qi = pi - K * vi;
            q[lane] = qi;
            __syncwarp();
            if (lane > k && lane < L)
                for (int j = k + 1; j < L; ++j) A[lane][j] -= fma(vi, q[j], qi * v[j]);
            __syncwarp();
            if (lane > k + 1 && lane < L) {
                A[lane][k] = 0.0;
                A[k][lane] = 0.0;
            }
            if (lane == k + 1) {
                A[lane][k] = alpha;
                A[k][lane] = alpha;
            }
            __syncwarp();
        }
        if (lane < L) {
            a[lane] = A[lane][lane];
            c2[lane] = lane > 0 ? A[lane][lane - 1] * A[lane][lane - 1] : 0.0;
        }
    }
    __syncthreads();
    const bool want_max = blockIdx.x == 0;
    const double r = tridiag_extreme(a, c2, L, want_max, NAN, red);
    if (tid == 0) nu[want_max ? 1 : 0] = r;
}

// Lambda_b and eta_b = 1/(1 + max(Lambda_b, 0)).
__global__ void lz_finalize_kernel(const double *rmin, const double *rmax, const double *nu, int separable,
                                   int B, double *Lambda, float *eta) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double lam;
    if (separable) {
        const double p0 = rmax[b] * nu[1], p1 = rmax[b] * nu[0], p2 = rmin[b] * nu[1], p3 = rmin[b] * nu[0];
        lam = fmax(fmax(p0, p1), fmax(p2, p3));
    } else {
        lam = rmax[b];
    }
    Lambda[b] = lam;
    eta[b] = (float)(1.0 / (1.0 + (lam > 0.0 ? lam : 0.0)));
}

__global__ void set_lambda_zero_kernel(int B, double *Lambda, float *eta) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    Lambda[b] = 0.0;
    eta[b] = 1.0f;
}

}  // namespace

cudaError_t launch_mu_tilde_extremes(const float *mu_dev, int L, double *nu, cudaStream_t st) {
    mu_tilde_extremes_kernel<<<2, kRitzThreads, 0, st>>>(mu_dev, L, nu);
    return cudaGetLastError();
}

#define LZ_CHECK(x)                      \
    do {                                 \
        cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess) {         \
            rc = -3;                     \
            goto done;                   \
        }                                \
    } while (0)

int estimate_lipschitz_grid(const LipschitzJob &job, cudaStream_t st, int *steps_out,
                            long long *launches_out) {
    const int B = job.B;
    if (steps_out) *steps_out = 0;
    if (launches_out) *launches_out = 0;
    long long nl = 0;
    if (job.L <= 1) {
        set_lambda_zero_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, job.Lambda, job.eta);
        if (launches_out) *launches_out = 1;
        return cudaGetLastError() == cudaSuccess ? 0 : -3;
    }
    LzGeom g;
    g.B = B;
    g.L = job.L;
    g.Lv = job.mu_sym ? 1 : job.L;
    g.H = job.H;
    g.W = job.W;
    g.P = job.P;
    g.conn = job.conn;
    g.nblk = (job.H * job.W + kLzThreads - 1) / kLzThreads;
    const long long dim = (long long)job.H * job.W * (job.mu_sym ? 1 : (job.L - 1));
    const int kmax = (int)std::min<long long>(dim, (long long)job.max_steps);
    const int ld = kmax + 1;
    const size_t vec = (size_t)B * g.Lv * job.H * job.P;
    constexpr int kChunk = 96;   // steps per graph replay between convergence checks
    int rc = 0;
    LzState S{};
    double *rmin = nullptr, *rmax = nullptr, *nu = nullptr;
    double *wd = nullptr;        // FP64 edge weights (scalar form)
    float *mu_dev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_mu = nullptr, ev_nu = nullptr;
    std::vector<double> hmin(B), hmax(B), pmin(B, NAN), pmax(B, NAN);
    std::vector<int> hstop(B);
    int k = 0;
    int have_prev = 0;   // the Ritz values of the previous check bound the next ones
    // cooperative form (scalar W): one launch per chunk of steps
    bool coop = false;
    LzCoop C{};
    int habort = 0;
    unsigned *wmax = nullptr, hwmax = 0;
    const void *coop_fn = nullptr;
    int coop_chunk = 0;          // pixels per block (tiled form)
    size_t coop_smem = 0;
    const size_t nw = (size_t)B * job.H * job.W * (job.conn == 8 ? 4 : 2);
    dim3 gridp(g.nblk, B);
    const int nblk_dense = (job.W + kLzThreads / 32 - 1) / (kLzThreads / 32);
    S.ld = ld;
    LZ_CHECK(cudaMallocAsync((void **)&S.R0, vec * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.R1, vec * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.R2, vec * sizeof(double), st));
    LZ_CHECK(cudaMemsetAsync(S.R1, 0, vec * sizeof(double), st));
    LZ_CHECK(cudaMemsetAsync(S.R2, 0, vec * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.alpha, (size_t)B * ld * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.nrm, (size_t)B * (ld + 1) * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.partial,
                             (size_t)B * (g.nblk + job.W / (kLzThreads / 32) + 1) * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.counter, (size_t)(B + 1) * sizeof(unsigned), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.stop, (size_t)B * sizeof(int), st));
    LZ_CHECK(cudaMallocAsync((void **)&S.kdev, sizeof(int), st));
    LZ_CHECK(cudaMallocAsync((void **)&rmin, (size_t)B * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&rmax, (size_t)B * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&nu, 2 * sizeof(double), st));
    LZ_CHECK(cudaMallocAsync((void **)&mu_dev, (size_t)job.L * job.L * sizeof(float), st));
    if (!job.Kdense && g.Lv == 1) {
        // the weights' magnitude decides whether the double-float form fits
        LZ_CHECK(cudaMallocAsync((void **)&wmax, sizeof(unsigned), st));
        LZ_CHECK(cudaMemsetAsync(wmax, 0, sizeof(unsigned), st));
        lz_absmax_kernel<<<(int)std::min<size_t>((nw + 255) / 256, 1024), 256, 0, st>>>(job.w, nw, wmax);
        LZ_CHECK(cudaGetLastError());
        LZ_CHECK(cudaMemcpyAsync(&hwmax, wmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        nl += 1;
    }
    LZ_CHECK(cudaMemsetAsync(S.alpha, 0, (size_t)B * ld * sizeof(double), st));
    LZ_CHECK(cudaMemsetAsync(S.nrm, 0, (size_t)B * (ld + 1) * sizeof(double), st));
    LZ_CHECK(cudaMemsetAsync(S.counter, 0, (size_t)(B + 1) * sizeof(unsigned), st));
    LZ_CHECK(cudaMemsetAsync(S.stop, 0, (size_t)B * sizeof(int), st));
    LZ_CHECK(cudaMemsetAsync(S.kdev, 0, sizeof(int), st));
    LZ_CHECK(cudaMemcpyAsync(mu_dev, job.mu_host, (size_t)job.L * job.L * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    LZ_CHECK(cudaStreamSynchronize(st));  // mu_host is pageable and owned by the caller

    if (!job.Kdense && g.Lv == 1) {
        // double-float vectors need |w| well inside the FP32 range (products
        // and squared norms stay finite, low parts stay normal); all blocks
        // of the cooperative launch must be resident at once: at most one per
        // SM and instance
        float wm = 0.f;
        std::memcpy(&wm, &hwmax, sizeof(float));
        int dev = 0, sms = 0, coop_ok = 0, occ = 0;
        LZ_CHECK(cudaGetDevice(&dev));
        LZ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LZ_CHECK(cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, dev));
        const int N = job.H * job.W;
        const int need = (N + kCoopThreads - 1) / kCoopThreads;
        // two SMs stay free for the label-space eigen-solve on the side stream
        const int avail = job.mu_sym && sms > 4 ? sms - 2 : sms;
        C.gx = std::max(1, std::min(need, B <= avail ? avail / B : 1));
        // contiguous pixel ranges staged in shared memory with their halo
        // rows when both fit (at most 8 pixels per worker thread); else the
        // strided form with every vector in L2
        coop_chunk = (N + C.gx - 1) / C.gx;
        const long long ppt = (coop_chunk + kCoopWorkers - 1) / kCoopWorkers;
        // weights (4 floats) and two double-float vectors per staged pixel
        coop_smem = (size_t)(coop_chunk + 4 * ((long long)job.W + 1)) * (4 * sizeof(float) + 2 * sizeof(float2));
        if (ppt > 8 || coop_smem > (size_t)220 * 1024) {
            coop_fn = (const void *)lz_chunk_strided_kernel;
            coop_smem = 0;
        } else {
            const bool c8 = job.conn == 8;
            coop_fn = ppt <= 1   ? (c8 ? (const void *)lz_chunk_halo_kernel<1, 4> : (const void *)lz_chunk_halo_kernel<1, 2>)
                      : ppt <= 2 ? (c8 ? (const void *)lz_chunk_halo_kernel<2, 4> : (const void *)lz_chunk_halo_kernel<2, 2>)
                      : ppt <= 4 ? (c8 ? (const void *)lz_chunk_halo_kernel<4, 4> : (const void *)lz_chunk_halo_kernel<4, 2>)
                                 : (c8 ? (const void *)lz_chunk_halo_kernel<8, 4> : (const void *)lz_chunk_halo_kernel<8, 2>);
            LZ_CHECK(cudaFuncSetAttribute(coop_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)coop_smem));
        }
        LZ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, coop_fn, kCoopThreads, coop_smem));
        if (coop_ok && occ >= 1 && B <= sms * occ && wm >= 0x1p-40f && wm <= 0x1p40f) {
            coop = true;
        } else {
            LZ_CHECK(cudaMallocAsync((void **)&wd, nw * sizeof(double), st));
            lz_weights_f64_kernel<<<(int)std::min<size_t>((nw + 255) / 256, 4096), 256, 0, st>>>(job.w, wd, nw);
            LZ_CHECK(cudaGetLastError());
            nl += 1;
        }
    }

    lz_init_kernel<<<gridp, kLzThreads, 0, st>>>(S.R0, g, 0x5eed5eedull);
    LZ_CHECK(cudaGetLastError());
    lz_norm0_kernel<<<gridp, kLzThreads, 0, st>>>(S, g);
    LZ_CHECK(cudaGetLastError());
    nl += 2;
    if (coop) {
        lz_split_kernel<<<(int)std::min<size_t>((vec + 255) / 256, 4096), 256, 0, st>>>(S.R0, vec);
        LZ_CHECK(cudaGetLastError());
        nl += 1;
    }

    LZ_CHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    if (coop) {
        LZ_CHECK(cudaMallocAsync((void **)&C.bar, 2 * sizeof(unsigned), st));
        LZ_CHECK(cudaMallocAsync((void **)&C.abort, sizeof(int), st));
        LZ_CHECK(cudaMallocAsync((void **)&C.part, (size_t)2 * B * C.gx * sizeof(double), st));
        LZ_CHECK(cudaMemsetAsync(C.bar, 0, 2 * sizeof(unsigned), st));
        LZ_CHECK(cudaMemsetAsync(C.abort, 0, sizeof(int), st));
    } else {
        // one graph of kChunk steps, captured once and replayed
        LZ_CHECK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < kChunk; ++i) {
            if (job.Kdense)
                lz_step_a_dense_kernel<<<dim3(nblk_dense, B), kLzThreads, 0, cap>>>(S, job.Kdense, g, nblk_dense);
            else if (g.Lv == 1)
                lz_step_a_scalar_kernel<<<gridp, kLzThreads, 0, cap>>>(S, wd, g);
            else
                lz_step_a_kernel<<<gridp, kLzThreads, 0, cap>>>(S, job.w, mu_dev, g);
            lz_step_b_kernel<<<gridp, kLzThreads, 0, cap>>>(S, g);
        }
        LZ_CHECK(cudaStreamEndCapture(cap, &graph));
        LZ_CHECK(cudaGraphInstantiate(&exec, graph, 0));
    }
    LZ_CHECK(cudaFuncSetAttribute(lz_ritz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * ld * sizeof(double))));
    if (job.mu_sym) {
        // the small eigen-solve of C mu C runs on the side stream, overlapped
        // with the Lanczos steps (it only needs mu, copied above)
        LZ_CHECK(cudaEventCreateWithFlags(&ev_mu, cudaEventDisableTiming));
        LZ_CHECK(cudaEventCreateWithFlags(&ev_nu, cudaEventDisableTiming));
        LZ_CHECK(cudaEventRecord(ev_mu, st));
        LZ_CHECK(cudaStreamWaitEvent(cap, ev_mu, 0));
        mu_tilde_extremes_kernel<<<2, kRitzThreads, 0, cap>>>(mu_dev, job.L, nu);
        LZ_CHECK(cudaGetLastError());
        LZ_CHECK(cudaEventRecord(ev_nu, cap));
    }
    while (k < kmax) {
        if (coop) {
            int k0 = k, k1 = std::min(k + kChunk, kmax);
            const float *wf = job.w;
            int chunk = coop_chunk;
            void *args[] = {&S, &wf, &g, &C, &k0, &k1, &chunk};
            LZ_CHECK(cudaLaunchCooperativeKernel(coop_fn, dim3(C.gx, B), dim3(kCoopThreads), args, coop_smem, st));
            nl += 1;
        } else {
            LZ_CHECK(cudaGraphLaunch(exec, st));
            nl += 2 * kChunk;
        }
        k = std::min(k + kChunk, kmax);
        lz_ritz_kernel<<<dim3(B, 2), kRitzThreads, 2 * ld * sizeof(double), st>>>(S.alpha, S.nrm, ld, k, S.stop,
                                                                                  have_prev, rmin, rmax);
        have_prev = 1;
        LZ_CHECK(cudaGetLastError());
        nl += 1;
        LZ_CHECK(cudaMemcpyAsync(hmin.data(), rmin, B * sizeof(double), cudaMemcpyDeviceToHost, st));
        LZ_CHECK(cudaMemcpyAsync(hmax.data(), rmax, B * sizeof(double), cudaMemcpyDeviceToHost, st));
        LZ_CHECK(cudaMemcpyAsync(hstop.data(), S.stop, B * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (coop) LZ_CHECK(cudaMemcpyAsync(&habort, C.abort, sizeof(int), cudaMemcpyDeviceToHost, st));
        LZ_CHECK(cudaStreamSynchronize(st));
        if (habort != 0) {
            rc = -5;   // a barrier wait ran out
            goto done;
        }
        bool all = true;
        for (int b = 0; b < B; ++b) {
            const double sc = fmax(fmax(fabs(hmin[b]), fabs(hmax[b])), 1e-300);
            const bool conv = hstop[b] != 0 || (fabs(hmax[b] - pmax[b]) <= job.tol * sc &&
                                                fabs(hmin[b] - pmin[b]) <= job.tol * sc);
            all = all && conv;
            pmin[b] = hmin[b];
            pmax[b] = hmax[b];
        }
        if (all) break;
    }
    if (job.mu_sym) LZ_CHECK(cudaStreamWaitEvent(st, ev_nu, 0));
    lz_finalize_kernel<<<(B + 127) / 128, 128, 0, st>>>(rmin, rmax, nu, job.mu_sym ? 1 : 0, B, job.Lambda,
                                                      job.eta);
    LZ_CHECK(cudaGetLastError());
    nl += job.mu_sym ? 2 : 1;
    if (steps_out) *steps_out = k;
    if (launches_out) *launches_out = nl;
done:
    if (ev_mu) cudaEventDestroy(ev_mu);
    if (ev_nu) cudaEventDestroy(ev_nu);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    double *ds[] = {S.R0, S.R1, S.R2, S.alpha, S.nrm, S.partial, rmin, rmax, nu, wd};
    for (double *p : ds)
        if (p) cudaFreeAsync(p, st);
    if (S.counter) cudaFreeAsync(S.counter, st);
    if (S.stop) cudaFreeAsync(S.stop, st);
    if (S.kdev) cudaFreeAsync(S.kdev, st);
    if (wmax) cudaFreeAsync(wmax, st);
    if (C.bar) cudaFreeAsync(C.bar, st);
    if (C.abort) cudaFreeAsync(C.abort, st);
    if (C.part) cudaFreeAsync(C.part, st);
    if (mu_dev) cudaFreeAsync(mu_dev, st);
    return rc;
}

}  // namespace proxmf
