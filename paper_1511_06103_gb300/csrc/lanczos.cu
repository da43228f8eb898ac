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
#include <vector>

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
        const double ref = fabs(st.alpha[(size_t)b * st.ld + k]) + st.nrm[(size_t)b * st.ld + k];
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
// are block partials summed in a fixed order by every block after a grid
// barrier, so all blocks hold the same alpha_k and beta_k and no launch or
// last-block tail separates the steps.  1/|u_k| and the recurrence
// coefficients are formed once per block and step: FP64 division is a long
// sequence on the narrow FP64 pipe of this part.

constexpr int kCoopThreads = 512;
constexpr long long kLzWaitCycles = 4000000000ll;   // ~2 s at 2 GHz per barrier wait

struct LzCoop {
    unsigned *bar;   // [0] arrivals, [1] generation
    int *abort;      // set once a barrier wait ran out; every later barrier fails
    double *part;    // [2][B][gx] block partials of alpha_k and |u_{k+1}|^2
    int gx;          // blocks per instance
};

// Grid-wide barrier of a cooperative launch with a bounded wait.  Thread 0
// arrives on the counter; the last arrival resets it and advances the
// generation word that the others poll.  Returns false in every thread of
// the block when this or another block's wait ran out.
__device__ bool coop_barrier(const LzCoop &c, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = c.bar + 1;
        volatile int *ab = c.abort;
        int good = *ab == 0;
        if (good) {
            const unsigned g0 = *gen;
            __threadfence();
            if (atomicAdd(c.bar, 1u) == nblocks - 1) {
                atomicExch(c.bar, 0u);
                __threadfence();
                atomicAdd(c.bar + 1, 1u);
            } else {
                const long long t0 = clock64();
                while (*gen == g0) {
                    if (*ab != 0) {
                        good = 0;
                        break;
                    }
                    if (clock64() - t0 > kLzWaitCycles) {
                        atomicExch(c.abort, 1);
                        good = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Sum of n partials in a fixed order (strided per thread, fixed-shape warp
// tree, warps in index order); every thread gets the same value.
__device__ double coop_sum(const double *p, int n, double *red, double *out) {
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += kCoopThreads) a += __ldcg(p + i);
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kCoopThreads / 32; ++k) s += red[k];
        *out = s;
    }
    __syncthreads();
    return *out;
}

// Block total of v into part[slot] (thread 0 writes).
__device__ void coop_partial(double v, double *red, double *part) {
    v = warp_sum(v);
    __syncthreads();   // red may still be read by a previous coop_sum
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kCoopThreads / 32; ++k) s += red[k];
        __stcg(part, s);
    }
}

// Steps k0 .. k1-1 of the scalar form (t = W v_k, symmetric weighted
// adjacency of the grid), same recurrence and stopping rule as the
// two-kernel form above.  Vectors written inside the launch are read through
// L2 only (__ldcg): L1 is not coherent across blocks.
__global__ void __launch_bounds__(kCoopThreads, 1)
lz_chunk_scalar_kernel(LzState st, const double *__restrict__ w, LzGeom g, LzCoop c, int k0, int k1) {
    __shared__ double red[kCoopThreads / 32];
    __shared__ double sh[4];
    const int b = blockIdx.y, bx = blockIdx.x, tid = threadIdx.x;
    const unsigned nblocks = gridDim.x * gridDim.y;
    const int N = g.H * g.W;
    const int nd = g.conn == 8 ? 4 : 2;
    const size_t base = (size_t)b * N;
    const double *wb = w + base * nd;
    double *pa = c.part + (size_t)b * c.gx;
    double *pb = c.part + ((size_t)g.B + b) * c.gx;
    const size_t ld = (size_t)st.ld;
    bool active = st.stop[b] == 0;
    double nk = st.nrm[b * ld + k0];   // |u_k|
    if (tid == 0) {
        sh[0] = active ? 1.0 / nk : 0.0;
        sh[1] = active && k0 > 0 ? nk / st.nrm[b * ld + k0 - 1] : 0.0;
    }
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const double inv = sh[0], cm = sh[1];
        const double *v = lz_buf(st, k % 3) + base;
        double *t = lz_buf(st, (k + 1) % 3) + base;
        const double *um = lz_buf(st, (k + 2) % 3) + base;
        // t = W v_k and the partial of alpha_k = v_k . t
        double dot = 0.0;
        if (active) {
            for (int p = bx * kCoopThreads + tid; p < N; p += c.gx * kCoopThreads) {
                const int y = p / g.W, x = p - y * g.W;
                double acc = 0.0;
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    if (d >= nd) break;
                    const int dy = d == 0 ? 0 : 1, dx = d == 0 ? 1 : (d == 1 ? 0 : (d == 2 ? 1 : -1));
                    const int yo = y + dy, xo = x + dx;
                    if (yo < g.H && xo >= 0 && xo < g.W)
                        acc = fma(__ldg(wb + (size_t)p * nd + d), __ldcg(v + (size_t)yo * g.W + xo), acc);
                    const int yi = y - dy, xi = x - dx;
                    if (yi >= 0 && xi >= 0 && xi < g.W) {
                        const size_t q = (size_t)yi * g.W + xi;
                        acc = fma(__ldg(wb + q * nd + d), __ldcg(v + q), acc);
                    }
                }
                const double r = acc * inv;
                __stcg(t + p, r);
                dot = fma(r, __ldcg(v + p), dot);
            }
        }
        coop_partial(dot * inv, red, pa + bx);
        if (!coop_barrier(c, nblocks)) return;
        const double alpha = coop_sum(pa, c.gx, red, sh + 2);
        // u_{k+1} = t - alpha_k v_k - |u_k| v_{k-1} and its squared norm
        double n2 = 0.0;
        if (active) {
            const double ca = alpha * inv;
            for (int p = bx * kCoopThreads + tid; p < N; p += c.gx * kCoopThreads) {
                double r = fma(-ca, __ldcg(v + p), __ldcg(t + p));
                if (k > 0) r = fma(-cm, __ldcg(um + p), r);
                __stcg(t + p, r);
                n2 = fma(r, r, n2);
            }
        }
        coop_partial(n2, red, pb + bx);
        if (!coop_barrier(c, nblocks)) return;
        const double s = coop_sum(pb, c.gx, red, sh + 3);
        if (active) {
            // every block derives the same values from the same sums
            if (tid == 0) {
                const double bk = sqrt(s);
                const double ref = fabs(alpha) + nk;
                const bool brk = !(bk > 1e-13 * ref) || !(bk > 1e-300);
                if (bx == 0) {
                    st.alpha[b * ld + k] = alpha;
                    st.nrm[b * ld + k + 1] = bk;
                    if (brk) st.stop[b] = k + 1;
                }
                sh[0] = brk ? 0.0 : 1.0 / bk;
                sh[1] = bk / nk;
                sh[2] = brk ? 1.0 : 0.0;
                sh[3] = bk;
            }
            __syncthreads();
            if (sh[2] != 0.0) active = false;
            nk = sh[3];
            __syncthreads();   // sh is rewritten by the next step's sums
        }
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
// c2[0] = 0).  It is the number of negative pivots of T - x I = L D L^T,
// read off as the sign changes along the leading principal minors
// p_i = det(T_{0..i} - x I) = (a_i - x) p_{i-1} - c2_i p_{i-2}: three FP64
// operations per row and no division (FP64 division is a long sequence on
// the narrow FP64 pipe).  A zero minor stands for the tiny pivot -tiny (a
// zero pivot counted negative, as in bisection with a minimum pivot), and
// the latest pair of minors is rescaled by 2^-+448 whenever both leave
// [2^-448, 2^448]; signs and exponents are read as integers.
__device__ int sturm_count_minors(const double *a, const double *c2, int n, double x, double tiny) {
    int cnt = 0;
    bool neg_prev = false;
    double pm2 = 0.0, pm1 = 1.0;
    for (int i = 0; i < n; ++i) {
        double pi = fma(a[i] - x, pm1, -c2[i] * pm2);
        if ((__double_as_longlong(pi) << 1) == 0) pi = -tiny * pm1;
        const int hi = __double2hiint(pi), hm = __double2hiint(pm1);
        const bool neg = hi < 0;
        cnt += neg != neg_prev;
        neg_prev = neg;
        const int em = max((hi >> 20) & 0x7FF, (hm >> 20) & 0x7FF);
        pm2 = pm1;
        pm1 = pi;
        if (em > 1023 + 448) {
            pm1 *= 0x1p-448;
            pm2 *= 0x1p-448;
        } else if (em < 1023 - 448) {
            pm1 *= 0x1p+448;
            pm2 *= 0x1p+448;
        }
    }
    return cnt;
}

// Largest (want_max) or smallest eigenvalue of the symmetric tridiagonal
// (a, c2) in shared memory, by multisection: each round the kRitzThreads
// threads of the block test as many interior points of the bracket.  Every
// thread of the block calls it and gets the same value.  A finite prev
// inside the Gershgorin interval bounds the wanted extreme from inside (by
// interlacing, the Ritz value of a shorter Lanczos run): the first round then
// tests points at growing distances beyond it, which brackets the extreme to
// about its change since prev and saves most of the rounds.
__device__ double tridiag_extreme(const double *a, const double *c2, int n, bool want_max, double prev,
                                  double *red) {
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
    const double tiny = fmax(amax, 1e-280) * 0x1p-200;
    if (isfinite(prev) && prev > lo && prev < hi) {
        const double delta = fmax(fabs(prev), 1e-300) * 1e-14;
        const double sc = exp2(0.5 * tid);
        const double x = want_max ? prev + delta * sc : prev - delta * sc;
        const int cnt = sturm_count_minors(a, c2, n, x, tiny);
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
        if (!(hi - lo > 1e-14 * fmax(fabs(lo), fabs(hi)) + 1e-300)) break;
        const double step = (hi - lo) / (double)(kRitzThreads + 1);
        const double x = lo + step * (double)(tid + 1);
        const int cnt = sturm_count_minors(a, c2, n, x, tiny);
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
        const size_t nw = (size_t)B * job.H * job.W * (job.conn == 8 ? 4 : 2);
        LZ_CHECK(cudaMallocAsync((void **)&wd, nw * sizeof(double), st));
        lz_weights_f64_kernel<<<(int)std::min<size_t>((nw + 255) / 256, 4096), 256, 0, st>>>(job.w, wd, nw);
        LZ_CHECK(cudaGetLastError());
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

    lz_init_kernel<<<gridp, kLzThreads, 0, st>>>(S.R0, g, 0x5eed5eedull);
    LZ_CHECK(cudaGetLastError());
    lz_norm0_kernel<<<gridp, kLzThreads, 0, st>>>(S, g);
    LZ_CHECK(cudaGetLastError());
    nl += 2;

    LZ_CHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    if (!job.Kdense && g.Lv == 1) {
        // all blocks must be resident at once: at most one per SM and instance
        int dev = 0, sms = 0, coop_ok = 0, occ = 0;
        LZ_CHECK(cudaGetDevice(&dev));
        LZ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LZ_CHECK(cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, dev));
        LZ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lz_chunk_scalar_kernel, kCoopThreads, 0));
        const int need = (job.H * job.W + kCoopThreads - 1) / kCoopThreads;
        if (coop_ok && occ >= 1 && B <= sms * occ) {
            C.gx = std::max(1, std::min(need, B <= sms ? sms / B : 1));
            coop = true;
        }
    }
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
            void *args[] = {&S, &wd, &g, &C, &k0, &k1};
            LZ_CHECK(cudaLaunchCooperativeKernel((const void *)lz_chunk_scalar_kernel, dim3(C.gx, B),
                                                 dim3(kCoopThreads), args, 0, st));
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
    if (C.bar) cudaFreeAsync(C.bar, st);
    if (C.abort) cudaFreeAsync(C.abort, st);
    if (C.part) cudaFreeAsync(C.part, st);
    if (mu_dev) cudaFreeAsync(mu_dev, st);
    return rc;
}

}  // namespace proxmf
