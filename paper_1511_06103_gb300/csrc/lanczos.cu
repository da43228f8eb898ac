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

// Sturm count: number of eigenvalues of the symmetric tridiagonal (a, c) < x.
__device__ int sturm_count(const double *a, const double *c, int n, double x, double pivmin) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
        const double off = i > 0 ? c[i - 1] * c[i - 1] / d : 0.0;
        d = a[i] - x - off;
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Extreme eigenvalues of the Lanczos tridiagonal of each instance, by
// multisection: warp 0 finds the largest, warp 1 the smallest; each round the
// 32 lanes test 32 interior points of the bracket.  With have_prev, the
// values in rmin / rmax come from a shorter tridiagonal of the same run: by
// interlacing they bound the new extremes from inside (the largest can only
// grow, the smallest only shrink), so the first round tests points at
// geometrically growing distances beyond them, which brackets the new value
// to about its change since the last check and saves most rounds of FP64
// Sturm sequences.
__global__ void lz_ritz_kernel(const double *alpha, const double *beta, int ld, int kcur, const int *stop,
                               int have_prev, double *rmin, double *rmax) {
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int n = kcur;
    if (stop[b] && stop[b] < n) n = stop[b];
    if (n <= 0) return;
    const double *a = alpha + (size_t)b * ld;
    const double *c = beta + (size_t)b * ld + 1;   // beta_k = nrm[k+1]
    double lo = INFINITY, hi = -INFINITY, amax = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? fabs(c[i - 1]) : 0.0) + (i + 1 < n ? fabs(c[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
        amax = fmax(amax, fabs(a[i]) + r);
    }
    const double pivmin = 1e-300 + amax * 1e-300;
    const bool want_max = wid == 0;
    if (have_prev) {
        const double prev = want_max ? rmax[b] : rmin[b];
        if (isfinite(prev) && prev > lo && prev < hi) {
            const double delta = fmax(fabs(prev), 1e-300) * 1e-14;
            const double x = want_max ? prev + delta * ldexp(1.0, lane) : prev - delta * ldexp(1.0, lane);
            const int cnt = sturm_count(a, c, n, x, pivmin);
            // max: the extreme lies beyond x  <=>  cnt < n ; min: <=> cnt >= 1... (cnt < 1 below x)
            const bool beyond = want_max ? (cnt < n) : (cnt >= 1);
            const unsigned m = __ballot_sync(0xffffffffu, beyond);
            const int nb = __popc(m);   // the extreme lies beyond the first nb points
            const double inner = nb == 0 ? prev : (want_max ? prev + delta * ldexp(1.0, nb - 1)
                                                             : prev - delta * ldexp(1.0, nb - 1));
            const double outer = nb == 32 ? (want_max ? hi : lo)
                                          : (want_max ? prev + delta * ldexp(1.0, nb) : prev - delta * ldexp(1.0, nb));
            if (want_max) {
                lo = inner;
                hi = fmin(outer, hi);
            } else {
                hi = inner;
                lo = fmax(outer, lo);
            }
        }
    }
    for (int round = 0; round < 64; ++round) {
        if (!(hi - lo > 1e-14 * fmax(fabs(lo), fabs(hi)) + 1e-300)) break;
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const int cnt = sturm_count(a, c, n, x, pivmin);
        // max: lambda_max >= x  <=>  cnt < n ; min: lambda_min < x  <=>  cnt >= 1
        const bool below = want_max ? (cnt < n) : (cnt < 1);
        const unsigned m = __ballot_sync(0xffffffffu, below);
        // "below" holds for a prefix of lanes (counts grow with x)
        const int nb = __popc(m);
        const double step = (hi - lo) / 33.0;
        const double nlo = nb > 0 ? lo + step * nb : lo;
        const double nhi = nb < 32 ? lo + step * (nb + 1) : hi;
        lo = nlo;
        hi = nhi;
    }
    __syncthreads();   // both warps have read their previous values
    if (lane == 0) {
        if (want_max)
            rmax[b] = 0.5 * (lo + hi);
        else
            rmin[b] = 0.5 * (lo + hi);
    }
}

// Extreme eigenvalues of C mu C (L x L, symmetric part) by cyclic Jacobi.
// One warp: lane 0 computes each rotation, all lanes apply it to the rows and
// columns of the matrix held in shared memory.
__global__ void mu_tilde_extremes_kernel(const float *mu, int L, double *nu) {
    __shared__ double A[kMaxLabels * kMaxLabels];
    __shared__ double rm[kMaxLabels], cm[kMaxLabels];
    __shared__ double cs_sn[2];
    __shared__ int stop_flag;
    const int lane = threadIdx.x;
    if (lane < L) {
        double r = 0.0, c = 0.0;
        for (int j = 0; j < L; ++j) {
            r += 0.5 * ((double)mu[lane * L + j] + (double)mu[j * L + lane]) / L;
            c += 0.5 * ((double)mu[j * L + lane] + (double)mu[lane * L + j]) / L;
        }
        rm[lane] = r;
        cm[lane] = c;
    }
    __syncwarp();
    double tm = 0.0;
    for (int j = 0; j < L; ++j) tm += rm[j] / L;
    for (int i = 0; i < L; ++i)
        if (lane < L)
            A[i * L + lane] =
                0.5 * ((double)mu[i * L + lane] + (double)mu[lane * L + i]) - rm[i] - cm[lane] + tm;
    __syncwarp();
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        if (lane < L)
            for (int j = 0; j < L; ++j) {
                const double v = A[lane * L + j] * A[lane * L + j];
                tot += v;
                if (j != lane) off += v;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        // off-diagonal mass below (1e-13 |A|)^2: the diagonal then holds the
        // eigenvalues to ~1e-26 relative (the error is second order in it)
        if (off <= 1e-26 * (tot > 0 ? tot : 1.0)) break;
        const double tiny = 1e-18 * sqrt(tot);
        for (int p = 0; p < L; ++p)
            for (int r = p + 1; r < L; ++r) {
                if (lane == 0) {
                    const double apr = A[p * L + r];
                    if (fabs(apr) <= tiny) {
                        stop_flag = 1;
                    } else {
                        stop_flag = 0;
                        const double theta = (A[r * L + r] - A[p * L + p]) / (2.0 * apr);
                        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        const double c = 1.0 / sqrt(t * t + 1.0);
                        cs_sn[0] = c;
                        cs_sn[1] = t * c;
                    }
                }
                __syncwarp();
                if (stop_flag) {
                    __syncwarp();
                    continue;
                }
                const double c = cs_sn[0], sn = cs_sn[1];
                if (lane < L) {
                    const double akp = A[lane * L + p], akr = A[lane * L + r];
                    A[lane * L + p] = c * akp - sn * akr;
                    A[lane * L + r] = sn * akp + c * akr;
                }
                __syncwarp();
                if (lane < L) {
                    const double apk = A[p * L + lane], ark = A[r * L + lane];
                    A[p * L + lane] = c * apk - sn * ark;
                    A[r * L + lane] = sn * apk + c * ark;
                }
                __syncwarp();
            }
    }
    if (lane == 0) {
        double lo = INFINITY, hi = -INFINITY;
        for (int i = 0; i < L; ++i) {
            lo = fmin(lo, A[i * L + i]);
            hi = fmax(hi, A[i * L + i]);
        }
        nu[0] = lo;
        nu[1] = hi;
    }
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
    mu_tilde_extremes_kernel<<<1, 32, 0, st>>>(mu_dev, L, nu);
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

    // one graph of kChunk steps, captured once and replayed
    LZ_CHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
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
    if (job.mu_sym) {
        // the small eigen-solve of C mu C runs on the side stream, overlapped
        // with the Lanczos steps (it only needs mu, copied above)
        LZ_CHECK(cudaEventCreateWithFlags(&ev_mu, cudaEventDisableTiming));
        LZ_CHECK(cudaEventCreateWithFlags(&ev_nu, cudaEventDisableTiming));
        LZ_CHECK(cudaEventRecord(ev_mu, st));
        LZ_CHECK(cudaStreamWaitEvent(cap, ev_mu, 0));
        mu_tilde_extremes_kernel<<<1, 32, 0, cap>>>(mu_dev, job.L, nu);
        LZ_CHECK(cudaGetLastError());
        LZ_CHECK(cudaEventRecord(ev_nu, cap));
    }
    while (k < kmax) {
        LZ_CHECK(cudaGraphLaunch(exec, st));
        nl += 2 * kChunk;
        k = std::min(k + kChunk, kmax);
        lz_ritz_kernel<<<B, 64, 0, st>>>(S.alpha, S.nrm, ld, k, S.stop, have_prev, rmin, rmax);
        have_prev = 1;
        LZ_CHECK(cudaGetLastError());
        nl += 1;
        LZ_CHECK(cudaMemcpyAsync(hmin.data(), rmin, B * sizeof(double), cudaMemcpyDeviceToHost, st));
        LZ_CHECK(cudaMemcpyAsync(hmax.data(), rmax, B * sizeof(double), cudaMemcpyDeviceToHost, st));
        LZ_CHECK(cudaMemcpyAsync(hstop.data(), S.stop, B * sizeof(int), cudaMemcpyDeviceToHost, st));
        LZ_CHECK(cudaStreamSynchronize(st));
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
    if (mu_dev) cudaFreeAsync(mu_dev, st);
    return rc;
}

}  // namespace proxmf
