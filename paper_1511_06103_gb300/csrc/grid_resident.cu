// grid_resident.cu -- the whole iteration loop of a small grid instance in one
// launch: a thread-block cluster per instance (up to 8 CTAs, each owning a
// slab of rows) holds log q and q of the current and the next iterate in
// shared memory and runs every step of the parallel proximal update (Sec. 3,
// Eq. method:update_natural) with its free energy (Eq. mf-objective) and
// stopping rule, with a cluster barrier between steps instead of a kernel
// launch.  Small solves (a 64 x 64 binary denoising grid, 50 steps) are
// bound by launch latency otherwise.
//
// Per step and pixel: the weighted neighbour sums S_out (edges leaving the
// pixel) and S_in (edges entering it) of q, m = mu S_out + mu^T S_in (one
// product of mu with S_out + S_in when mu is symmetric), the pixel's term
// q . (U + m / 2 + log q) of F(q^t), and the update
//   a = -eta (U + m) + (1 - eta) log q,   log q' = a - logsumexp(a).
// F is summed in double-float (pairs of floats: FP64 is the narrow pipe of
// this part and one SM does all the work) and reduced in a fixed order; thread 0
// records it, applies the stopping rule |F_t - F_{t-1}| <= rel_tol |F_t|
// (the instance then stops after this step's update, as in the tiled form)
// and flags a non-finite F.  The final log q goes to the buffer in which the
// tiled form would leave it.
#include <cooperative_groups.h>

#include <cmath>

#include "dfloat.cuh"
#include "internal.h"

namespace proxmf {

namespace {

namespace cg = cooperative_groups;

// Cluster of up to 8 CTAs per instance; CTA r of the cluster owns rows
// [r * rows, min(H, (r + 1) * rows)) and keeps log q and q of them (current
// and next iterate) in its shared memory.  Neighbour rows of the adjacent
// CTAs are read through distributed shared memory; one cluster barrier per
// step publishes the new iterate and the CTAs' free-energy partials, which
// every CTA then sums in rank order (so all of them take the same stopping
// decision).
template <int LT, int NT>
__global__ void __launch_bounds__(NT, 1) grid_resident_kernel(const GridResidentLaunch a) {
    extern __shared__ float rsm[];
    __shared__ float red_h[NT / 32], red_l[NT / 32];
    __shared__ float part_h[2], part_l[2];   // this CTA's F partial, by step parity
    __shared__ int stop_flag;
    cg::cluster_group cluster = cg::this_cluster();
    const int nc = (int)cluster.num_blocks(), r = (int)cluster.block_rank();
    const int b = blockIdx.y, tid = threadIdx.x;
    const int H = a.H, W = a.W, L = a.L, LP = a.LP;
    const int nd = a.conn == 8 ? 4 : 2;
    const int rows = (H + nc - 1) / nc;
    const int y0 = min(H, r * rows), y1 = min(H, y0 + rows);
    const int npix = (y1 - y0) * W;
    const int NLc = rows * W * LP;              // slab floats per array
    float *sA = rsm, *qA = sA + NLc, *sB = qA + NLc, *qB = sB + NLc, *mus = qB + NLc;
    const size_t gbase = ((size_t)b * H + y0) * W * LP;   // first own value in the global arrays
    const float *Ub = a.U + gbase;
    const float *wb = a.w + (size_t)b * H * W * nd;
    const float eta = a.eta[b];
    for (int i = tid; i < npix * LP; i += NT) {
        const bool live = i % LP < L;
        const float s = a.s_in[gbase + i];
        sA[i] = s;
        qA[i] = live ? __expf(s) : 0.f;
        sB[i] = live ? 0.f : kPadLogQ;
        qB[i] = 0.f;
    }
    for (int i = tid; i < L * L; i += NT) mus[i] = a.mu[i];
    if (tid == 0) stop_flag = 0;
    cluster.sync();   // every slab is loaded before any neighbour reads it

    float *sc = sA, *qc = qA, *sn = sB, *qn = qB;
    double f_prev = 0.0;   // thread 0
    for (int t = 0; t < a.nsteps; ++t) {
        // q of the row above / below the slab, in the adjacent CTAs
        const float *q_up = r > 0 ? cluster.map_shared_rank(qc, r - 1) : nullptr;
        const float *q_dn = r + 1 < nc ? cluster.map_shared_rank(qc, r + 1) : nullptr;
        float fh = 0.f, fl = 0.f;   // compensated sum of the pixel terms (double-float)
        for (int lp = tid; lp < npix; lp += NT) {
            const int ly = lp / W, x = lp - ly * W, y = y0 + ly;
            float So[LT], Si[LT];
#pragma unroll
            for (int l = 0; l < LT; ++l) So[l] = Si[l] = 0.f;
            for (int d = 0; d < nd; ++d) {
                const int dy = d == 0 ? 0 : 1, dx = d == 0 ? 1 : (d == 1 ? 0 : (d == 2 ? 1 : -1));
                const int yo = y + dy, xo = x + dx;
                if (yo < H && xo >= 0 && xo < W) {
                    const float wv = wb[((size_t)y * W + x) * nd + d];
                    // rows below the slab live in the next CTA (its row 0)
                    const float *qr = yo < y1 ? qc + ((yo - y0) * W + xo) * LP : q_dn + xo * LP;
#pragma unroll
                    for (int l = 0; l < LT; ++l)
                        if (l < L) So[l] = fmaf(wv, qr[l], So[l]);
                }
                const int yi = y - dy, xi = x - dx;
                if (yi >= 0 && xi >= 0 && xi < W) {
                    const float wv = wb[((size_t)yi * W + xi) * nd + d];
                    // rows above the slab live in the previous CTA (its last row)
                    const float *qr = yi >= y0 ? qc + ((yi - y0) * W + xi) * LP : q_up + ((rows - 1) * W + xi) * LP;
#pragma unroll
                    for (int l = 0; l < LT; ++l)
                        if (l < L) Si[l] = fmaf(wv, qr[l], Si[l]);
                }
            }
            const float *sr = sc + lp * LP, *qr = qc + lp * LP, *ur = Ub + (size_t)lp * LP;
            float av[LT];
            float mx = -INFINITY, fp = 0.f;
#pragma unroll
            for (int l = 0; l < LT; ++l) {
                av[l] = -INFINITY;
                if (l >= L) continue;
                float m = 0.f;
                if (a.mu_sym) {
#pragma unroll
                    for (int k = 0; k < LT; ++k)
                        if (k < L) m = fmaf(mus[l * L + k], So[k] + Si[k], m);
                } else {
#pragma unroll
                    for (int k = 0; k < LT; ++k)
                        if (k < L) m = fmaf(mus[l * L + k], So[k], fmaf(mus[k * L + l], Si[k], m));
                }
                const float s = sr[l], q = qr[l], u = ur[l];
                fp = fmaf(q, u + 0.5f * m + s, fp);
                av[l] = fmaf(-eta, u + m, (1.f - eta) * s);
                mx = fmaxf(mx, av[l]);
            }
            float z = 0.f;
#pragma unroll
            for (int l = 0; l < LT; ++l)
                if (l < L) z += __expf(av[l] - mx);
            const float lz = mx + __logf(z);
#pragma unroll
            for (int l = 0; l < LT; ++l)
                if (l < L) {
                    const float v = av[l] - lz;
                    sn[lp * LP + l] = v;
                    qn[lp * LP + l] = __expf(v);
                }
            float se, ee;
            two_sum(fh, fp, se, ee);
            fh = se;
            fl = __fadd_rn(fl, ee);
        }
        // this CTA's part of F(q^t): fixed-shape double-float warp trees, then
        // the warps' values by warp 0 (FP64 is the narrow pipe of this part)
        const df fw = warp_sum_df(df_fast_two_sum(fh, fl));
        if ((tid & 31) == 0) {
            red_h[tid >> 5] = fw.h;
            red_l[tid >> 5] = fw.l;
        }
        __syncthreads();
        if (tid < 32) {
            const df v = warp_sum_df(tid < NT / 32 ? df{red_h[tid], red_l[tid]} : df{0.f, 0.f});
            if (tid == 0) {
                part_h[t & 1] = v.h;
                part_l[t & 1] = v.l;
            }
        }
        cluster.sync();   // the new iterate and every CTA's partial are visible cluster-wide
        if (tid < 32) {
            // lane j reads rank j's partial; a fixed-shape tree sums them
            df v = {0.f, 0.f};
            if (tid < nc) {
                const float *ph = cluster.map_shared_rank(part_h, tid), *pl = cluster.map_shared_rank(part_l, tid);
                v = df{ph[t & 1], pl[t & 1]};
            }
            v = warp_sum_df(v);
            if (tid == 0) {
                const double F = df_to(v);
                const bool stop = a.rel_tol > 0.0 && t > 0 && fabs(F - f_prev) <= a.rel_tol * fabs(F);
                if (r == 0) {
                    if (t < a.trace_cap) a.f_trace[(size_t)b * a.trace_cap + t] = F;
                    a.f_cur[b] = F;
                    if (!isfinite(F)) atomicExch(a.status, -6);
                    if (stop) a.done[b] = t + 1;
                }
                stop_flag = stop ? 1 : 0;
                f_prev = F;
            }
        }
        __syncthreads();
        float *ts = sc, *tq = qc;
        sc = sn;
        qc = qn;
        sn = ts;
        qn = tq;
        if (stop_flag) break;
    }
    for (int i = tid; i < npix * LP; i += NT) a.s_out[gbase + i] = sc[i];
    cluster.sync();   // no CTA leaves while another may still read its partials
}

template <int LT, int NT>
cudaError_t launch_resident(const GridResidentLaunch &a, int nc, size_t smem, cudaStream_t st) {
    static SmemOptIn optin;   // the opt-in above 48 KB, once per device
    const cudaError_t attr = smem_optin(optin, grid_resident_kernel<LT, NT>, kResidentMaxSmem);
    if (attr != cudaSuccess) return attr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc, a.B, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeClusterDimension;
    attrs[0].val.clusterDim.x = nc;
    attrs[0].val.clusterDim.y = 1;
    attrs[0].val.clusterDim.z = 1;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, grid_resident_kernel<LT, NT>, a);
}

}  // namespace

// CTAs per instance (a portable cluster) and the shared memory of each
static int resident_ctas(int H) {
    int n = 1;
    while (2 * n <= kResidentCtas && 2 * n <= H) n *= 2;   // 1, 2, 4 or 8, at most one per row
    return n;
}

size_t grid_resident_smem(int H, int W, int L, int LP) {
    const int rows = (H + resident_ctas(H) - 1) / resident_ctas(H);
    return (size_t)4 * rows * W * LP * sizeof(float) + (size_t)L * L * sizeof(float);
}

bool grid_resident_fits(int H, int W, int L, int LP) {
    return L <= 16 && grid_resident_smem(H, W, L, LP) <= kResidentMaxSmem;
}

cudaError_t launch_grid_resident(const GridResidentLaunch &a, cudaStream_t st) {
    if (!grid_resident_fits(a.H, a.W, a.L, a.LP)) return cudaErrorInvalidValue;
    const size_t smem = grid_resident_smem(a.H, a.W, a.L, a.LP);
    const int nc = resident_ctas(a.H);
    if (a.L <= 2) return launch_resident<2, 512>(a, nc, smem, st);
    if (a.L <= 4) return launch_resident<4, 512>(a, nc, smem, st);
    if (a.L <= 8) return launch_resident<8, 512>(a, nc, smem, st);
    return launch_resident<16, 512>(a, nc, smem, st);
}

}  // namespace proxmf
