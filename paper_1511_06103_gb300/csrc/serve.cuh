// serve.cuh -- device side of the serving loop: one persistent launch per
// iteration advances every in-flight grid CRF, whatever its label count,
// connectivity or symmetry of mu.
//
// The host keeps a table of slots in device memory (one admitted request
// each) and one tile table over all running slots (slot list and prefix sums
// of their tile counts).  The launch walks every tile of every running slot
// with a grid-stride loop; a tile dispatches on its slot's kernel label count
// (a switch over the instantiated counts) and runs the fixed-rule step of
// Sec. 3.1-3.2 on it with connectivity and symmetry taken at run time.  The
// last tile of a slot finishes that slot's free energy in a fixed order,
// advances its iteration count and retires it when the stopping rule holds,
// so a request's result does not depend on which other requests share the
// GPU.  Results are published to host-mapped memory.
#pragma once

#include "grid_step.cuh"

namespace proxmf {

struct ServeSlot {
    const float *U;          // [N][LP]
    float *s[2];             // [N][LP] ping-pong log q
    const float *w;          // [N][nd]
    const float2 *mu_out, *mu_in;
    double *partial;         // [nblk]
    unsigned *counter;       // [1]
    const float *eta;        // [1] device
    int L, LT, H, W, nbx, nblk, conn, sym;
    int max_iters;
    double rel_tol;
    // device-maintained
    int it;                  // steps taken (state parity)
    int active;              // 1 while running
    double F_prev;
};

struct ServeResult {         // host-mapped
    int done;                // 1 once retired
    int iters;
    double F;                // F of the state before the last step
};

struct ServeTable {
    int count;                          // running slots
    int slots[kMaxServeSlots];
    int prefix[kMaxServeSlots + 1];     // tile offsets
};

// Dynamic shared memory of one serving tile with kernel label count LT:
// the q tile with its halo, the tile's own log q, mu and mu^T as pairs.
__host__ __device__ constexpr size_t serve_tile_smem(int LT) {
    return ((size_t)(GY + 2) * (GX + 2) * tile_stride(storage_labels(LT)) +
            (size_t)GT * tile_stride(storage_labels(LT))) * 4 +
           (size_t)2 * LT * (((LT + 1) / 2 + 1) / 2 * 2) * 8;
}

// One 32 x 8 tile of one request: a1-a4 for its pixels with the fixed step,
// and the tile's free-energy partial, returned in thread 0.  All threads of
// the block call it; conn (4 or 8) and sym (mu symmetric) are uniform per
// request.  The shared memory is the caller's dynamic buffer.
template <int LT>
__device__ __forceinline__ double serve_tile(const TileJob &j, int conn, bool sym, int bx, int by, uint8_t *smem,
                                             double *red) {
    constexpr int LP = storage_labels(LT);
    constexpr int NP = (LT + 1) / 2;
    constexpr int NPP = (NP + 1) / 2 * 2;
    constexpr int LS = tile_stride(LP);
    constexpr int TW = GX + 2;
    constexpr int HALO = 2 * TW + 2 * GY;
    constexpr bool MASK = (LT == LP);
    float *qt = reinterpret_cast<float *>(smem);
    float *sown = qt + (GY + 2) * TW * LS;
    float2 *mus = reinterpret_cast<float2 *>(sown + GT * LS);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * GX + tx;
    const int x0 = bx * GX, y0 = by * GY;
    const int x = x0 + tx, y = y0 + ty;
    const int H = j.H, W = j.W, L = j.L, nd = conn == 8 ? 4 : 2;
    const bool inside = (x < W) && (y < H);
    const size_t p = (size_t)y * W + x;
    __syncthreads();   // shared memory of a previous tile is no longer read

    for (int i = tid; i < LT * NPP; i += GT) {
        mus[i] = j.mu_out[i];
        if (!sym) mus[LT * NPP + i] = j.mu_in[i];
    }
    float2 s[LP / 2];
    if (inside) {
        load_px<LP>(s, j.s_in + p * LP);
    } else {
#pragma unroll
        for (int i = 0; i < LP / 2; ++i) s[i] = splat2(kPadLogQ);
    }
    if (tid < HALO) {
        int hr, hc;
        if (tid < TW) {
            hr = 0;
            hc = tid;
        } else if (tid < 2 * TW) {
            hr = GY + 1;
            hc = tid - TW;
        } else {
            const int k = tid - 2 * TW;
            hr = 1 + (k >> 1);
            hc = (k & 1) ? TW - 1 : 0;
        }
        const int gy = y0 - 1 + hr, gx = x0 - 1 + hc;
        float2 h[LP / 2];
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            load_px<LP>(h, j.s_in + ((size_t)gy * W + gx) * LP);
        } else {
#pragma unroll
            for (int i = 0; i < LP / 2; ++i) h[i] = splat2(kPadLogQ);
        }
        put_cell<LP>(qt + (hr * TW + hc) * LS, h);
    }
    put_cell<LP>(qt + ((ty + 1) * TW + tx + 1) * LS, s);
    store_px<LP>(sown + tid * LS, s);

    float wo[4] = {0.f, 0.f, 0.f, 0.f}, wi[4] = {0.f, 0.f, 0.f, 0.f};
    if (inside) {
        const float *wb = j.w;
        if (nd == 4) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(wb + p * 4));
            wo[0] = t.x;
            wo[1] = t.y;
            wo[2] = t.z;
            wo[3] = t.w;
        } else {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(wb + p * 2));
            wo[0] = t.x;
            wo[1] = t.y;
        }
        if (x > 0) wi[0] = __ldg(wb + (p - 1) * nd + 0);
        if (y > 0) wi[1] = __ldg(wb + (p - W) * nd + 1);
        if (nd == 4) {
            if (x > 0 && y > 0) wi[2] = __ldg(wb + (p - W - 1) * nd + 2);
            if (x + 1 < W && y > 0) wi[3] = __ldg(wb + (p - W + 1) * nd + 3);
        }
    }
    __syncthreads();

    const float *c_r = qt + ((ty + 1) * TW + tx + 2) * LS;
    const float *c_d = qt + ((ty + 2) * TW + tx + 1) * LS;
    const float *c_dr = qt + ((ty + 2) * TW + tx + 2) * LS;
    const float *c_dl = qt + ((ty + 2) * TW + tx) * LS;
    const float *c_l = qt + ((ty + 1) * TW + tx) * LS;
    const float *c_u = qt + (ty * TW + tx + 1) * LS;
    const float *c_ul = qt + (ty * TW + tx) * LS;
    const float *c_ur = qt + (ty * TW + tx + 2) * LS;

    // a1: m = mu S_out + mu^T S_in (= mu (S_out + S_in) for symmetric mu)
    float2 m[NP], S[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        m[k] = splat2(0.f);
        S[k] = splat2(0.f);
    }
    acc_cell<NP>(S, c_r, wo[0]);
    acc_cell<NP>(S, c_d, wo[1]);
    if (nd == 4) {
        acc_cell<NP>(S, c_dr, wo[2]);
        acc_cell<NP>(S, c_dl, wo[3]);
    }
    if (sym) {
        acc_cell<NP>(S, c_l, wi[0]);
        acc_cell<NP>(S, c_u, wi[1]);
        if (nd == 4) {
            acc_cell<NP>(S, c_ul, wi[2]);
            acc_cell<NP>(S, c_ur, wi[3]);
        }
    }
    pair_matvec<LT, NP, NPP>(m, mus, S);
    if (!sym) {
#pragma unroll
        for (int k = 0; k < NP; ++k) S[k] = splat2(0.f);
        acc_cell<NP>(S, c_l, wi[0]);
        acc_cell<NP>(S, c_u, wi[1]);
        if (nd == 4) {
            acc_cell<NP>(S, c_ul, wi[2]);
            acc_cell<NP>(S, c_ur, wi[3]);
        }
        pair_matvec<LT, NP, NPP>(m, mus + LT * NPP, S);
    }

    // a2-a4 with this pixel's free-energy term
    float2 u[LP / 2];
    if (inside) {
        load_px<LP>(u, j.U + p * LP);
    } else {
#pragma unroll
        for (int i = 0; i < LP / 2; ++i) u[i] = splat2(0.f);
    }
#pragma unroll
    for (int i = 0; i < LP / 4; ++i) {
        const float4 v = reinterpret_cast<const float4 *>(sown + tid * LS)[i];
        s[2 * i] = make_float2(v.x, v.y);
        s[2 * i + 1] = make_float2(v.z, v.w);
    }
    if constexpr (LP == 2) s[0] = *reinterpret_cast<const float2 *>(sown + tid * LS);
    float2 qc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) qc[k] = splat2(0.f);
    acc_cell<NP>(qc, qt + ((ty + 1) * TW + tx + 1) * LS, 1.f);
    const float eta = j.eta;
    const float2 neta = splat2(-eta), ome = splat2(1.f - eta), half = splat2(0.5f);
    float2 f2 = splat2(0.f);
    float mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 g = add2(u[k], m[k]);
        const float2 h = add2(fma2(half, m[k], u[k]), s[k]);
        f2 = fma2(qc[k], h, f2);
        float2 av = fma2(neta, g, mul2(ome, s[k]));
        const int l0 = 2 * k, l1 = 2 * k + 1;
        if ((MASK && l0 >= L)) av.x = -INFINITY;
        if ((MASK && l1 >= L) || l1 >= LT) av.y = -INFINITY;
        s[k] = av;
        mx = fmaxf(mx, fmaxf(av.x, av.y));
    }
    float z = 0.f;
#pragma unroll
    for (int k = 0; k < NP; ++k) z += __expf(s[k].x - mx) + __expf(s[k].y - mx);
    const float2 nlse = splat2(-(mx + __logf(z)));
    if (inside) {
        float2 o[LP / 2];
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            if (k < NP) {
                o[k] = add2(s[k], nlse);
                const int l0 = 2 * k, l1 = 2 * k + 1;
                if ((MASK && l0 >= L)) o[k].x = kPadLogQ;
                if ((MASK && l1 >= L) || l1 >= LT) o[k].y = kPadLogQ;
            } else {
                o[k] = splat2(kPadLogQ);
            }
        }
        store_px<LP>(j.s_out + p * LP, o);
    }
    // a5: the tile's F partial (double-float warp trees, FP64 across warps)
    const df fw = warp_sum_df(df{inside ? f2.x + f2.y : 0.f, 0.f});
    if ((tid & 31) == 0) red[tid >> 5] = df_to(fw);
    __syncthreads();
    double bs = 0.0;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < GT / 32; ++k) bs += red[k];
    }
    return bs;
}

// The kernel label counts instantiated for serving (kernel_labels of any L).
#define PROXMF_SERVE_LTS(X) X(2) X(4) X(8) X(12) X(16) X(20) X(21) X(24) X(28) X(32)

__global__ void __launch_bounds__(GT, 2) serve_step_kernel(ServeSlot *slots, const ServeTable *table,
                                                           ServeResult *results) {
    extern __shared__ __align__(16) uint8_t ssm[];
    __shared__ int sh_slot, sh_local, sh_last;
    __shared__ double red[GT / 32];
    const int tid = threadIdx.y * GX + threadIdx.x;
    const int count = table->count;
    const int total = table->prefix[count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        if (tid == 0) {
            // the slot whose tile range holds t: largest k with prefix[k] <= t
            int lo = 0, hi = count - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (table->prefix[mid] <= t)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            sh_slot = table->slots[lo];
            sh_local = t - table->prefix[lo];
        }
        __syncthreads();
        const int si = sh_slot, local = sh_local;
        ServeSlot &sl = slots[si];
        const int active = *(volatile int *)&sl.active;
        const int it = *(volatile int *)&sl.it;
        if (!active) {
            __syncthreads();
            continue;
        }
        TileJob j;
        j.s_in = sl.s[it & 1];
        j.s_out = sl.s[(it + 1) & 1];
        j.U = sl.U;
        j.w = sl.w;
        j.mu_out = sl.mu_out;
        j.mu_in = sl.mu_in;
        j.mu_p = sl.mu_out;
        j.eta = *sl.eta;
        j.adaptive = false;
        j.adapt_d = 0.f;
        j.L = sl.L;
        j.H = sl.H;
        j.W = sl.W;
        j.update = 1;
        const int bx = local % sl.nbx, by = local / sl.nbx;
        double bs = 0.0;
        switch (sl.LT) {
#define PROXMF_SERVE_CASE(V)                                                  \
    case V:                                                                   \
        bs = serve_tile<V>(j, sl.conn, sl.sym != 0, bx, by, ssm, red);        \
        break;
            PROXMF_SERVE_LTS(PROXMF_SERVE_CASE)
#undef PROXMF_SERVE_CASE
            default:
                break;
        }
        if (tid == 0) {
            sl.partial[local] = bs;
            __threadfence();
            sh_last = atomicAdd(sl.counter, 1u) == (unsigned)(sl.nblk - 1);
        }
        __syncthreads();
        if (sh_last) {
            __threadfence();
            double acc = 0.0;
            for (int k = tid; k < sl.nblk; k += GT) acc += __ldcg(sl.partial + k);
            acc = warp_sum_f64(acc);
            if ((tid & 31) == 0) red[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                double F = 0.0;
#pragma unroll
                for (int k = 0; k < GT / 32; ++k) F += red[k];
                *sl.counter = 0u;
                const int nit = it + 1;
                bool stop = nit >= sl.max_iters || !isfinite(F);
                if (sl.rel_tol > 0.0 && it > 0 && fabs(F - sl.F_prev) <= sl.rel_tol * fabs(F)) stop = true;
                sl.F_prev = F;
                sl.it = nit;
                if (stop) {
                    sl.active = 0;
                    ServeResult *r = results + si;
                    r->F = F;
                    r->iters = nit;
                    __threadfence_system();
                    *(volatile int *)&r->done = 1;
                    __threadfence_system();
                }
                __threadfence();
            }
        }
        __syncthreads();
    }
}

}  // namespace proxmf
