// tma_maps.cu -- host-side tensor maps of the TMA-staged grid step
// (grid_tma.cuh).  A tensor map is a 128-byte descriptor built on the host
// and passed to the kernel as a parameter; nothing here touches the device.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "grid_step.cuh"
#include "tma_maps.h"

namespace proxmf {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// A pixel-major array [B][H][W][pitch] (FP32 or BF16) as a 4-D view; a box
// of {box0, box1, box2, 1} with box0 >= pitch (labels past pitch are
// zero-filled).
cudaError_t encode_4d(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int esize, int B, int H, int W,
                      int pitch, int box0, int box1, int box2) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (enc == nullptr) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0u) return cudaErrorInvalidValue;
    const cuuint64_t px = (cuuint64_t)pitch * esize;
    if (px % 16 != 0) return cudaErrorInvalidValue;
    cuuint64_t dims[4] = {(cuuint64_t)pitch, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    cuuint64_t strides[3] = {px, px * (cuuint64_t)W, px * (cuuint64_t)W * (cuuint64_t)H};
    cuuint32_t box[4] = {(cuuint32_t)box0, (cuuint32_t)box1, (cuuint32_t)box2, 1u};
    cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult r = enc(m, dt, 4, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t encode_state(CUtensorMap *m, const float *base, int B, int H, int W, int LP, int box0, int box1,
                         int box2) {
    return encode_4d(m, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, B, H, W, LP, box0, box1, box2);
}

cudaError_t encode_grid_maps(GridTmaMaps *m, const GridStepLaunch &l, int LP, int CS) {
    cudaError_t e = encode_state(&m->s_in, l.s_in, l.B, l.H, l.W, LP, CS, GX + 2, GY + 2);
    if (e == cudaSuccess) e = encode_state(&m->U, l.U, l.B, l.H, l.W, LP, CS, GX, GY);
    if (e == cudaSuccess) e = encode_state(&m->s_out, l.s_out, l.B, l.H, l.W, LP, CS, GX, GY);
    if (e == cudaSuccess) e = encode_state(&m->s_out2, l.s_out, l.B, l.H, l.W, LP, CS, GX, 2);
    return e;
}

cudaError_t encode_grid_tc_maps(GridTmaTcMaps *m, const GridStepLaunch &l, int LP, int CS, int C16, int UP) {
    cudaError_t e = encode_state(&m->s_int, l.s_in, l.B, l.H, l.W, LP, CS, GX, GY);
    if (e == cudaSuccess) e = encode_state(&m->s_row, l.s_in, l.B, l.H, l.W, LP, CS, GX + 2, 1);
    if (e == cudaSuccess) e = encode_state(&m->s_col, l.s_in, l.B, l.H, l.W, LP, CS, 1, GY);
    if (e == cudaSuccess)
        e = encode_4d(&m->U16, l.U16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, l.B, l.H, l.W, UP, C16, GX, GY);
    if (e == cudaSuccess) e = encode_state(&m->s_out, l.s_out, l.B, l.H, l.W, LP, CS, GX, GY);
    return e;
}

}  // namespace proxmf
