// tma_maps.h -- tensor maps of pixel-major FP32 arrays (tma_maps.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace proxmf {

// [B][H][W][LP] FP32 as a 4-D view with boxes of {box0, box1, box2, 1}
// (box0 >= LP: the labels past LP are zero-filled, as are cells outside the
// image).  base must be 16-byte aligned and LP * 4 a multiple of 16.
cudaError_t encode_state(CUtensorMap *m, const float *base, int B, int H, int W, int LP, int box0, int box1,
                         int box2);

}  // namespace proxmf
