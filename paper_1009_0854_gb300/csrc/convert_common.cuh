// convert_common.cuh -- what the single-image conversion kernels
// (k_convert.cu) and the batched ones (k_batch.cuh) share: the staged
// linearisation table, the batched kernels' launch shapes, and the per-form
// entry points of the batched kernels.  Those are instantiated once per
// cube-root form, each in its own translation unit (k_batch_exact.cu,
// k_batch_rat4.cu, k_batch_rat6.cu, k_batch_poly.cu), so the forms compile
// in parallel.
#pragma once

#include "engine.cuh"
#include "internal.h"
#include "pixel.cuh"

namespace mact {

// Linearisation table staged in shared memory: none (HSI, SCT), 256 FP32
// entries, or 256 FP64 entries (polynomial cube-root variant).
enum { kNoTable = 0, kTable32 = 1, kTable64 = 2 };

__device__ __forceinline__ void load_table(int kind, const float *gamma, double *sg)
{
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        if (kind == kTable32) reinterpret_cast<float *>(sg)[i] = gamma[i];
        else if (kind == kTable64) sg[i] = reinterpret_cast<const double *>(gamma + 256)[i];
    }
}

// Supported launch shapes of the batched kernels (threads, sub-blocks): 16 to
// 32 pixels per thread, tiles of 2048 to 8192 pixels.
#define MACT_BATCH_SHAPES(X) X(128, 4) X(256, 4) X(512, 4) X(256, 8) X(128, 8)

// Batched kernels of one cube-root form (EXACT: libm; else RDEG 4 or 6: the
// rational's degree, 0: the FP64 polynomial): resident CTAs per SM for a
// shape, and launches from a device work list or a by-value list.
template <bool EXACT, int RDEG>
int batch_occ(const BatchCfg &cfg);

template <bool EXACT, int RDEG>
cudaError_t batch_launch(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                         unsigned long long *d_ctr, int grid, cudaStream_t s, const BatchCfg &cfg);

template <bool EXACT, int RDEG>
cudaError_t batch_launch_param(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total, int grid,
                               cudaStream_t s, const BatchCfg &cfg);

}  // namespace mact
