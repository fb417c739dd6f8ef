// convert_common.cuh -- what the single-image conversion kernels
// (k_convert.cu) and the batched ones (k_batch.cuh) share: the staged
// linearisation table, the batched kernels' launch shapes, and the entry
// points of the batched kernels.  Those are instantiated once per
// (cube-root form, launch shape) pair, each in its own object built from
// k_batch_inst.cu, so the pairs compile in parallel.
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
// rational's degree, 0: the FP64 polynomial) and one launch shape (T threads,
// S sub-blocks): resident CTAs per SM of the device-list or (param) the
// by-value kernel, and launches from a device work list or a by-value list.
// Each (form, shape) pair is instantiated in its own object (k_batch_inst.cu).
template <bool EXACT, int RDEG, int T, int S>
int batch_occ_shape(bool param);
template <bool EXACT, int RDEG, int T, int S>
cudaError_t batch_launch_shape(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                               unsigned long long *d_ctr, int grid, cudaStream_t s);
template <bool EXACT, int RDEG, int T, int S>
cudaError_t batch_launch_param_shape(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total,
                                     int grid, cudaStream_t s);

// The same for a form, dispatched on the shape.
template <bool EXACT, int RDEG>
int batch_occ(const BatchCfg &cfg, bool param)
{
#define MACT_OCC(T, S) if (cfg.threads == T && cfg.subs == S) return batch_occ_shape<EXACT, RDEG, T, S>(param);
    MACT_BATCH_SHAPES(MACT_OCC)
#undef MACT_OCC
    return 1;
}

template <bool EXACT, int RDEG>
cudaError_t batch_launch(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                         unsigned long long *d_ctr, int grid, cudaStream_t s, const BatchCfg &cfg)
{
#define MACT_LAUNCH(T, S) \
    if (cfg.threads == T && cfg.subs == S) return batch_launch_shape<EXACT, RDEG, T, S>(h, d_imgs, count, total, d_ctr, grid, s);
    MACT_BATCH_SHAPES(MACT_LAUNCH)
#undef MACT_LAUNCH
    return cudaErrorInvalidValue;
}

template <bool EXACT, int RDEG>
cudaError_t batch_launch_param(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total, int grid,
                               cudaStream_t s, const BatchCfg &cfg)
{
#define MACT_LAUNCH(T, S) \
    if (cfg.threads == T && cfg.subs == S) return batch_launch_param_shape<EXACT, RDEG, T, S>(h, list, count, total, grid, s);
    MACT_BATCH_SHAPES(MACT_LAUNCH)
#undef MACT_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace mact
