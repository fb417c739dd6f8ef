// k_batch.cuh -- the batched conversion kernels (a tile work list over many
// images of any spaces and dtypes) and their launchers.  Included only by
// k_batch_inst.cu, which the build compiles once per (cube-root form, launch
// shape) pair, each object instantiating one pair with MACT_BATCH_SHAPE, so
// the 20 pairs compile in parallel.
//
// The device-list kernel pulls tiles with an atomic counter, so uneven
// images and spaces balance dynamically across CTAs; its last CTA resets the
// counters, so consecutive launches need no memset.
#pragma once

#include "convert_common.cuh"

namespace mact {

template <typename OutT, bool EXACT, int RDEG, int THREADS, int SUBS>
__device__ __forceinline__ void batch_tile(const ImageDesc &im, int64_t t, const float *sgam,
                                           const Coeffs &co, uint4 *sbuf)
{
    float *scr = reinterpret_cast<float *>(sbuf + TileShape<THREADS, SUBS>::vecs);
    if (im.space == MACT_CIELAB) {
        const OpCielab<EXACT, RDEG, sizeof(OutT) == 4> op{sgam, co};   // FP16 planes: no Newton step
        process_tile<THREADS, OutT, false, decltype(op), SUBS>(im, t, op, sbuf, nullptr, scr);
    } else if (im.space == MACT_CIELUV) {
        const OpCieluv<EXACT, RDEG, sizeof(OutT) == 4> op{sgam, co};
        process_tile<THREADS, OutT, false, decltype(op), SUBS>(im, t, op, sbuf, nullptr, scr);
    } else if (im.space == MACT_HSI) {
        const OpHsi<EXACT> op{co};
        process_tile<THREADS, OutT, false, decltype(op), SUBS>(im, t, op, sbuf, nullptr, scr);
    } else {
        const OpSct<EXACT> op{co};
        process_tile<THREADS, OutT, false, decltype(op), SUBS>(im, t, op, sbuf, nullptr, scr);
    }
}

template <bool EXACT, int RDEG, int THREADS, int SUBS>
__global__ void __launch_bounds__(THREADS)
k_batch(const ImageDesc *__restrict__ imgs, int32_t count, int64_t total,
        unsigned long long *__restrict__ ctr, const __grid_constant__ Coeffs co,
        const float *__restrict__ gamma)
{
    __shared__ double sgam64[256];
    __shared__ uint4 sbuf[TileShape<THREADS, SUBS>::vecs + TileShape<THREADS, SUBS>::scratch];
    __shared__ long long s_tile;
    __shared__ int s_img;
    load_table((!EXACT && RDEG == 0) ? kTable64 : kTable32, gamma, sgam64);
    const float *sgam = reinterpret_cast<const float *>(sgam64);
    for (;;) {
        __syncthreads();   // previous tile finished with sbuf / s_tile
        if (threadIdx.x == 0) {
            long long t = (long long)atomicAdd(&ctr[0], 1ull);
            s_tile = t;
            if (t < total) {
                // last image whose first tile is <= t (list sorted by tile_begin)
                int lo = 0, hi = count - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (imgs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
                }
                s_img = lo;
            }
        }
        __syncthreads();
        const long long t = s_tile;
        if (t >= total) break;
        const ImageDesc &im = imgs[s_img];
        const int64_t lt = t - im.tile_begin;
        if (im.dtype == MACT_F16) batch_tile<__half, EXACT, RDEG, THREADS, SUBS>(im, lt, sgam, co, sbuf);
        else batch_tile<float, EXACT, RDEG, THREADS, SUBS>(im, lt, sgam, co, sbuf);
    }
    // the last CTA out resets the counters for the next launch on the list
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long done = atomicAdd(&ctr[1], 1ull);
        if (done == (unsigned long long)gridDim.x - 1) {
            atomicExch(&ctr[0], 0ull);
            atomicExch(&ctr[1], 0ull);
        }
    }
}

// The same batched conversion for short lists, with the work list passed in
// the kernel's parameter block instead of device memory: the launch needs no
// copy and no device counter.  Tiles are uniform (all full but each image's
// last), so CTAs take them grid-stride, t = blockIdx.x + k * gridDim.x.
template <bool EXACT, int RDEG, int THREADS, int SUBS>
__global__ void __launch_bounds__(THREADS)
k_batch_param(const __grid_constant__ ParamList list, int32_t count, int64_t total,
              const __grid_constant__ Coeffs co, const float *__restrict__ gamma)
{
    __shared__ double sgam64[256];
    __shared__ uint4 sbuf[TileShape<THREADS, SUBS>::vecs + TileShape<THREADS, SUBS>::scratch];
    load_table((!EXACT && RDEG == 0) ? kTable64 : kTable32, gamma, sgam64);
    const float *sgam = reinterpret_cast<const float *>(sgam64);
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        __syncthreads();   // previous tile finished with sbuf
        // last image whose first tile is <= t (the list is sorted by tile_begin)
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (list.img[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
        }
        const ImageDesc &im = list.img[lo];
        const int64_t lt = t - im.tile_begin;
        if (im.dtype == MACT_F16) batch_tile<__half, EXACT, RDEG, THREADS, SUBS>(im, lt, sgam, co, sbuf);
        else batch_tile<float, EXACT, RDEG, THREADS, SUBS>(im, lt, sgam, co, sbuf);
    }
}

// Per-shape entry points (declared in convert_common.cuh): resident CTAs per
// SM of the device-list kernel or (param) of the by-value kernel, and
// launches of either.  Each form is sized by its own figure: the by-value
// kernel holds its list in the parameter block and can need more registers,
// which must not shrink the device-list kernel's grid.
template <bool EXACT, int RDEG, int T, int S>
int batch_occ_shape(bool param)
{
    struct Occ {
        int list, param;
    };
    static const Occ occ = [] {   // thread-safe one-time init
        int o = 0, op = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batch<EXACT, RDEG, T, S>, T, 0);
        cudaError_t ep = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, k_batch_param<EXACT, RDEG, T, S>, T, 0);
        return Occ{(e != cudaSuccess || o <= 0) ? 1 : o, (ep != cudaSuccess || op <= 0) ? 1 : op};
    }();
    return param ? occ.param : occ.list;
}

template <bool EXACT, int RDEG, int T, int S>
cudaError_t batch_launch_shape(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                               unsigned long long *d_ctr, int grid, cudaStream_t s)
{
    k_batch<EXACT, RDEG, T, S><<<grid, T, 0, s>>>(d_imgs, count, total, d_ctr, h.co, h.d_gamma);
    return cudaGetLastError();
}

template <bool EXACT, int RDEG, int T, int S>
cudaError_t batch_launch_param_shape(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total,
                                     int grid, cudaStream_t s)
{
    k_batch_param<EXACT, RDEG, T, S><<<grid, T, 0, s>>>(list, count, total, h.co, h.d_gamma);
    return cudaGetLastError();
}

}  // namespace mact

// Explicit instantiation of one (form, shape) pair's entry points (inside
// namespace mact).
#define MACT_BATCH_SHAPE(EXACT, RDEG, T, S)                                                                  \
    template int batch_occ_shape<EXACT, RDEG, T, S>(bool);                                                    \
    template cudaError_t batch_launch_shape<EXACT, RDEG, T, S>(const mact_ctx &, const ImageDesc *, int32_t,  \
                                                               int64_t, unsigned long long *, int, cudaStream_t); \
    template cudaError_t batch_launch_param_shape<EXACT, RDEG, T, S>(const mact_ctx &, const ParamList &,     \
                                                                     int32_t, int64_t, int, cudaStream_t);
