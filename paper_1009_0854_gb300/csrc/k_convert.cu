// k_convert.cu -- RGB -> CIELAB / HSI / SCT kernels on the streaming tile
// engine (engine.cuh), single-image and batched forms.
//
// The single-image kernel is persistent (grid = SMs x resident CTAs) and
// walks the image's tiles with a grid stride.  The batched kernel pulls
// tiles of many images from a device work list with an atomic counter, so
// uneven images and spaces balance dynamically across CTAs; its last CTA
// resets the counters, so consecutive launches need no memset.
#include "engine.cuh"
#include "internal.h"
#include "pixel.cuh"

namespace mact {

int64_t tiles_of(const ImageDesc &im)
{
    if (im.width <= 0 || im.height <= 0) return 0;
    return im.height * im.tiles_per_row;
}

using Shape = TileShape<kThreads>;

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

template <class Op, typename OutT, int TABLE>
__global__ void __launch_bounds__(kThreads)
k_image(const __grid_constant__ ImageDesc im, const __grid_constant__ Coeffs co,
        const float *__restrict__ gamma, int64_t ntiles)
{
    __shared__ double sgam[256];
    __shared__ uint4 sbuf[Shape::vecs + Shape::scratch];
    load_table(TABLE, gamma, sgam);
    const Op op{reinterpret_cast<const float *>(sgam), co};
    run_image<kThreads, OutT, false>(im, ntiles, op, sbuf, nullptr, reinterpret_cast<float *>(sbuf + Shape::vecs));
}

// HSI and SCT operators take no table; give them the same aggregate shape.
template <class Op>
struct WithTable : Op {
    __device__ WithTable(const float *, const Coeffs &c) : Op{c} {}
};

template <class Op, typename OutT, int GAMMA>
static cudaError_t launch_one(const mact_ctx &h, const ImageDesc &im, cudaStream_t s)
{
    const int64_t nt = tiles_of(im);
    if (nt == 0) return cudaSuccess;
    // resident CTAs per SM of this instantiation (thread-safe one-time init)
    static const int occ = [] {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_image<Op, OutT, GAMMA>, kThreads, 0);
        return (e != cudaSuccess || o <= 0) ? 1 : o;
    }();
    const int64_t cap = (int64_t)h.num_sms * occ;
    const int64_t grid = nt < cap ? nt : cap;
    k_image<Op, OutT, GAMMA><<<(unsigned)grid, kThreads, 0, s>>>(im, h.co, h.d_gamma, nt);
    return cudaGetLastError();
}

template <typename OutT>
static cudaError_t dispatch_space(const mact_ctx &h, const ImageDesc &im, cudaStream_t s)
{
    const bool exact = h.cfg.exact != 0;
    const bool rat = h.co.lab_rational != 0;
    switch (im.space) {
    case MACT_CIELAB:
        if (exact) return launch_one<OpCielab<true, 4>, OutT, kTable32>(h, im, s);
        if (rat && h.co.lab_deg == 6) return launch_one<OpCielab<false, 6>, OutT, kTable32>(h, im, s);
        if (rat) return launch_one<OpCielab<false, 4>, OutT, kTable32>(h, im, s);
        return launch_one<OpCielab<false, 0>, OutT, kTable64>(h, im, s);
    case MACT_HSI:
        if (exact) return launch_one<WithTable<OpHsi<true>>, OutT, kNoTable>(h, im, s);
        return launch_one<WithTable<OpHsi<false>>, OutT, kNoTable>(h, im, s);
    default:
        if (exact) return launch_one<WithTable<OpSct<true>>, OutT, kNoTable>(h, im, s);
        return launch_one<WithTable<OpSct<false>>, OutT, kNoTable>(h, im, s);
    }
}

cudaError_t launch_convert(const mact_ctx &h, const ImageDesc &im, cudaStream_t s)
{
    if (im.dtype == MACT_F16) return dispatch_space<__half>(h, im, s);
    return dispatch_space<float>(h, im, s);
}

// ------------------------------------------------------------ batched form

template <typename OutT, bool EXACT, int RDEG, int THREADS, int SUBS>
__device__ __forceinline__ void batch_tile(const ImageDesc &im, int64_t t, const float *sgam,
                                           const Coeffs &co, uint4 *sbuf)
{
    float *scr = reinterpret_cast<float *>(sbuf + TileShape<THREADS, SUBS>::vecs);
    if (im.space == MACT_CIELAB) {
        const OpCielab<EXACT, RDEG> op{sgam, co};
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

// Supported launch shapes (threads, sub-blocks): 16 to 32 pixels per thread,
// tiles of 2048 to 8192 pixels.
#define MACT_BATCH_SHAPES(X) X(128, 4) X(256, 4) X(512, 4) X(256, 8) X(128, 8)

bool batch_cfg_supported(const BatchCfg &cfg)
{
#define MACT_SUPPORTED(T, S) if (cfg.threads == T && cfg.subs == S) return true;
    MACT_BATCH_SHAPES(MACT_SUPPORTED)
#undef MACT_SUPPORTED
    return false;
}

template <bool EXACT, int RDEG, int THREADS, int SUBS>
static int occ_batch()
{
    static const int occ = [] {   // thread-safe one-time init
        int o = 0, op = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batch<EXACT, RDEG, THREADS, SUBS>,
                                                                      THREADS, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, k_batch_param<EXACT, RDEG, THREADS, SUBS>,
                                                              THREADS, 0);
        if (op < o) o = op;   // one figure serves both forms
        return (e != cudaSuccess || o <= 0) ? 1 : o;
    }();
    return occ;
}

template <bool EXACT, int RDEG>
static int occ_shape(const BatchCfg &cfg)
{
#define MACT_OCC(T, S) if (cfg.threads == T && cfg.subs == S) return occ_batch<EXACT, RDEG, T, S>();
    MACT_BATCH_SHAPES(MACT_OCC)
#undef MACT_OCC
    return 1;
}

int batch_blocks_per_sm(const mact_ctx &h, const BatchCfg &cfg)
{
    if (h.cfg.exact) return occ_shape<true, 4>(cfg);
    if (!h.co.lab_rational) return occ_shape<false, 0>(cfg);
    return h.co.lab_deg == 6 ? occ_shape<false, 6>(cfg) : occ_shape<false, 4>(cfg);
}

template <bool EXACT, int RDEG>
static cudaError_t launch_shape(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                                unsigned long long *d_ctr, int grid, cudaStream_t s, const BatchCfg &cfg)
{
#define MACT_LAUNCH(T, S)                                                                               \
    if (cfg.threads == T && cfg.subs == S) {                                                            \
        k_batch<EXACT, RDEG, T, S><<<grid, T, 0, s>>>(d_imgs, count, total, d_ctr, h.co, h.d_gamma);     \
        return cudaGetLastError();                                                                      \
    }
    MACT_BATCH_SHAPES(MACT_LAUNCH)
#undef MACT_LAUNCH
    return cudaErrorInvalidValue;
}

template <bool EXACT, int RDEG>
static cudaError_t launch_shape_param(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total,
                                      int grid, cudaStream_t s, const BatchCfg &cfg)
{
#define MACT_LAUNCH(T, S)                                                                               \
    if (cfg.threads == T && cfg.subs == S) {                                                            \
        k_batch_param<EXACT, RDEG, T, S><<<grid, T, 0, s>>>(list, count, total, h.co, h.d_gamma);        \
        return cudaGetLastError();                                                                      \
    }
    MACT_BATCH_SHAPES(MACT_LAUNCH)
#undef MACT_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_param(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total, int grid,
                               cudaStream_t s, const BatchCfg &cfg)
{
    if (count < 1 || count > kParamImages) return cudaErrorInvalidValue;
    if (h.cfg.exact) return launch_shape_param<true, 4>(h, list, count, total, grid, s, cfg);
    if (!h.co.lab_rational) return launch_shape_param<false, 0>(h, list, count, total, grid, s, cfg);
    if (h.co.lab_deg == 6) return launch_shape_param<false, 6>(h, list, count, total, grid, s, cfg);
    return launch_shape_param<false, 4>(h, list, count, total, grid, s, cfg);
}

cudaError_t launch_batch(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                         unsigned long long *d_ctr, int grid, cudaStream_t s, const BatchCfg &cfg)
{
    if (h.cfg.exact) return launch_shape<true, 4>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
    if (!h.co.lab_rational) return launch_shape<false, 0>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
    if (h.co.lab_deg == 6) return launch_shape<false, 6>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
    return launch_shape<false, 4>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
}

}  // namespace mact
