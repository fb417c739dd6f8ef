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

int64_t tiles_of(const ImageDesc &im) { return tiles_of_t<kThreads>(im); }

using Shape = TileShape<kThreads>;

// Linearisation table staged in shared memory: none (HSI, SCT), 256 FP32
// entries, or 256 FP64 entries (polynomial cube-root variant).
enum { kNoTable = 0, kTable32 = 1, kTable64 = 2 };

__device__ __forceinline__ void load_table(int kind, const float *gamma, double *sg)
{
    if (kind == kTable32) reinterpret_cast<float *>(sg)[threadIdx.x] = gamma[threadIdx.x];
    else if (kind == kTable64) sg[threadIdx.x] = reinterpret_cast<const double *>(gamma + 256)[threadIdx.x];
}

template <class Op, typename OutT, int TABLE>
__global__ void __launch_bounds__(kThreads)
k_image(const __grid_constant__ ImageDesc im, const __grid_constant__ Coeffs co,
        const float *__restrict__ gamma, int64_t ntiles)
{
    __shared__ double sgam[256];
    __shared__ uint4 sbuf[Shape::vecs];
    load_table(TABLE, gamma, sgam);
    const Op op{reinterpret_cast<const float *>(sgam), co};
    run_image<kThreads, OutT, false>(im, ntiles, op, sbuf, nullptr);
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
    static int occ = 0;   // resident CTAs per SM of this instantiation
    if (occ == 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_image<Op, OutT, GAMMA>,
                                                                      kThreads, 0);
        occ = (e != cudaSuccess || o <= 0) ? 1 : o;
    }
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
        if (exact) return launch_one<OpCielab<true, true>, OutT, kTable32>(h, im, s);
        if (rat) return launch_one<OpCielab<false, true>, OutT, kTable32>(h, im, s);
        return launch_one<OpCielab<false, false>, OutT, kTable64>(h, im, s);
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

template <typename OutT, bool EXACT, bool RAT>
__device__ __forceinline__ void batch_tile(const ImageDesc &im, int64_t t, const float *sgam,
                                           const Coeffs &co, uint4 *sbuf)
{
    if (im.space == MACT_CIELAB) {
        const OpCielab<EXACT, RAT> op{sgam, co};
        process_tile<kThreads, OutT, false>(im, t, op, sbuf, nullptr);
    } else if (im.space == MACT_HSI) {
        const OpHsi<EXACT> op{co};
        process_tile<kThreads, OutT, false>(im, t, op, sbuf, nullptr);
    } else {
        const OpSct<EXACT> op{co};
        process_tile<kThreads, OutT, false>(im, t, op, sbuf, nullptr);
    }
}

template <bool EXACT, bool RAT>
__global__ void __launch_bounds__(kThreads)
k_batch(const ImageDesc *__restrict__ imgs, int32_t count, int64_t total,
        unsigned long long *__restrict__ ctr, const __grid_constant__ Coeffs co,
        const float *__restrict__ gamma)
{
    __shared__ double sgam64[256];
    __shared__ uint4 sbuf[Shape::vecs];
    __shared__ long long s_tile;
    __shared__ int s_img;
    load_table((!EXACT && !RAT) ? kTable64 : kTable32, gamma, sgam64);
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
        if (im.dtype == MACT_F16) batch_tile<__half, EXACT, RAT>(im, lt, sgam, co, sbuf);
        else batch_tile<float, EXACT, RAT>(im, lt, sgam, co, sbuf);
    }
    // the last CTA out resets the counters for the next launch on the handle
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long done = atomicAdd(&ctr[1], 1ull);
        if (done == (unsigned long long)gridDim.x - 1) {
            atomicExch(&ctr[0], 0ull);
            atomicExch(&ctr[1], 0ull);
        }
    }
}

template <bool EXACT, bool RAT>
static int occ_batch()
{
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batch<EXACT, RAT>, kThreads, 0);
        occ = (e != cudaSuccess || o <= 0) ? 1 : o;
    }
    return occ;
}

int batch_blocks_per_sm(const mact_ctx &h)
{
    if (h.cfg.exact) return occ_batch<true, true>();
    return h.co.lab_rational ? occ_batch<false, true>() : occ_batch<false, false>();
}

cudaError_t launch_batch(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                         unsigned long long *d_ctr, int grid, cudaStream_t s)
{
    if (h.cfg.exact)
        k_batch<true, true><<<grid, kThreads, 0, s>>>(d_imgs, count, total, d_ctr, h.co, h.d_gamma);
    else if (h.co.lab_rational)
        k_batch<false, true><<<grid, kThreads, 0, s>>>(d_imgs, count, total, d_ctr, h.co, h.d_gamma);
    else
        k_batch<false, false><<<grid, kThreads, 0, s>>>(d_imgs, count, total, d_ctr, h.co, h.d_gamma);
    return cudaGetLastError();
}

}  // namespace mact
