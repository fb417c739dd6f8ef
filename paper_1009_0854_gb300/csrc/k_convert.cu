// k_convert.cu -- RGB -> CIELAB / HSI / SCT kernels on the streaming tile
// engine (engine.cuh): the single-image form, and the dispatch of the batched
// form to its per-form translation units (k_batch.cuh, k_batch_*.cu).
//
// The single-image kernel is persistent (grid = SMs x resident CTAs) and
// walks the image's tiles with a grid stride.
#include "convert_common.cuh"

namespace mact {

int64_t tiles_of(const ImageDesc &im)
{
    if (im.width <= 0 || im.height <= 0) return 0;
    return im.height * im.tiles_per_row;
}

using Shape = TileShape<kThreads>;

// HSI and SCT operators take no table; give them the same aggregate shape.
template <class Op>
struct WithTable : Op {
    __device__ WithTable(const float *, const Coeffs &c) : Op{c} {}
};

// Minimum resident CTAs per SM each single-image kernel is compiled for (the
// second __launch_bounds__ argument; 0 = no hint, the compiler's own register
// budget).  Measured per kernel on the 2^24 cube and a 16384^2 image: a hint
// of 1 (96-127 registers) makes MACT SCT and CIELUV with FP32 planes 8-9%
// faster on the large image; 4 (64 registers) makes both HSI forms with FP32
// planes 1-6% faster on the cube; with FP16 planes MACT CIELAB gains 4% at 4
// and CIELUV 2% at 3.  The others are fastest with no hint.
template <class Op, typename OutT>
struct ImageMinCtas {
    static constexpr int value = 0;
};
template <> struct ImageMinCtas<WithTable<OpSct<false>>, float> { static constexpr int value = 1; };
template <> struct ImageMinCtas<OpCieluv<false, 4, true>, float> { static constexpr int value = 1; };
template <> struct ImageMinCtas<WithTable<OpHsi<false>>, float> { static constexpr int value = 4; };
template <> struct ImageMinCtas<WithTable<OpHsi<true>>, float> { static constexpr int value = 4; };
template <> struct ImageMinCtas<OpCielab<false, 4, false>, __half> { static constexpr int value = 4; };
template <> struct ImageMinCtas<OpCieluv<false, 4, false>, __half> { static constexpr int value = 3; };

template <class Op, typename OutT, int TABLE>
__global__ void __launch_bounds__(kThreads, ImageMinCtas<Op, OutT>::value)
k_image(const __grid_constant__ ImageDesc im, const __grid_constant__ Coeffs co,
        const float *__restrict__ gamma, int64_t ntiles)
{
    __shared__ double sgam[256];
    __shared__ uint4 sbuf[Shape::vecs + Shape::scratch];
    load_table(TABLE, gamma, sgam);
    const Op op{reinterpret_cast<const float *>(sgam), co};
    run_image<kThreads, OutT, false>(im, ntiles, op, sbuf, nullptr, reinterpret_cast<float *>(sbuf + Shape::vecs));
}

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
    constexpr bool NR = sizeof(OutT) == 4;   // Newton step on the reciprocal for FP32 planes only
    switch (im.space) {
    case MACT_CIELAB:
        if (exact) return launch_one<OpCielab<true, 4>, OutT, kTable32>(h, im, s);
        if (rat && h.co.lab_deg == 6) return launch_one<OpCielab<false, 6, NR>, OutT, kTable32>(h, im, s);
        if (rat) return launch_one<OpCielab<false, 4, NR>, OutT, kTable32>(h, im, s);
        return launch_one<OpCielab<false, 0>, OutT, kTable64>(h, im, s);
    case MACT_CIELUV:
        if (exact) return launch_one<OpCieluv<true, 4>, OutT, kTable32>(h, im, s);
        if (rat && h.co.lab_deg == 6) return launch_one<OpCieluv<false, 6, NR>, OutT, kTable32>(h, im, s);
        if (rat) return launch_one<OpCieluv<false, 4, NR>, OutT, kTable32>(h, im, s);
        return launch_one<OpCieluv<false, 0>, OutT, kTable64>(h, im, s);
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

bool batch_cfg_supported(const BatchCfg &cfg)
{
#define MACT_SUPPORTED(T, S) if (cfg.threads == T && cfg.subs == S) return true;
    MACT_BATCH_SHAPES(MACT_SUPPORTED)
#undef MACT_SUPPORTED
    return false;
}

int batch_blocks_per_sm(const mact_ctx &h, const BatchCfg &cfg, bool param)
{
    if (h.cfg.exact) return batch_occ<true, 4>(cfg, param);
    if (!h.co.lab_rational) return batch_occ<false, 0>(cfg, param);
    return h.co.lab_deg == 6 ? batch_occ<false, 6>(cfg, param) : batch_occ<false, 4>(cfg, param);
}

cudaError_t launch_batch_param(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total, int grid,
                               cudaStream_t s, const BatchCfg &cfg)
{
    if (count < 1 || count > kParamImages) return cudaErrorInvalidValue;
    if (h.cfg.exact) return batch_launch_param<true, 4>(h, list, count, total, grid, s, cfg);
    if (!h.co.lab_rational) return batch_launch_param<false, 0>(h, list, count, total, grid, s, cfg);
    if (h.co.lab_deg == 6) return batch_launch_param<false, 6>(h, list, count, total, grid, s, cfg);
    return batch_launch_param<false, 4>(h, list, count, total, grid, s, cfg);
}

cudaError_t launch_batch(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count, int64_t total,
                         unsigned long long *d_ctr, int grid, cudaStream_t s, const BatchCfg &cfg)
{
    if (h.cfg.exact) return batch_launch<true, 4>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
    if (!h.co.lab_rational) return batch_launch<false, 0>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
    if (h.co.lab_deg == 6) return batch_launch<false, 6>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
    return batch_launch<false, 4>(h, d_imgs, count, total, d_ctr, grid, s, cfg);
}

}  // namespace mact
