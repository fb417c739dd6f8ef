// internal.h -- host-side state of a libmact handle and the launchers each
// kernel file provides.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace mact {
// Launch shape of the batched kernel: threads per CTA, sub-blocks per tile
// (tile = threads * 4 * subs pixels) and resident CTAs per SM (0: as many as
// fit).  Chosen by mact_autotune_batch; the default is 256 x 4 x full.
struct BatchCfg {
    int threads = 256;
    int subs = 4;
    int ctas_per_sm = 0;
    int64_t tile_px() const { return (int64_t)threads * 4 * subs; }
};
}  // namespace mact

struct mact_ctx {
    int device = 0;
    int num_sms = 0;
    // 1: the device addresses any host memory through the host page tables,
    // and pointers are not checked; 0: only device, pinned and registered host
    // memory, checked before every launch
    int any_host = 0;
    mact_config cfg{};
    mact::Coeffs co{};
    float *d_gamma = nullptr;            // 256 FP32 then 256 FP64 entries (Eq. equ_rgb_lin of each code)

    // batched form: a ring of work-list slots, so consecutive calls pipeline
    // (a slot is reused only after the call that last used it has copied its
    // list and finished its kernel)
    struct BatchSlot {
        mact::ImageDesc *h_work = nullptr;   // pinned staging
        void *d_work = nullptr;              // [256 B: 2 x u64 counters][ImageDesc x cap]
        int64_t cap = 0;
        cudaEvent_t ev_copy = nullptr;       // staging copy finished
        cudaEvent_t ev_kernel = nullptr;     // batch kernel finished
    };
    static constexpr int kBatchSlots = 4;
    std::mutex batch_mu;
    BatchSlot batch_slots[kBatchSlots];
    int batch_next = 0;
    mact::BatchCfg batch_cfg;            // used by mact_convert_batch and new plans

    // LUT interpolation from an unpacked LUT with n > 17: packed copy
    // (launch_lut_pack), repacked on every call, grown on demand
    std::mutex lut_mu;
    float *d_lut4 = nullptr;
    int64_t lut4_cap = 0;                // nodes
    cudaEvent_t ev_lut = nullptr;        // last interpolation kernel that read d_lut4

    // differentiable CIELAB: per-CTA partial sums of the loss (SMs x 8 doubles)
    std::mutex grad_mu;
    double *d_partial = nullptr;
    cudaEvent_t ev_grad = nullptr;       // last loss reduction that read d_partial
};

namespace mact {

void set_error(const std::string &msg);
mact_status cuda_status(cudaError_t e, const char *what);

// k_convert.cu
cudaError_t launch_convert(const mact_ctx &h, const ImageDesc &im, cudaStream_t s);
cudaError_t launch_batch(const mact_ctx &h, const ImageDesc *d_imgs, int32_t count,
                         int64_t total_tiles, unsigned long long *d_counters, int grid,
                         cudaStream_t s, const BatchCfg &cfg = BatchCfg());
// the same for at most kParamImages images, the list passed by value in the
// kernel parameters (no device list, no counters)
cudaError_t launch_batch_param(const mact_ctx &h, const ParamList &list, int32_t count, int64_t total_tiles,
                               int grid, cudaStream_t s, const BatchCfg &cfg);
// resident CTAs per SM of the device-list kernel, or (param) of the by-value one
int batch_blocks_per_sm(const mact_ctx &h, const BatchCfg &cfg = BatchCfg(), bool param = false);
bool batch_cfg_supported(const BatchCfg &cfg);

constexpr int kLutSmemMaxN = 17;   // largest LUT staged whole in every CTA's shared memory

// k_lut_inst.cu (one object per method): interpolation from a packed float3
// LUT (lut) or a float4 copy (lut4), and from the caching layout
template <int METHOD, bool SEL>
cudaError_t lut_interp_method(const mact_ctx &h, const float *lut, const float4 *lut4, int n, const uint8_t *rgb,
                              int64_t npix, float *const out[3], int32_t *sel, cudaStream_t s);
template <int METHOD, bool SEL>
cudaError_t lut_cached_method(const mact_ctx &h, const float4 *cache, int n, const uint8_t *rgb, int64_t npix,
                              float *const out[3], int32_t *sel, cudaStream_t s);

// k_lut.cu
cudaError_t launch_lut_build(const mact_ctx &h, int n, float *d_lut, cudaStream_t s);
// nodes from d_lut4 (the packed layout of launch_lut_pack) when given, else
// from d_lut (float3); n > 17 needs d_lut4
cudaError_t launch_lut_interp(const mact_ctx &h, int method, const float *d_lut, const float4 *d_lut4, int n,
                              const uint8_t *d_rgb, int64_t npix, float *const out[3], int32_t *d_sel,
                              cudaStream_t s);
bool lut_needs_pack(int n);
cudaError_t launch_lut_pack4(const float *d_lut, int n, float4 *d_lut4, cudaStream_t s);
// the packed layout of mact_lut_pack (19 n^3 floats, m = n^3): float4
// nodes[m], float4 B-edge xy[m], float4 R-edge xy[m], float2 B-edge z[m],
// float2 R-edge z[m], float2 node xy plane[m], float node z plane[m].  Every
// array starts at a multiple of its element size times m bytes from a
// 16-byte aligned base (float4 arrays first, then float2, then float), so
// each is aligned to its element size for any n.
constexpr int kLutPackedFloats = 19;
struct PackedLut {
    const float4 *nodes;
    const float4 *bxy, *rxy;
    const float2 *bz, *rz;
    const float2 *pxy;
    const float *pz;
};
__host__ __device__ inline PackedLut packed_lut(const float4 *p, int n)
{
    const int64_t m = (int64_t)n * n * n;
    PackedLut k;
    k.nodes = p;
    k.bxy = p + m;
    k.rxy = p + 2 * m;
    k.bz = reinterpret_cast<const float2 *>(p + 3 * m);
    k.rz = k.bz + m;
    k.pxy = k.rz + m;
    k.pz = reinterpret_cast<const float *>(k.pxy + m);
    return k;
}
cudaError_t launch_lut_pack(const float *d_lut, int n, float *d_packed, cudaStream_t s);
cudaError_t launch_lut_cache_build(const float *d_lut, int n, float4 *d_cache, cudaStream_t s);

// k_lut_hsi.cu: HSI LUT of (cos H, sin H, S, I) nodes, trilinear with the
// angular hue mix
cudaError_t launch_lut_build_hsi(int n, float4 *d_lut4, cudaStream_t s);
cudaError_t launch_lut_interp_hsi(const mact_ctx &h, const float4 *d_lut4, int n, const uint8_t *d_rgb,
                                  int64_t npix, float *const out[3], cudaStream_t s);
cudaError_t launch_lut_interp_cached(const mact_ctx &h, int method, const float4 *d_cache, int n,
                                     const uint8_t *d_rgb, int64_t npix, float *const out[3], int32_t *d_sel,
                                     cudaStream_t s);

// k_grad.cu
cudaError_t launch_lab_forward(const mact_ctx &h, const float *x, int64_t nb, int64_t hw, float *lab,
                               cudaStream_t s);
cudaError_t launch_lab_backward(const mact_ctx &h, const float *x, const float *glab, int64_t nb, int64_t hw,
                                float *gx, cudaStream_t s);
cudaError_t launch_lab_delta_e(const mact_ctx &h, const float *x, const float *tgt, int64_t nb, int64_t hw,
                               float *loss, float *gx, double *partial, cudaStream_t s);

// k_eps.cu: error statistics over all 2^24 colours (target 0..2: space of the
// handle's transform; 3: LUT method with float4 nodes)
cudaError_t run_cube_error(const mact_ctx &h, int target, int method, const float4 *d_lut4, int n,
                           double out[2], cudaStream_t s);

// tile count of an image descriptor (height x tiles per row)
int64_t tiles_of(const ImageDesc &im);

// api.cu: argument validation of one image, and its engine descriptor for
// tiles of tile_px pixels
mact_status check_image(const mact_image *img);
ImageDesc make_desc(const mact_image &img, int64_t tile_px = kTile);

// api.cu: whether the kernels may dereference p (see mact_host_memory_access);
// check_image_access applies it to an image's four pointers
mact_status check_access(const mact_ctx &h, const void *p, const char *what);
mact_status check_image_access(const mact_ctx &h, const mact_image &img);

}  // namespace mact
