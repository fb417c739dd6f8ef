// noalloc.cu -- mact_convert_batch_static: the batched conversion with its
// scratch memory (tile counters + image work list) in a fixed device array
// compiled into the library, for callers that must not allocate.
//
// Who needs it: code that runs where a cudaMalloc is not allowed or not
// wanted -- a real-time or safety-certified pipeline whose memory is fixed
// at start-up, a host callback or a plug-in that must not touch the
// allocator, a process whose device memory is fully reserved by another
// framework's pool.  mact_convert_batch grows its work list with
// cudaMalloc/cudaMallocHost on demand; this entry point never allocates.
//
// The scratch is g_batch_scratch below: 256 bytes of counters followed by
// room for kStaticMaxImages image descriptors.  Every GPU that loads the
// library holds it until the process exits.  Host code cannot use the
// symbol as a device address, so each device's address is looked up once
// with cudaGetSymbolAddress (with that device current) and cached.
//
// The work list reaches the array without any host staging buffer: each
// chunk of descriptors travels by value in the parameter block of a small
// upload kernel (the launch copies the parameters when it is enqueued, so no
// host memory is read after the call returns), and that kernel writes the
// chunk into the array.  The first chunk also zeroes the tile counters.
// Lists of at most kParamImages images skip the array altogether: they go by
// value to the batched kernel itself, exactly as in mact_convert_batch.
#include <mutex>

#include "internal.h"

namespace mact {

constexpr int32_t kStaticMaxImages = 1024;
constexpr size_t kStaticCounterBytes = 256;
constexpr size_t kStaticScratchBytes = kStaticCounterBytes + kStaticMaxImages * sizeof(ImageDesc);
constexpr int kStaticMaxDevices = 64;
// descriptors per upload launch: 256 x 88 B = 22.5 KB of kernel parameters
// (within the 32,764-byte parameter limit of CUDA 12.1 and later)
constexpr int32_t kStaticChunk = 256;

static __device__ __align__(256) unsigned char g_batch_scratch[kStaticScratchBytes];

struct StaticChunk {
    ImageDesc img[kStaticChunk];
};
static_assert(sizeof(StaticChunk) + 16 <= 32764, "upload chunk exceeds the kernel parameter limit");
static_assert(kStaticMaxImages % kStaticChunk == 0, "whole chunks");

// Writes descriptors [first, first + n) of the work list; zero_ctr: also
// reset the two tile counters (the array keeps the previous call's values).
__global__ void __launch_bounds__(kStaticChunk)
k_static_upload(const __grid_constant__ StaticChunk chunk, int32_t n, int32_t first, int32_t zero_ctr)
{
    ImageDesc *list = reinterpret_cast<ImageDesc *>(g_batch_scratch + kStaticCounterBytes);
    const int i = threadIdx.x;
    if (i < n) list[first + i] = chunk.img[i];
    if (zero_ctr && i < 2) reinterpret_cast<unsigned long long *>(g_batch_scratch)[i] = 0ull;
}

namespace {

std::mutex g_static_mu;                       // guards the table below
void *g_static_ptr[kStaticMaxDevices];        // device address of g_batch_scratch, per device

// Device address of the scratch array on the current device (set-up on the
// first call per device).  Called with g_static_mu held.
mact_status static_scratch(int dev, void **out)
{
    if (dev < 0 || dev >= kStaticMaxDevices) {
        set_error("mact_convert_batch_static: device ordinal out of range");
        return MACT_E_UNSUPPORTED;
    }
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch_static: cudaGetSymbolAddress");
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return MACT_OK;
}

}  // namespace

}  // namespace mact

using namespace mact;

extern "C" mact_status mact_convert_batch_static(mact_handle h, const mact_image *imgs, int32_t count,
                                                 mact_stream stream)
{
    if (!h) {
        set_error("mact_convert_batch_static: NULL handle");
        return MACT_E_INVAL;
    }
    if (count < 0 || count > kStaticMaxImages) {
        set_error("mact_convert_batch_static: count must be 0..1024 (the size of the static work list)");
        return MACT_E_INVAL;
    }
    if (count > 0 && !imgs) {
        set_error("mact_convert_batch_static: imgs is NULL");
        return MACT_E_INVAL;
    }
    for (int32_t i = 0; i < count; ++i) {
        mact_status st = check_image(&imgs[i]);
        if (st == MACT_OK) st = check_image_access(*h, imgs[i]);
        if (st != MACT_OK) return st;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch_static: cudaGetDevice");
    if (dev != h->device) {
        // the handle's coefficient and gamma pointers belong to its own device
        set_error("mact_convert_batch_static: the current device is not the handle's device");
        return MACT_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BatchCfg cfg;
    {
        std::lock_guard<std::mutex> lock(h->batch_mu);
        cfg = h->batch_cfg;
    }
    // resident CTAs per SM of the kernel form that runs: by value or from the list
    auto per_sm_of = [&](bool param) {
        int per_sm = batch_blocks_per_sm(*h, cfg, param);
        return (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) ? cfg.ctas_per_sm : per_sm;
    };

    int32_t nonempty = 0;
    for (int32_t i = 0; i < count; ++i) nonempty += (imgs[i].width != 0 && imgs[i].height != 0);
    if (nonempty == 0) return MACT_OK;
    if (nonempty <= kParamImages) {   // short list: by value to the batched kernel, no scratch
        ParamList list{};
        int64_t total = 0;
        int32_t n = 0;
        for (int32_t i = 0; i < count; ++i) {
            if (imgs[i].width == 0 || imgs[i].height == 0) continue;
            ImageDesc d = make_desc(imgs[i], cfg.tile_px());
            d.tile_begin = total;
            total += tiles_of(d);
            list.img[n++] = d;
        }
        int64_t grid = (int64_t)h->num_sms * per_sm_of(true);
        if (grid > total) grid = total;
        return cuda_status(launch_batch_param(*h, list, n, total, (int)grid, s, cfg),
                           "mact_convert_batch_static launch");
    }

    std::lock_guard<std::mutex> lock(g_static_mu);
    void *scratch = nullptr;
    mact_status st = static_scratch(dev, &scratch);
    if (st != MACT_OK) return st;
    unsigned long long *d_ctr = reinterpret_cast<unsigned long long *>(scratch);
    ImageDesc *d_imgs = reinterpret_cast<ImageDesc *>(static_cast<unsigned char *>(scratch) + kStaticCounterBytes);

    StaticChunk chunk;   // on the host stack; copied into each launch's parameters
    int64_t total = 0;
    int32_t n = 0, fill = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (imgs[i].width == 0 || imgs[i].height == 0) continue;
        ImageDesc d = make_desc(imgs[i], cfg.tile_px());
        d.tile_begin = total;
        total += tiles_of(d);
        chunk.img[fill++] = d;
        ++n;
        if (fill == kStaticChunk || n == nonempty) {
            k_static_upload<<<1, kStaticChunk, 0, s>>>(chunk, fill, n - fill, n == fill ? 1 : 0);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch_static: work list upload");
            fill = 0;
        }
    }
    int64_t grid = (int64_t)h->num_sms * per_sm_of(false);
    if (grid > total) grid = total;
    return cuda_status(launch_batch(*h, d_imgs, n, total, d_ctr, (int)grid, s, cfg),
                       "mact_convert_batch_static launch");
}
