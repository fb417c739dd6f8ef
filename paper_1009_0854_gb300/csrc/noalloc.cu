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
#include <mutex>

#include "internal.h"

namespace mact {

constexpr int32_t kStaticMaxImages = 1024;
constexpr size_t kStaticCounterBytes = 256;
constexpr size_t kStaticScratchBytes = kStaticCounterBytes + kStaticMaxImages * sizeof(ImageDesc);
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_batch_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mu;                       // guards the tables below
void *g_static_ptr[kStaticMaxDevices];        // device address of g_batch_scratch, per device
ImageDesc g_static_host[kStaticMaxImages];    // host-side work list staging (static, not heap)

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
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_static_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch_static: cudaGetDevice");
    void *scratch = nullptr;
    mact_status st = static_scratch(dev, &scratch);
    if (st != MACT_OK) return st;

    int64_t total = 0;
    int32_t n = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (imgs[i].width == 0 || imgs[i].height == 0) continue;
        ImageDesc d = make_desc(imgs[i]);
        d.tile_begin = total;
        total += tiles_of(d);
        g_static_host[n++] = d;
    }
    if (total == 0) return MACT_OK;
    unsigned long long *d_ctr = reinterpret_cast<unsigned long long *>(scratch);
    ImageDesc *d_imgs = reinterpret_cast<ImageDesc *>(static_cast<unsigned char *>(scratch) + kStaticCounterBytes);
    // the array keeps the previous call's contents: the tile counters must
    // start at zero.  The copy is from pageable host memory, so it has
    // consumed g_static_host when cudaMemcpyAsync returns.
    e = cudaMemsetAsync(d_ctr, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_imgs, g_static_host, n * sizeof(ImageDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch_static: work list upload");
    int64_t grid = (int64_t)h->num_sms * batch_blocks_per_sm(*h);
    if (grid > total) grid = total;
    return cuda_status(launch_batch(*h, d_imgs, n, total, d_ctr, (int)grid, s), "mact_convert_batch_static launch");
}
