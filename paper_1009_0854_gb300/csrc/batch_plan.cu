// batch_plan.cu -- the batched form for repeated work lists, and its
// autotuner.
//
// A plan fixes one list of images (pointers, sizes, spaces, dtypes) and a
// launch shape: the device work list is built and uploaded once, so each
// launch is a single kernel with no host work, no copies and no allocation.
// That makes it capturable: mact_batch_plan_graph_launch captures the launch
// into a CUDA graph once and replays the graph afterwards (the kernel's tile
// counters reset themselves at the end of every launch).
//
// mact_autotune_batch times every supported launch shape (threads per CTA,
// pixels per thread -- hence tile size -- and resident CTAs per SM) on the
// caller's own images and keeps the fastest in the handle.
#include <cstring>
#include <vector>

#include "internal.h"

struct mact_batch_plan {
    mact_handle h = nullptr;
    mact::BatchCfg cfg;
    void *d_buf = nullptr;           // [256 B counters][ImageDesc x n]
    int32_t n = 0;
    int64_t total = 0;
    int grid = 0;
    cudaStream_t cap = nullptr;      // private stream used only to capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace mact {

static mact_status plan_build(mact_handle h, const mact_image *imgs, int32_t count, const BatchCfg &cfg,
                              mact_batch_plan **out)
{
    if (!h || !out) { set_error("mact_batch_plan_create: NULL argument"); return MACT_E_INVAL; }
    if (count < 0 || (count > 0 && !imgs)) { set_error("mact_batch_plan_create: bad image list"); return MACT_E_INVAL; }
    if (!batch_cfg_supported(cfg)) { set_error("unsupported batch launch shape"); return MACT_E_UNSUPPORTED; }
    for (int32_t i = 0; i < count; ++i) {
        mact_status st = check_image(&imgs[i]);
        if (st == MACT_OK) st = check_image_access(*h, imgs[i]);
        if (st != MACT_OK) return st;
    }
    std::vector<ImageDesc> list;
    list.reserve(count);
    int64_t total = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (imgs[i].width == 0 || imgs[i].height == 0) continue;
        ImageDesc d = make_desc(imgs[i], cfg.tile_px());
        d.tile_begin = total;
        total += tiles_of(d);
        list.push_back(d);
    }
    mact_batch_plan *p = new (std::nothrow) mact_batch_plan();
    if (!p) return MACT_E_NOMEM;
    p->h = h;
    p->cfg = cfg;
    p->n = (int32_t)list.size();
    p->total = total;
    int per_sm = batch_blocks_per_sm(*h, cfg);
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    int64_t grid = (int64_t)h->num_sms * per_sm;
    p->grid = (int)(grid < total ? grid : (total > 0 ? total : 1));
    cudaError_t e = cudaMalloc(&p->d_buf, 256 + list.size() * sizeof(ImageDesc) + 16);
    if (e == cudaSuccess) e = cudaMemset(p->d_buf, 0, 256);
    if (e == cudaSuccess && !list.empty())
        e = cudaMemcpy(static_cast<char *>(p->d_buf) + 256, list.data(), list.size() * sizeof(ImageDesc),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mact_status st = cuda_status(e, "mact_batch_plan_create");
        if (p->d_buf) cudaFree(p->d_buf);
        delete p;
        return st;
    }
    *out = p;
    return MACT_OK;
}

static cudaError_t plan_enqueue(mact_batch_plan *p, cudaStream_t s)
{
    if (p->total == 0) return cudaSuccess;
    auto *ctr = static_cast<unsigned long long *>(p->d_buf);
    auto *imgs = reinterpret_cast<const ImageDesc *>(static_cast<char *>(p->d_buf) + 256);
    return launch_batch(*p->h, imgs, p->n, p->total, ctr, p->grid, s, p->cfg);
}

}  // namespace mact

using namespace mact;

extern "C" {

mact_status mact_batch_plan_create(mact_handle h, const mact_image *imgs, int32_t count, mact_batch_plan_t *out)
{
    if (!h) { set_error("mact_batch_plan_create: NULL handle"); return MACT_E_INVAL; }
    return plan_build(h, imgs, count, h->batch_cfg, out);
}

mact_status mact_batch_plan_launch(mact_batch_plan_t p, mact_stream stream)
{
    if (!p) { set_error("mact_batch_plan_launch: NULL plan"); return MACT_E_INVAL; }
    return cuda_status(plan_enqueue(p, (cudaStream_t)stream), "mact_batch_plan_launch");
}

mact_status mact_batch_plan_graph_launch(mact_batch_plan_t p, mact_stream stream)
{
    if (!p) { set_error("mact_batch_plan_graph_launch: NULL plan"); return MACT_E_INVAL; }
    cudaError_t e = cudaSuccess;
    if (!p->exec) {
        if (!p->cap) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = plan_enqueue(p, p->cap);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(p->cap, &g);
            if (le != cudaSuccess) e = le;
            if (e == cudaSuccess) {
                p->graph = g;
                e = cudaGraphInstantiate(&p->exec, p->graph, 0);
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        if (e != cudaSuccess) return cuda_status(e, "mact_batch_plan_graph_launch: capture");
    }
    return cuda_status(cudaGraphLaunch(p->exec, (cudaStream_t)stream), "mact_batch_plan_graph_launch");
}

mact_status mact_batch_plan_destroy(mact_batch_plan_t p)
{
    if (!p) { set_error("mact_batch_plan_destroy: NULL plan"); return MACT_E_INVAL; }
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->d_buf) cudaFree(p->d_buf);
    delete p;
    return MACT_OK;
}

mact_status mact_autotune_batch(mact_handle h, const mact_image *imgs, int32_t count, int32_t reps,
                                mact_tune_entry *table, int32_t table_cap, int32_t *n_entries)
{
    if (!h) { set_error("mact_autotune_batch: NULL handle"); return MACT_E_INVAL; }
    if (reps < 1) reps = 5;
    static const int shapes[][2] = {{128, 4}, {256, 4}, {512, 4}, {256, 8}, {128, 8}};
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_status(e, "mact_autotune_batch");
    BatchCfg best = h->batch_cfg;
    float best_ms = 1e30f;
    int32_t k = 0;
    mact_status st = MACT_OK;
    for (const auto &sh : shapes) {
        BatchCfg probe;
        probe.threads = sh[0];
        probe.subs = sh[1];
        const int full = batch_blocks_per_sm(*h, probe);
        const int cands[2] = {0, full > 2 ? full / 2 : 0};
        for (int ci = 0; ci < 2; ++ci) {
            if (ci == 1 && cands[1] == 0) continue;
            BatchCfg cfg = probe;
            cfg.ctas_per_sm = cands[ci];
            mact_batch_plan *p = nullptr;
            st = plan_build(h, imgs, count, cfg, &p);
            if (st != MACT_OK) break;
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = plan_enqueue(p, s);
            if (e == cudaSuccess) e = cudaEventRecord(a, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = plan_enqueue(p, s);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            mact_batch_plan_destroy(p);
            if (e != cudaSuccess) break;
            ms /= (float)reps;
            if (table && k < table_cap) {
                table[k].threads = cfg.threads;
                table[k].px_per_thread = 4 * cfg.subs;
                table[k].ctas_per_sm = cfg.ctas_per_sm ? cfg.ctas_per_sm : full;
                table[k].ms = ms;
            }
            ++k;
            if (ms < best_ms) {
                best_ms = ms;
                best = cfg;
            }
        }
        if (st != MACT_OK || e != cudaSuccess) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    if (st != MACT_OK) return st;
    if (e != cudaSuccess) return cuda_status(e, "mact_autotune_batch");
    {
        std::lock_guard<std::mutex> lock(h->batch_mu);
        h->batch_cfg = best;
    }
    if (n_entries) *n_entries = k;
    return MACT_OK;
}

mact_status mact_set_batch_shape(mact_handle h, int32_t threads, int32_t px_per_thread, int32_t ctas_per_sm)
{
    if (!h) { set_error("mact_set_batch_shape: NULL handle"); return MACT_E_INVAL; }
    BatchCfg cfg;
    cfg.threads = threads;
    cfg.subs = px_per_thread / 4;
    cfg.ctas_per_sm = ctas_per_sm < 0 ? 0 : ctas_per_sm;
    if (px_per_thread % 4 != 0 || !batch_cfg_supported(cfg)) {
        set_error("unsupported batch launch shape");
        return MACT_E_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(h->batch_mu);
    h->batch_cfg = cfg;
    return MACT_OK;
}

mact_status mact_get_batch_shape(mact_handle h, int32_t *threads, int32_t *px_per_thread, int32_t *ctas_per_sm)
{
    if (!h || !threads || !px_per_thread || !ctas_per_sm) { set_error("NULL argument"); return MACT_E_INVAL; }
    std::lock_guard<std::mutex> lock(h->batch_mu);
    *threads = h->batch_cfg.threads;
    *px_per_thread = 4 * h->batch_cfg.subs;
    *ctas_per_sm = h->batch_cfg.ctas_per_sm;
    return MACT_OK;
}

}  // extern "C"
