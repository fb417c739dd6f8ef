// serve.cpp -- the served form: a conversion server with continuous
// batching over one GPU.
//
// Requests (one image each, host or device buffers, any space and dtype)
// are queued by mact_serve_submit.  Host buffers the kernel can address
// (pinned; any host memory where the device walks the host page tables) are
// read and written in place by the kernel in direct mode (the default); the
// others, and all host buffers in staged mode, go through a device staging
// arena.  One scheduler thread repeats a tick:
//   1. admit queued requests in arrival order while a slot is free, the
//      bytes every admitted request reads and writes (its input and output,
//      in place or staged) stay within the memory budget, and -- for staged
//      buffers -- the device staging arena (the budget's size, allocated
//      once at create) has room for the request's staged input and output;
//   2. for the requests admitted in this tick: copy host inputs to their
//      staging on the H2D stream, then -- on the compute stream, after
//      those copies -- convert all of them with ONE launch of the batched
//      work-list kernel, then copy host outputs back on the D2H stream;
//   3. retire requests whose completion event has fired (latency = submit
//      to completion seen by the scheduler), release their slot and arena
//      range; the events fire in admission order, so only the oldest is
//      queried.
// Requests that arrive while earlier ones are on the GPU are admitted in the
// next tick, so copies of one batch overlap the kernel of another
// (iteration-level continuous batching).  Nothing waits on the device
// without a bound: the scheduler polls events; mact_serve_wait and
// mact_serve_destroy take timeouts.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace mact {

namespace {

using Clock = std::chrono::steady_clock;

// NVTX range for profilers (Nsight Systems): the scheduler's admit, launch
// and retire steps appear as named ranges on its thread.  Without a tool
// attached, push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

double ms_since(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

enum ReqState { kQueued = 0, kInFlight = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

// Timing events of one tick's batch, shared by its requests: start (on the
// H2D stream, before the batch's input copies), in (after them), comp (after
// the kernel, on the compute stream).
struct BatchEvents {
    cudaEvent_t start = nullptr, in = nullptr, comp = nullptr;
    ~BatchEvents()
    {
        if (start) cudaEventDestroy(start);
        if (in) cudaEventDestroy(in);
        if (comp) cudaEventDestroy(comp);
    }
};

struct Request {
    uint64_t ticket = 0;
    mact_image img{};          // as submitted
    bool in_host = false, out_host = false;   // staged through the arena (else read/written in place)
    size_t in_bytes = 0, out_bytes = 0, elem = 4;
    size_t off = 0, len = 0;   // arena range
    size_t footprint = 0;      // input + output bytes, charged to the budget while admitted
    uint8_t *d_in = nullptr;
    void *d_out[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_out = nullptr;      // before the request's output copies (D2H stream)
    cudaEvent_t ev_done = nullptr;     // after them
    std::shared_ptr<BatchEvents> bev;
    Clock::time_point t_submit, t_admit, t_done;
    int state = kQueued;
    int64_t pixels = 0;
    std::string err;                   // why the request failed (reported by poll and wait)
};

// First-fit allocator over [0, size) in 256-byte units.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t len, size_t *off)
    {
        len = (len + 255) & ~size_t(255);
        if (len == 0) { *off = 0; return true; }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                size_t rest = it->second - len, start = it->first + len;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len)
    {
        len = (len + 255) & ~size_t(255);
        if (len == 0) return;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

enum PtrKind { kDevice = 0, kPinned = 1, kPageable = 2 };

PtrKind pointer_kind(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear: unknown pointers are pageable host memory
        return kPageable;
    }
    if (a.type == cudaMemoryTypeUnregistered) return kPageable;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer == p ? kPinned : kPageable;
    return kDevice;
}

}  // namespace

}  // namespace mact

using namespace mact;

struct mact_server {
    mact_handle h = nullptr;
    int device = 0;
    size_t budget = 0;
    int max_slots = 0;
    int mode = MACT_SERVE_DIRECT;          // how host buffers of new requests are used
    int fail_every = 0;                    // host-side fault injection (tests): fail every k-th batch
    int64_t batches_started = 0;
    void *arena_base = nullptr;
    Arena arena;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;

    std::mutex mu;
    std::condition_variable cv_work;     // submit -> scheduler
    std::condition_variable cv_done;     // scheduler -> waiters
    std::deque<Request *> queue;
    std::deque<Request *> inflight;      // admission order = completion order (one D2H stream)
    std::map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;

    // statistics over retired requests: submit-to-completion latency, and its
    // stages (admission wait on the host; on the device, the batch's input
    // copies, then kernel including its wait for the compute stream, then the
    // request's output copy including its wait for earlier output copies)
    size_t inflight_bytes = 0;           // footprints of the admitted, unretired requests (<= budget)
    size_t inflight_bytes_max = 0;
    std::vector<double> latencies;
    std::vector<double> st_queue, st_h2d, st_comp, st_d2h;
    double d2h_bytes = 0.0, d2h_busy_ms = 0.0;   // output copies to host: bytes, summed copy time
    int64_t pixels_done = 0, batches = 0, failed = 0;
    Clock::time_point t_first, t_last;
    bool any_done = false;
};

namespace mact {

static void fail_locked(mact_server *s, Request *r, const char *what, cudaError_t e)
{
    r->state = kFailed;
    r->t_done = Clock::now();
    r->err = std::string(what) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
    s->failed++;
}

// Wait, with a bound, until the server's three streams (which only the
// scheduler thread feeds) have drained; true if they all have.  After a
// failed tick, arena ranges are released only then: a range whose copies or
// kernel cannot be shown complete is leaked rather than reused under work in
// flight.
static bool streams_drained_within(const mact_server *s, double ms)
{
    const auto t0 = Clock::now();
    const cudaStream_t st[3] = {s->s_h2d, s->s_comp, s->s_d2h};
    for (int k = 0; k < 3;) {
        const cudaError_t q = cudaStreamQuery(st[k]);
        if (q == cudaSuccess) { ++k; continue; }
        if (q != cudaErrorNotReady) {
            cudaGetLastError();
            return false;
        }
        if (ms_since(t0, Clock::now()) > ms) return false;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return true;
}

// One scheduler tick: admit, launch, retire.  Returns true if it did work.
static bool serve_tick(mact_server *s)
{
    std::vector<Request *> batch;
    {
        NvtxRange range("mact_serve admit");
        std::unique_lock<std::mutex> lk(s->mu);
        while (!s->queue.empty() && (int)s->inflight.size() + (int)batch.size() < s->max_slots) {
            Request *r = s->queue.front();
            if (s->inflight_bytes + r->footprint > s->budget) break;   // FIFO: wait for budget
            size_t off = 0;
            if (!s->arena.alloc(r->in_bytes + r->out_bytes, &off)) break;   // FIFO: wait for room
            s->queue.pop_front();
            r->off = off;
            r->len = r->in_bytes + r->out_bytes;
            r->state = kInFlight;
            r->t_admit = Clock::now();
            s->inflight_bytes += r->footprint;
            s->inflight_bytes_max = std::max(s->inflight_bytes_max, s->inflight_bytes);
            batch.push_back(r);
        }
    }
    bool worked = !batch.empty();
    if (worked) {
        NvtxRange range("mact_serve launch");
        // stage pointers and H2D copies
        std::vector<mact_image> imgs;
        imgs.reserve(batch.size());
        auto bev = std::make_shared<BatchEvents>();
        cudaError_t e = cudaEventCreate(&bev->start);
        if (e == cudaSuccess) e = cudaEventCreate(&bev->in);
        if (e == cudaSuccess) e = cudaEventCreate(&bev->comp);
        if (e == cudaSuccess) e = cudaEventRecord(bev->start, s->s_h2d);
        for (Request *r : batch) {
            uint8_t *base = static_cast<uint8_t *>(s->arena_base) + r->off;
            mact_image im = r->img;
            const int64_t W = im.width, H = im.height;
            if (r->in_host) {
                r->d_in = base;
                const size_t sp = H == 1 ? (size_t)(3 * W) : (size_t)im.pitch_bytes;   // one row: pitch unused
                if (e == cudaSuccess) {
                    if (sp == (size_t)(3 * W))   // contiguous rows: one linear copy
                        e = cudaMemcpyAsync(r->d_in, im.rgb, (size_t)(3 * W) * H, cudaMemcpyHostToDevice, s->s_h2d);
                    else
                        e = cudaMemcpy2DAsync(r->d_in, 3 * W, im.rgb, sp, 3 * W, H, cudaMemcpyHostToDevice,
                                              s->s_h2d);
                }
                im.rgb = r->d_in;
                im.pitch_bytes = 3 * W;
            }
            if (r->out_host) {
                uint8_t *ob = base + ((r->in_bytes + 255) & ~size_t(255));
                for (int c = 0; c < 3; ++c) {
                    r->d_out[c] = ob + (size_t)c * W * H * r->elem;
                    im.out[c] = r->d_out[c];
                }
                im.out_pitch_elems = W;
            }
            imgs.push_back(im);
        }
        if (e == cudaSuccess) e = cudaEventRecord(bev->in, s->s_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->s_comp, bev->in, 0);
        mact_status st = MACT_OK;
        bool injected = false;
        if (e == cudaSuccess) {
            if (s->fail_every > 0 && ++s->batches_started % s->fail_every == 0) {
                st = MACT_E_NOMEM;   // injected on the host, after the input copies are enqueued
                injected = true;
            } else {
                st = mact_convert_batch(s->h, imgs.data(), (int32_t)imgs.size(), s->s_comp);
            }
        }
        if (e == cudaSuccess && st == MACT_OK) e = cudaEventRecord(bev->comp, s->s_comp);
        if (e == cudaSuccess && st == MACT_OK) e = cudaStreamWaitEvent(s->s_d2h, bev->comp, 0);
        for (Request *r : batch) {
            if (e != cudaSuccess || st != MACT_OK) break;
            const mact_image &im = r->img;
            const int64_t W = im.width, H = im.height;
            if (e == cudaSuccess) e = cudaEventCreate(&r->ev_out);
            if (e == cudaSuccess) e = cudaEventRecord(r->ev_out, s->s_d2h);
            if (r->out_host) {
                const size_t dp = H == 1 ? (size_t)W * r->elem : (size_t)im.out_pitch_elems * r->elem;
                const size_t row = (size_t)W * r->elem;
                const bool planes_adjacent = dp == row &&
                    static_cast<char *>(im.out[1]) == static_cast<char *>(im.out[0]) + row * H &&
                    static_cast<char *>(im.out[2]) == static_cast<char *>(im.out[1]) + row * H;
                if (planes_adjacent) {   // one linear copy of all three planes
                    e = cudaMemcpyAsync(im.out[0], r->d_out[0], 3 * row * H, cudaMemcpyDeviceToHost, s->s_d2h);
                } else {
                    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
                        if (dp == row)
                            e = cudaMemcpyAsync(im.out[c], r->d_out[c], row * H, cudaMemcpyDeviceToHost, s->s_d2h);
                        else
                            e = cudaMemcpy2DAsync(im.out[c], dp, r->d_out[c], row, row, H, cudaMemcpyDeviceToHost,
                                                  s->s_d2h);
                    }
                }
            }
            if (e == cudaSuccess) e = cudaEventCreate(&r->ev_done);
            if (e == cudaSuccess) e = cudaEventRecord(r->ev_done, s->s_d2h);
            r->bev = bev;
        }
        const bool failed = e != cudaSuccess || st != MACT_OK;
        // on failure, copies or the kernel already enqueued may still touch
        // the batch's arena ranges: release them only once the streams have
        // drained (bounded wait, outside the lock)
        const bool releasable = !failed || streams_drained_within(s, 5000.0);
        std::unique_lock<std::mutex> lk(s->mu);
        s->batches++;
        for (Request *r : batch) {
            if (failed || !r->ev_done) {
                fail_locked(s, r,
                            injected ? "mact_serve: batched conversion failed (injected)"
                                     : (st != MACT_OK ? "mact_serve: batched conversion failed" : "mact_serve"),
                            e);
                if (r->ev_out) cudaEventDestroy(r->ev_out);
                if (r->ev_done) cudaEventDestroy(r->ev_done);
                r->ev_out = r->ev_done = nullptr;
                r->bev.reset();
                if (releasable) {
                    s->arena.release(r->off, r->len);
                    s->inflight_bytes -= r->footprint;
                }
            } else {
                s->inflight.push_back(r);
            }
        }
        if (failed) s->cv_done.notify_all();
    }
    // retire: every request's completion event is recorded on the one D2H
    // stream, so they fire in admission order; query the oldest only
    NvtxRange range("mact_serve retire");
    std::unique_lock<std::mutex> lk(s->mu);
    bool retired = false;
    while (!s->inflight.empty()) {
        Request *r = s->inflight.front();
        cudaError_t q = cudaEventQuery(r->ev_done);
        if (q == cudaErrorNotReady) break;
        r->t_done = Clock::now();
        if (q == cudaSuccess) {
            r->state = kDone;
            s->latencies.push_back(ms_since(r->t_submit, r->t_done));
            float h2d = 0.0f, comp = 0.0f, d2h = 0.0f, copy = 0.0f;
            if (r->bev && cudaEventElapsedTime(&h2d, r->bev->start, r->bev->in) == cudaSuccess &&
                cudaEventElapsedTime(&comp, r->bev->in, r->bev->comp) == cudaSuccess &&
                cudaEventElapsedTime(&d2h, r->bev->comp, r->ev_done) == cudaSuccess &&
                cudaEventElapsedTime(&copy, r->ev_out, r->ev_done) == cudaSuccess) {
                s->st_queue.push_back(ms_since(r->t_submit, r->t_admit));
                s->st_h2d.push_back(h2d);
                s->st_comp.push_back(comp);
                s->st_d2h.push_back(d2h);
                if (r->out_host) {
                    s->d2h_bytes += (double)r->out_bytes;
                    s->d2h_busy_ms += copy;
                }
            } else {
                cudaGetLastError();
            }
            s->pixels_done += r->pixels;
            if (!s->any_done) { s->t_first = r->t_submit; s->any_done = true; }
            s->t_last = r->t_done;
        } else {
            fail_locked(s, r, "mact_serve: conversion or output copy failed", q);
        }
        cudaEventDestroy(r->ev_done);
        r->ev_done = nullptr;
        if (r->ev_out) cudaEventDestroy(r->ev_out);
        r->ev_out = nullptr;
        r->bev.reset();
        s->arena.release(r->off, r->len);
        s->inflight_bytes -= r->footprint;
        s->inflight.pop_front();
        retired = true;
    }
    if (retired) s->cv_done.notify_all();
    return worked || retired;
}

static void serve_loop(mact_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool worked = serve_tick(s);
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        if (!worked) {
            if (s->inflight.empty() && s->queue.empty())
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else
                s->cv_work.wait_for(lk, std::chrono::microseconds(20));   // poll completions
        }
    }
}

}  // namespace mact

extern "C" {

mact_status mact_serve_create(mact_handle h, size_t mem_budget_bytes, int32_t max_slots, mact_server_t *out)
{
    if (!h || !out) { set_error("mact_serve_create: NULL argument"); return MACT_E_INVAL; }
    if (max_slots < 1 || max_slots > 65536) { set_error("max_slots must be 1..65536"); return MACT_E_INVAL; }
    if (mem_budget_bytes < 4096) { set_error("mem_budget_bytes must be at least 4096"); return MACT_E_INVAL; }
    mact_server *s = new (std::nothrow) mact_server();
    if (!s) return MACT_E_NOMEM;
    s->h = h;
    s->device = h->device;
    s->budget = mem_budget_bytes & ~size_t(255);
    s->max_slots = max_slots;
    cudaError_t e = cudaSetDevice(s->device);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, s->budget);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        mact_status st = cuda_status(e, "mact_serve_create");
        if (s->arena_base) cudaFree(s->arena_base);
        if (s->s_h2d) cudaStreamDestroy(s->s_h2d);
        if (s->s_comp) cudaStreamDestroy(s->s_comp);
        if (s->s_d2h) cudaStreamDestroy(s->s_d2h);
        delete s;
        return st;
    }
    s->arena.reset(s->budget);
    if (const char *k = std::getenv("MACT_SERVE_FAIL_EVERY")) s->fail_every = std::atoi(k);
    s->worker = std::thread(serve_loop, s);
    *out = s;
    return MACT_OK;
}

mact_status mact_serve_set_mode(mact_server_t s, int32_t mode)
{
    if (!s) { set_error("mact_serve_set_mode: NULL server"); return MACT_E_INVAL; }
    if (mode != MACT_SERVE_DIRECT && mode != MACT_SERVE_STAGED) { set_error("unknown serve mode"); return MACT_E_INVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    s->mode = mode;
    return MACT_OK;
}

mact_status mact_serve_submit(mact_server_t s, const mact_image *img, uint64_t *ticket)
{
    if (!s || !img || !ticket) { set_error("mact_serve_submit: NULL argument"); return MACT_E_INVAL; }
    mact_status st = check_image(img);
    if (st != MACT_OK) return st;
    Request *r = new (std::nothrow) Request();
    if (!r) return MACT_E_NOMEM;
    r->img = *img;
    r->elem = img->dtype == MACT_F16 ? 2 : 4;
    r->pixels = img->width * img->height;
    if (r->pixels > 0) {
        const PtrKind kin = pointer_kind(img->rgb);
        const PtrKind kout = pointer_kind(img->out[0]);
        if ((kout == kDevice) != (pointer_kind(img->out[1]) == kDevice) ||
            (kout == kDevice) != (pointer_kind(img->out[2]) == kDevice)) {
            delete r;
            set_error("mact_serve_submit: output planes must all be on the host or all on the device");
            return MACT_E_INVAL;
        }
        // host memory is staged through the arena unless the kernel can
        // address it in place and the server runs in direct mode
        int mode;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            mode = s->mode;
        }
        auto staged = [&](PtrKind k) {
            if (k == kDevice) return false;
            if (mode == MACT_SERVE_STAGED) return true;
            return k == kPageable && !s->h->any_host;
        };
        r->in_host = staged(kin);
        r->out_host = false;
        for (int c = 0; c < 3; ++c) r->out_host = r->out_host || staged(pointer_kind(img->out[c]));
    }
    r->in_bytes = r->in_host ? (size_t)(3 * r->pixels) : 0;
    r->out_bytes = r->out_host ? (size_t)(3 * r->pixels) * r->elem : 0;
    r->footprint = (size_t)(3 * r->pixels) * (1 + r->elem);
    const size_t need = ((r->in_bytes + 255) & ~size_t(255)) + ((r->out_bytes + 255) & ~size_t(255));
    if (need > s->budget || r->footprint > s->budget) {
        delete r;
        set_error("mact_serve_submit: the request's input and output exceed the server's memory budget");
        return MACT_E_NOMEM;
    }
    r->in_bytes = (r->in_bytes + 255) & ~size_t(255);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete r; set_error("mact_serve_submit: server is shutting down"); return MACT_E_BUSY; }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        if (r->pixels == 0) {
            r->state = kDone;
            r->t_done = r->t_submit;
        } else {
            s->queue.push_back(r);
        }
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return MACT_OK;
}

mact_status mact_serve_poll(mact_server_t s, uint64_t ticket, int32_t *done, double *latency_ms)
{
    if (!s || !done) { set_error("mact_serve_poll: NULL argument"); return MACT_E_INVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("mact_serve_poll: unknown ticket"); return MACT_E_INVAL; }
    Request *r = it->second;
    *done = (r->state == kDone || r->state == kFailed || r->state == kCancelled) ? 1 : 0;
    if (latency_ms) *latency_ms = *done ? ms_since(r->t_submit, r->t_done) : 0.0;
    if (r->state == kFailed) {
        set_error(r->err);
        return MACT_E_CUDA;
    }
    return MACT_OK;
}

mact_status mact_serve_wait(mact_server_t s, uint64_t ticket, double timeout_ms, double *latency_ms)
{
    if (!s) { set_error("mact_serve_wait: NULL server"); return MACT_E_INVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("mact_serve_wait: unknown ticket"); return MACT_E_INVAL; }
    Request *r = it->second;
    auto pred = [r] { return r->state == kDone || r->state == kFailed || r->state == kCancelled; };
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) {
        set_error("mact_serve_wait: timed out");
        return MACT_E_TIMEOUT;
    }
    if (latency_ms) *latency_ms = ms_since(r->t_submit, r->t_done);
    if (r->state == kFailed) {
        set_error(r->err);
        return MACT_E_CUDA;
    }
    return MACT_OK;
}

mact_status mact_serve_cancel(mact_server_t s, uint64_t ticket)
{
    if (!s) { set_error("mact_serve_cancel: NULL server"); return MACT_E_INVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("mact_serve_cancel: unknown ticket"); return MACT_E_INVAL; }
    Request *r = it->second;
    if (r->state != kQueued) { set_error("mact_serve_cancel: request already admitted"); return MACT_E_BUSY; }
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    r->state = kCancelled;
    r->t_done = Clock::now();
    s->cv_done.notify_all();
    return MACT_OK;
}

mact_status mact_serve_release(mact_server_t s, uint64_t ticket)
{
    if (!s) { set_error("mact_serve_release: NULL server"); return MACT_E_INVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) { set_error("mact_serve_release: unknown ticket"); return MACT_E_INVAL; }
    Request *r = it->second;
    if (r->state == kQueued || r->state == kInFlight) { set_error("mact_serve_release: request pending"); return MACT_E_BUSY; }
    s->reqs.erase(it);
    delete r;
    return MACT_OK;
}

mact_status mact_serve_stats(mact_server_t s, mact_serve_stats_t *out)
{
    if (!s || !out) { set_error("mact_serve_stats: NULL argument"); return MACT_E_INVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    auto pct = [](std::vector<double> v, double p) {
        if (v.empty()) return 0.0;
        std::sort(v.begin(), v.end());
        size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * (v.size() - 1) + 0.5));
        return v[k];
    };
    out->queue_p50_ms = pct(s->st_queue, 0.50);
    out->h2d_p50_ms = pct(s->st_h2d, 0.50);
    out->compute_p50_ms = pct(s->st_comp, 0.50);
    out->d2h_p50_ms = pct(s->st_d2h, 0.50);
    out->queue_p99_ms = pct(s->st_queue, 0.99);
    out->h2d_p99_ms = pct(s->st_h2d, 0.99);
    out->compute_p99_ms = pct(s->st_comp, 0.99);
    out->d2h_p99_ms = pct(s->st_d2h, 0.99);
    out->d2h_copy_gbs = s->d2h_busy_ms > 0 ? s->d2h_bytes / (s->d2h_busy_ms * 1e-3) / 1e9 : 0.0;
    out->d2h_busy_ms = s->d2h_busy_ms;
    std::vector<double> l = s->latencies;
    out->completed = (int64_t)l.size();
    out->failed = s->failed;
    out->batches = s->batches;
    out->queued = (int64_t)s->queue.size();
    out->in_flight = (int64_t)s->inflight.size();
    out->pixels = s->pixels_done;
    out->inflight_bytes_max = (int64_t)s->inflight_bytes_max;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        out->p50_ms = pct(l, 0.50);
        out->p99_ms = pct(l, 0.99);
        out->max_ms = l.back();
        const double span = ms_since(s->t_first, s->t_last);
        out->gpix_per_s = span > 0 ? (double)s->pixels_done / (span * 1e-3) / 1e9 : 0.0;
    }
    return MACT_OK;
}

mact_status mact_serve_destroy(mact_server_t s, double timeout_ms)
{
    if (!s) { set_error("mact_serve_destroy: NULL server"); return MACT_E_INVAL; }
    mact_status st = MACT_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
        // bounded drain: everything queued or in flight must finish in time
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                 [s] { return s->queue.empty() && s->inflight.empty(); })) {
            // cancel what was never admitted; in-flight work still completes
            for (Request *r : s->queue) { r->state = kCancelled; r->t_done = Clock::now(); }
            s->queue.clear();
            st = MACT_E_TIMEOUT;
            set_error("mact_serve_destroy: drain timed out; queued requests cancelled");
        }
    }
    s->cv_work.notify_all();
    s->worker.join();   // the loop ends once in-flight work has retired
    cudaStreamSynchronize(s->s_h2d);
    cudaStreamSynchronize(s->s_comp);
    cudaStreamSynchronize(s->s_d2h);
    cudaStreamDestroy(s->s_h2d);
    cudaStreamDestroy(s->s_comp);
    cudaStreamDestroy(s->s_d2h);
    cudaFree(s->arena_base);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return st;
}

}  // extern "C"
