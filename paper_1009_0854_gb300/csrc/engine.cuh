// engine.cuh -- the streaming tile engine shared by the transform and LUT
// kernels: interleaved uint8 RGB in, three planes (and optionally a
// per-pixel int32) out.
//
// The work is HBM-bound by design (3 bytes read, 12 (FP32) or 6 (FP16) bytes
// written per pixel, nothing reused), so the engine's job is to keep the
// per-pixel instruction count low and the memory system busy:
//   * a tile is THREADS x 4*SUBS pixels (SUBS = 4 or 8 sub-blocks; 12 or 24
//     bytes of input per thread); every thread loads exactly 3*SUBS/4 16-byte
//     vectors of it (coalesced, streaming hint) and stages them in shared
//     memory;
//   * each thread then de-interleaves 4 consecutive pixels at a time from
//     three 32-bit shared-memory words (stride 3 words across a warp: no bank
//     conflicts), SUBS times per tile, and writes each plane's 4 results as
//     one 16-byte (FP32) or 8-byte (FP16) streaming store -- a warp writes
//     512 contiguous bytes per store instruction;
//   * for contiguous, aligned images the persistent loop prefetches the next
//     tile into registers while it computes the current one, and computes
//     tile addresses with one multiply (no per-tile division);
//   * pitched rows, misaligned pointers and the final partial tile take a
//     guarded path (byte loads, per-pixel stores) that gives identical values.
#pragma once

#include "common.cuh"

namespace mact {

constexpr int kSubBlocks = 4;                        // default sub-blocks per tile

template <int THREADS, int SUBS = kSubBlocks>
struct TileShape {
    static_assert(SUBS % 4 == 0, "whole 16-byte vectors per thread");
    static constexpr int sub = THREADS * kPxPerThread;   // pixels per sub-block
    static constexpr int px = sub * SUBS;                // pixels per tile
    static constexpr int vpt = 3 * SUBS / 4;             // 16-byte input vectors per thread
    static constexpr int vecs = vpt * THREADS;           // 16-byte input vectors per tile
    static constexpr int scratch = THREADS;              // 16-byte vectors of transpose scratch (shifted path)
};

template <int THREADS, int SUBS = kSubBlocks>
__host__ __device__ inline int64_t tiles_of_t(const ImageDesc &im)
{
    constexpr int P = TileShape<THREADS, SUBS>::px;
    if (im.width <= 0 || im.height <= 0) return 0;
    return im.height * ((im.width + P - 1) / P);
}

// An image is streamable when it is one contiguous row with every base
// pointer aligned for the vector accesses.
template <typename OutT, bool SEL>
__device__ __forceinline__ bool streamable(const ImageDesc &im, const int32_t *sel)
{
    constexpr uintptr_t omask = sizeof(OutT) == 4 ? 15 : 7;
    uintptr_t oa = reinterpret_cast<uintptr_t>(im.out[0]) | reinterpret_cast<uintptr_t>(im.out[1]) |
                   reinterpret_cast<uintptr_t>(im.out[2]);
    bool ok = im.height == 1 && ((reinterpret_cast<uintptr_t>(im.rgb) & 15) == 0) && ((oa & omask) == 0);
    if (SEL) ok = ok && ((reinterpret_cast<uintptr_t>(sel) & 15) == 0);
    return ok;
}

template <int THREADS, int SUBS>
__device__ __forceinline__ void load_tile(uint4 (&v)[TileShape<THREADS, SUBS>::vpt], const uint8_t *in)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(in) + threadIdx.x;
#pragma unroll
    for (int k = 0; k < TileShape<THREADS, SUBS>::vpt; ++k) v[k] = __ldcs(p + k * THREADS);
}

template <int THREADS, int SUBS>
__device__ __forceinline__ void stage_tile(uint4 *sbuf, const uint4 (&v)[TileShape<THREADS, SUBS>::vpt])
{
#pragma unroll
    for (int k = 0; k < TileShape<THREADS, SUBS>::vpt; ++k) sbuf[threadIdx.x + k * THREADS] = v[k];
}

// Apply op (one pixel per call: op(r, g, b, o0, o1, o2) returns an int id)
// to the 4 pixels of sub-block s owned by this thread.
template <int THREADS, class Op>
__device__ __forceinline__ void apply4(const uint4 *sbuf, int s, const Op &op, float (&v)[3][4], int (&sl)[4])
{
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(sbuf) + s * 3 * THREADS + 3 * threadIdx.x;
    const uint32_t w0 = sw[0], w1 = sw[1], w2 = sw[2];
    // bytes: w0 = r0 g0 b0 r1 | w1 = g1 b1 r2 g2 | w2 = b2 r3 g3 b3
    sl[0] = op(w0 & 255u, (w0 >> 8) & 255u, (w0 >> 16) & 255u, v[0][0], v[1][0], v[2][0]);
    sl[1] = op(w0 >> 24, w1 & 255u, (w1 >> 8) & 255u, v[0][1], v[1][1], v[2][1]);
    sl[2] = op((w1 >> 16) & 255u, w1 >> 24, w2 & 255u, v[0][2], v[1][2], v[2][2]);
    sl[3] = op((w2 >> 8) & 255u, (w2 >> 16) & 255u, w2 >> 24, v[0][3], v[1][3], v[2][3]);
}

// Full, aligned tile: sbuf holds its input; outputs start at o* (+ sel).
template <int THREADS, int SUBS, typename OutT, bool SEL, class Op>
__device__ __forceinline__ void compute_full(const uint4 *sbuf, const Op &op, OutT *o0, OutT *o1, OutT *o2,
                                             int32_t *sel)
{
    // an explicit count: a bare "#pragma unroll" here compiles to more
    // registers (63 vs 48 for MACT CIELAB) and spills in the LUT kernels
#pragma unroll(SUBS)
    for (int s = 0; s < SUBS; ++s) {
        float v[3][4];
        int sl[4];
        apply4<THREADS>(sbuf, s, op, v, sl);
        const int p = s * TileShape<THREADS>::sub + kPxPerThread * threadIdx.x;
        store4(o0 + p, v[0][0], v[0][1], v[0][2], v[0][3]);
        store4(o1 + p, v[1][0], v[1][1], v[1][2], v[1][3]);
        store4(o2 + p, v[2][0], v[2][1], v[2][2], v[2][3]);
        if (SEL) __stcs(reinterpret_cast<int4 *>(sel + p), make_int4(sl[0], sl[1], sl[2], sl[3]));
    }
}

// Full tile with 16-byte aligned input but output planes aligned only to
// their element size (adjacent planes of W*H elements, W*H not a multiple of
// 4): each warp passes its 128 values per plane through 512 bytes of shared
// scratch, so that every warp store writes 32 consecutive elements instead of
// four strided scalar stores per thread.  scr: THREADS*4 floats.
template <int THREADS, int SUBS, typename OutT, class Op>
__device__ __forceinline__ void compute_full_shifted(const uint4 *sbuf, float *scr, const Op &op, OutT *o0,
                                                     OutT *o1, OutT *o2)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *w = scr + 128 * warp;
#pragma unroll(SUBS)
    for (int s = 0; s < SUBS; ++s) {
        float v[3][4];
        int sl[4];
        apply4<THREADS>(sbuf, s, op, v, sl);
        // this thread holds pixels wb + 4*lane + j of the warp's 128 (j < 4)
        const int wb = s * TileShape<THREADS>::sub + 128 * warp;
        OutT *dst[3] = {o0 + wb, o1 + wb, o2 + wb};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            __syncwarp();
            *reinterpret_cast<float4 *>(w + 4 * lane) = make_float4(v[c][0], v[c][1], v[c][2], v[c][3]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k) store1(dst[c] + lane + 32 * k, w[lane + 32 * k]);
        }
    }
}

// Guarded tile of cnt <= px pixels at any alignment.  Ends with a barrier
// already passed after the staging; the caller synchronises before reusing
// sbuf.
// Stage nb input bytes into shared memory: 16-byte loads for the aligned
// bulk when in is 16-byte aligned, single bytes otherwise and for the rest.
template <int THREADS>
__device__ __forceinline__ void stage_bytes(uint4 *sbuf, const uint8_t *in, int nb)
{
    uint8_t *sb = reinterpret_cast<uint8_t *>(sbuf);
    int i0 = 0;
    if ((reinterpret_cast<uintptr_t>(in) & 15) == 0) {
        const int nv = nb >> 4;
        const uint4 *p = reinterpret_cast<const uint4 *>(in);
        for (int i = threadIdx.x; i < nv; i += THREADS) sbuf[i] = __ldcs(p + i);
        i0 = nv << 4;
    }
    for (int i = i0 + threadIdx.x; i < nb; i += THREADS) sb[i] = in[i];
}

// The compute half of the guarded path: sbuf already holds the tile's
// 3*cnt input bytes (staged and synchronised by the caller).
template <int THREADS, int SUBS, typename OutT, bool SEL, class Op>
__device__ __forceinline__ void compute_guarded_staged(const uint4 *sbuf, int cnt, const Op &op, OutT *o0,
                                                       OutT *o1, OutT *o2, int32_t *sel)
{
    for (int s = 0; s < SUBS; ++s) {
        const int p = s * TileShape<THREADS>::sub + kPxPerThread * threadIdx.x;
        if (p >= cnt) break;
        float v[3][4];
        int sl[4];
        apply4<THREADS>(sbuf, s, op, v, sl);
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            if (p + j < cnt) {
                store1(o0 + p + j, v[0][j]);
                store1(o1 + p + j, v[1][j]);
                store1(o2 + p + j, v[2][j]);
                if (SEL) sel[p + j] = sl[j];
            }
        }
    }
}

template <int THREADS, int SUBS, typename OutT, bool SEL, class Op>
__device__ __forceinline__ void compute_guarded(uint4 *sbuf, const uint8_t *in, int cnt, const Op &op, OutT *o0,
                                                OutT *o1, OutT *o2, int32_t *sel)
{
    stage_bytes<THREADS>(sbuf, in, 3 * cnt);
    __syncthreads();
    compute_guarded_staged<THREADS, SUBS, OutT, SEL>(sbuf, cnt, op, o0, o1, o2, sel);
}

// Partial tile (cnt < px pixels) with element-aligned outputs: staged like
// the guarded path, stored through the warp transpose of the shifted path
// with a bound on each element.  Whole warps stay together (the bound on a
// warp's first pixel is warp-uniform); pixels past cnt are computed from
// stale shared bytes and not stored.
template <int THREADS, int SUBS, typename OutT, class Op>
__device__ __forceinline__ void compute_tail_shifted(uint4 *sbuf, float *scr, const uint8_t *in, int cnt,
                                                     const Op &op, OutT *o0, OutT *o1, OutT *o2)
{
    stage_bytes<THREADS>(sbuf, in, 3 * cnt);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float *w = scr + 128 * warp;
    for (int s = 0; s < SUBS; ++s) {
        const int wb = s * TileShape<THREADS>::sub + 128 * warp;
        if (wb >= cnt) break;
        float v[3][4];
        int sl[4];
        apply4<THREADS>(sbuf, s, op, v, sl);
        OutT *dst[3] = {o0 + wb, o1 + wb, o2 + wb};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            __syncwarp();
            *reinterpret_cast<float4 *>(w + 4 * lane) = make_float4(v[c][0], v[c][1], v[c][2], v[c][3]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = lane + 32 * k;
                if (wb + i < cnt) store1(dst[c] + i, w[i]);
            }
        }
    }
}

// Tile t of image im (any geometry): the vector path when full and aligned;
// the shifted path when full with aligned input and element-aligned output
// (scr given: THREADS*4 floats of shared scratch); else the guarded path.
// The caller synchronises before reusing sbuf.
template <int THREADS, typename OutT, bool SEL, class Op, int SUBS = kSubBlocks>
__device__ __forceinline__ void process_tile(const ImageDesc &im, int64_t t, const Op &op, uint4 *sbuf,
                                             int32_t *sel, float *scr = nullptr)
{
    constexpr int P = TileShape<THREADS, SUBS>::px;
    const uint32_t tpr = (uint32_t)im.tiles_per_row;     // < 2^31 (checked on the host)
    const uint32_t tt = (uint32_t)t;
    const uint32_t row = tt / tpr;
    const int64_t x0 = (int64_t)(tt - row * tpr) * P;
    const int64_t rem_px = im.width - x0;
    const int cnt = rem_px < P ? (int)rem_px : P;
    const uint8_t *in = im.rgb + (int64_t)row * im.pitch + 3 * x0;
    const int64_t off = (int64_t)row * im.opitch + x0;
    OutT *o0 = reinterpret_cast<OutT *>(im.out[0]) + off;
    OutT *o1 = reinterpret_cast<OutT *>(im.out[1]) + off;
    OutT *o2 = reinterpret_cast<OutT *>(im.out[2]) + off;
    int32_t *sl = SEL ? sel + off : nullptr;
    constexpr uintptr_t omask = sizeof(OutT) == 4 ? 15 : 7;
    uintptr_t oa = reinterpret_cast<uintptr_t>(o0) | reinterpret_cast<uintptr_t>(o1) |
                   reinterpret_cast<uintptr_t>(o2);
    if (SEL) oa |= reinterpret_cast<uintptr_t>(sl);
    const bool full_in = cnt == P && ((reinterpret_cast<uintptr_t>(in) & 15) == 0);
    const bool shifted = !SEL && scr != nullptr && (oa & (sizeof(OutT) - 1)) == 0;
    if (full_in && ((oa & omask) == 0 || shifted)) {
        uint4 v[TileShape<THREADS, SUBS>::vpt];
        load_tile<THREADS, SUBS>(v, in);
        stage_tile<THREADS, SUBS>(sbuf, v);
        __syncthreads();
        if ((oa & omask) == 0) compute_full<THREADS, SUBS, OutT, SEL>(sbuf, op, o0, o1, o2, sl);
        else compute_full_shifted<THREADS, SUBS, OutT>(sbuf, scr, op, o0, o1, o2);
    } else if (shifted) {
        compute_tail_shifted<THREADS, SUBS, OutT>(sbuf, scr, in, cnt, op, o0, o1, o2);
    } else {
        compute_guarded<THREADS, SUBS, OutT, SEL>(sbuf, in, cnt, op, o0, o1, o2, sl);
    }
}

// Whole image, persistent CTA loop.  Streamable images run the prefetching
// vector loop over their full tiles and hand the partial last tile to the
// guarded path; everything else walks tiles through process_tile.
template <int THREADS, typename OutT, bool SEL, class Op, int SUBS = kSubBlocks>
__device__ __forceinline__ void run_image(const ImageDesc &im, int64_t ntiles, const Op &op, uint4 *sbuf,
                                          int32_t *sel, float *scr = nullptr)
{
    constexpr int P = TileShape<THREADS, SUBS>::px;
    if (streamable<OutT, SEL>(im, sel)) {
        const int64_t nfull = im.width / P;
        OutT *b0 = reinterpret_cast<OutT *>(im.out[0]);
        OutT *b1 = reinterpret_cast<OutT *>(im.out[1]);
        OutT *b2 = reinterpret_cast<OutT *>(im.out[2]);
        int64_t t = blockIdx.x;
        uint4 v[TileShape<THREADS, SUBS>::vpt];
        if (t < nfull) load_tile<THREADS, SUBS>(v, im.rgb + 3 * P * t);
        for (; t < nfull; t += gridDim.x) {
            __syncthreads();                 // previous tile's readers are done
            stage_tile<THREADS, SUBS>(sbuf, v);
            __syncthreads();
            const int64_t tn = t + gridDim.x;
            if (tn < nfull) load_tile<THREADS, SUBS>(v, im.rgb + 3 * P * tn);   // in flight during compute
            const int64_t o = P * t;
            compute_full<THREADS, SUBS, OutT, SEL>(sbuf, op, b0 + o, b1 + o, b2 + o, SEL ? sel + o : nullptr);
        }
        if (nfull < ntiles && blockIdx.x == (unsigned)(nfull % gridDim.x)) {
            __syncthreads();
            const int64_t o = P * nfull;
            if (!SEL && scr != nullptr)
                compute_tail_shifted<THREADS, SUBS, OutT>(sbuf, scr, im.rgb + 3 * o, (int)(im.width - o), op, b0 + o,
                                                          b1 + o, b2 + o);
            else
                compute_guarded<THREADS, SUBS, OutT, SEL>(sbuf, im.rgb + 3 * o, (int)(im.width - o), op, b0 + o,
                                                          b1 + o, b2 + o, SEL ? sel + o : nullptr);
        }
        return;
    }
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        process_tile<THREADS, OutT, SEL, Op, SUBS>(im, t, op, sbuf, sel, scr);
    }
}

}  // namespace mact
