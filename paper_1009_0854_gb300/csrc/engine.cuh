// engine.cuh -- the streaming tile engine shared by the transform and LUT
// kernels: interleaved uint8 RGB in, three planes (and optionally a
// per-pixel int32) out, THREADS x 4 pixels per CTA tile.
//
// Data path per tile (HBM-bound: 3 bytes read and 12 (FP32) or 6 (FP16)
// bytes written per pixel, nothing reused):
//   1. 3/4 of the threads each load one 16-byte vector of the tile's
//      12*THREADS input bytes (coalesced, streaming cache hint) into shared
//      memory;
//   2. every thread de-interleaves 4 consecutive pixels from three 32-bit
//      shared-memory words (stride 3 words across a warp: conflict-free) and
//      applies the operator;
//   3. every thread writes its 4 results per plane as one 16-byte (FP32) or
//      8-byte (FP16) streaming store, so a warp writes 512 contiguous bytes.
// Short tiles (image tail) and misaligned ones (pitched rows, odd pointers)
// take a byte-wise load and per-pixel stores instead.
#pragma once

#include "common.cuh"

namespace mact {

template <int THREADS>
struct TileShape {
    static constexpr int px = THREADS * kPxPerThread;
    static constexpr int vecs = px * 3 / 16;
};

template <int THREADS>
__host__ __device__ inline int64_t tiles_of_t(const ImageDesc &im)
{
    constexpr int P = TileShape<THREADS>::px;
    if (im.width <= 0 || im.height <= 0) return 0;
    return im.height * ((im.width + P - 1) / P);
}

// Process tile t of image im with operator op.  sbuf holds
// TileShape<THREADS>::vecs uint4.  If SEL, op's integer result is written to
// sel (same geometry as the output planes).  Ends with sbuf still in use by
// other threads: the caller must __syncthreads() before reusing it.
template <int THREADS, typename OutT, bool SEL, class Op>
__device__ __forceinline__ void process_tile(const ImageDesc &im, int64_t t, const Op &op, uint4 *sbuf,
                                             int32_t *sel)
{
    constexpr int P = TileShape<THREADS>::px;
    constexpr int V = TileShape<THREADS>::vecs;
    const int tid = threadIdx.x;
    const int64_t row = t / im.tiles_per_row;
    const int64_t x0 = (t - row * im.tiles_per_row) * P;
    const int64_t rem_px = im.width - x0;
    const int cnt = rem_px < P ? (int)rem_px : P;
    const uint8_t *in = im.rgb + row * im.pitch + 3 * x0;
    const int64_t off = row * im.opitch + x0;
    OutT *o0 = reinterpret_cast<OutT *>(im.out[0]) + off;
    OutT *o1 = reinterpret_cast<OutT *>(im.out[1]) + off;
    OutT *o2 = reinterpret_cast<OutT *>(im.out[2]) + off;
    constexpr uintptr_t omask = sizeof(OutT) == 4 ? 15 : 7;
    uintptr_t oa = reinterpret_cast<uintptr_t>(o0) | reinterpret_cast<uintptr_t>(o1) |
                   reinterpret_cast<uintptr_t>(o2);
    if (SEL) oa |= reinterpret_cast<uintptr_t>(sel + off);
    const bool fast = cnt == P && ((reinterpret_cast<uintptr_t>(in) & 15) == 0) && ((oa & omask) == 0);
    if (fast) {
        if (tid < V) sbuf[tid] = __ldcs(reinterpret_cast<const uint4 *>(in) + tid);
    } else {
        uint8_t *sb = reinterpret_cast<uint8_t *>(sbuf);
        for (int i = tid; i < 3 * cnt; i += THREADS) sb[i] = in[i];
    }
    __syncthreads();

    const uint32_t *sw = reinterpret_cast<const uint32_t *>(sbuf) + 3 * tid;
    const uint32_t w0 = sw[0], w1 = sw[1], w2 = sw[2];
    // bytes: w0 = r0 g0 b0 r1 | w1 = g1 b1 r2 g2 | w2 = b2 r3 g3 b3
    float v[3][4];
    int s[4];
    s[0] = op(w0 & 255u, (w0 >> 8) & 255u, (w0 >> 16) & 255u, v[0][0], v[1][0], v[2][0]);
    s[1] = op(w0 >> 24, w1 & 255u, (w1 >> 8) & 255u, v[0][1], v[1][1], v[2][1]);
    s[2] = op((w1 >> 16) & 255u, w1 >> 24, w2 & 255u, v[0][2], v[1][2], v[2][2]);
    s[3] = op((w2 >> 8) & 255u, (w2 >> 16) & 255u, w2 >> 24, v[0][3], v[1][3], v[2][3]);

    const int p0 = kPxPerThread * tid;
    if (fast) {
        store4(o0 + p0, v[0][0], v[0][1], v[0][2], v[0][3]);
        store4(o1 + p0, v[1][0], v[1][1], v[1][2], v[1][3]);
        store4(o2 + p0, v[2][0], v[2][1], v[2][2], v[2][3]);
        if (SEL) __stcs(reinterpret_cast<int4 *>(sel + off + p0), make_int4(s[0], s[1], s[2], s[3]));
    } else {
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            if (p0 + j < cnt) {
                store1(o0 + p0 + j, v[0][j]);
                store1(o1 + p0 + j, v[1][j]);
                store1(o2 + p0 + j, v[2][j]);
                if (SEL) sel[off + p0 + j] = s[j];
            }
        }
    }
}

}  // namespace mact
