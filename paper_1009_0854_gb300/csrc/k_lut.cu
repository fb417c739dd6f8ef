// k_lut.cu -- 3D-LUT packing and the trilinear / prism / pyramidal /
// tetrahedral interpolators (Section "Comparison with 3D Lookup Table
// Interpolation Methods"), on the streaming tile engine.
//
// Extraction is bit-identical to an integer implementation: along each axis
// s = v (n-1), idx = s div 255, rem = s mod 255, and the code v = 255 uses
// idx = n-2, rem = 255; the fraction is rem * fl(1/255), computed per pixel
// in registers.  Simplex choices compare
// fractions, which order exactly as the integer remainders do
// (rem -> rem * fl(1/255) is strictly increasing on 0..255 in FP32).  The
// interpolation formulas run on packed FP32 pairs (R/G channels) plus a
// scalar (B channel), rounded exactly as scalar FMA chains.
//
// This file holds the packing kernels and the dispatch on the method; the
// interpolation kernels are in k_lut_interp.cuh, compiled once per method
// (k_lut_inst.cu) so the methods build in parallel.
//
// LUT placement: for n <= 17 every CTA stages the whole LUT in shared memory
// as float4 nodes (17^3 x 16 B = 78.6 KB), so a node is one 16-byte shared
// load.  Larger LUTs (33^3: 575 KB as float4) do not fit and are read as
// float4 nodes from global memory through L1 (L2 resident), trilinear as
// 4 B-edge records (xy and z pairs) instead of 8 nodes: either a copy the
// caller packed once (mact_lut_pack), or one repacked into handle scratch on
// every call.  (Staging per 4096-pixel tile only the box of nodes
// the tile touches was measured 3-23% slower on the cube, and 5x slower on
// noise, where every tile falls back to global memory: not kept.)
#include <atomic>

#include "internal.h"

namespace mact {

// --------------------------------------------------------------- packing

__global__ void k_lut_build(int n, float *__restrict__ lut, mact_rgb_def d)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= n * n * n) return;
    const int k = node % n, j = (node / n) % n, i = node / (n * n);
    const int idx[3] = {i, j, k};
    double lin[3];
    for (int c = 0; c < 3; ++c) {
        double kp = (double)idx[c] / (double)(n - 1);
        lin[c] = kp < d.gamma_threshold ? kp / d.gamma_slope
                                        : pow((kp + d.gamma_offset) / (1.0 + d.gamma_offset), d.gamma_exponent);
    }
    double f[3];
    for (int c = 0; c < 3; ++c) {
        double t = (d.rgb_to_xyz[3 * c] * lin[0] + d.rgb_to_xyz[3 * c + 1] * lin[1] +
                    d.rgb_to_xyz[3 * c + 2] * lin[2]) / d.white[c];
        f[c] = t > 0.008856 ? cbrt(t) : 7.787 * t + 16.0 / 116.0;
    }
    lut[3 * node + 0] = (float)(116.0 * f[1] - 16.0);
    lut[3 * node + 1] = (float)(500.0 * (f[0] - f[1]));
    lut[3 * node + 2] = (float)(200.0 * (f[1] - f[2]));
}

cudaError_t launch_lut_build(const mact_ctx &h, int n, float *d_lut, cudaStream_t s)
{
    const int nodes = n * n * n;
    k_lut_build<<<(nodes + 255) / 256, 256, 0, s>>>(n, d_lut, h.cfg.rgb);
    return cudaGetLastError();
}

// packed float3 nodes -> float4 nodes (the fourth lane unused)
__global__ void k_lut_pack4(const float *__restrict__ lut, int nodes, float4 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nodes) out[i] = make_float4(lut[3 * i], lut[3 * i + 1], lut[3 * i + 2], 0.0f);
}

// Edge records of the packed layout, from its float4 nodes: for node i and
// an axis (B: next node i + 1; R: next node i + n^2), xy[i] = (x_i, y_i, x_j,
// y_j) and z[i] = (z_i, z_j) with j the next node along the axis -- the two
// ends of the edge that starts at node i (a node at the end of its row along
// the axis repeats itself; no cell starts there).  In a LUT too large for
// shared memory, trilinear interpolation reads its 8 nodes as 4 B edges and
// prism its 6 as 3 R edges; the pyramid reads single nodes from the dense xy
// (float2) and z (float) planes written here too; tetrahedral reads the
// 16-byte nodes.
__global__ void k_lut_edges(const float4 *__restrict__ nodes4, int n, float4 *__restrict__ bxy,
                            float2 *__restrict__ bz, float4 *__restrict__ rxy, float2 *__restrict__ rz,
                            float2 *__restrict__ pxy, float *__restrict__ pz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nn = n * n;
    if (i >= nn * n) return;
    const float4 a = nodes4[i];
    const float4 b = (i % n) != n - 1 ? nodes4[i + 1] : a;
    const float4 r = i / nn != n - 1 ? nodes4[i + nn] : a;
    bxy[i] = make_float4(a.x, a.y, b.x, b.y);
    bz[i] = make_float2(a.z, b.z);
    rxy[i] = make_float4(a.x, a.y, r.x, r.y);
    rz[i] = make_float2(a.z, r.z);
    pxy[i] = make_float2(a.x, a.y);
    pz[i] = a.z;
}

// "Caching" layout (the paper's second implementation of each LUT method:
// the differences between neighbouring lattice nodes are precomputed and
// stored with each node): one 128-byte record per cell (i, j, k), i.e. per
// lower corner, holding c000 and the seven differences c_xyz - c000 as
// float4, slot x*4 + y*2 + z (x = R, y = G, z = B offset).  A pixel reads its
// whole neighbourhood from one cache line.
__global__ void k_lut_cache_build(const float *__restrict__ lut, int n, float4 *__restrict__ cache)
{
    const int m = n - 1;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= m * m * m) return;
    const int k = cell % m, j = (cell / m) % m, i = cell / (m * m);
    const int64_t b0 = ((int64_t)(i * n + j) * n + k) * 3;
    float4 *rec = cache + (int64_t)cell * 8;
    const float c0x = lut[b0], c0y = lut[b0 + 1], c0z = lut[b0 + 2];
    rec[0] = make_float4(c0x, c0y, c0z, 0.0f);
    for (int slot = 1; slot < 8; ++slot) {
        const int x = slot >> 2, y = (slot >> 1) & 1, z = slot & 1;
        const int64_t o = ((int64_t)((i + x) * n + (j + y)) * n + (k + z)) * 3;
        rec[slot] = make_float4(lut[o] - c0x, lut[o + 1] - c0y, lut[o + 2] - c0z, 0.0f);
    }
}

cudaError_t launch_lut_cache_build(const float *d_lut, int n, float4 *d_cache, cudaStream_t s)
{
    const int cells = (n - 1) * (n - 1) * (n - 1);
    k_lut_cache_build<<<(cells + 255) / 256, 256, 0, s>>>(d_lut, n, d_cache);
    return cudaGetLastError();
}

cudaError_t launch_lut_interp(const mact_ctx &h, int method, const float *d_lut, const float4 *d_lut4, int n,
                              const uint8_t *d_rgb, int64_t npix, float *const out[3], int32_t *d_sel,
                              cudaStream_t s)
{
#define MACT_LUT_CASE(SEL)                                                                                     \
    switch (method) {                                                                                           \
    case MACT_TRILINEAR: return lut_interp_method<MACT_TRILINEAR, SEL>(h, d_lut, d_lut4, n, d_rgb, npix, out, d_sel, s); \
    case MACT_PRISM: return lut_interp_method<MACT_PRISM, SEL>(h, d_lut, d_lut4, n, d_rgb, npix, out, d_sel, s);     \
    case MACT_PYRAMID: return lut_interp_method<MACT_PYRAMID, SEL>(h, d_lut, d_lut4, n, d_rgb, npix, out, d_sel, s); \
    default: return lut_interp_method<MACT_TETRA, SEL>(h, d_lut, d_lut4, n, d_rgb, npix, out, d_sel, s);            \
    }
    if (d_sel) MACT_LUT_CASE(true)
    MACT_LUT_CASE(false)
#undef MACT_LUT_CASE
}

bool lut_needs_pack(int n) { return n > kLutSmemMaxN; }

cudaError_t launch_lut_interp_cached(const mact_ctx &h, int method, const float4 *d_cache, int n,
                                     const uint8_t *d_rgb, int64_t npix, float *const out[3], int32_t *d_sel,
                                     cudaStream_t s)
{
    if (d_sel) {
        switch (method) {
        case MACT_TRILINEAR: return lut_cached_method<MACT_TRILINEAR, true>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
        case MACT_PRISM: return lut_cached_method<MACT_PRISM, true>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
        case MACT_PYRAMID: return lut_cached_method<MACT_PYRAMID, true>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
        default: return lut_cached_method<MACT_TETRA, true>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
        }
    }
    switch (method) {
    case MACT_TRILINEAR: return lut_cached_method<MACT_TRILINEAR, false>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
    case MACT_PRISM: return lut_cached_method<MACT_PRISM, false>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
    case MACT_PYRAMID: return lut_cached_method<MACT_PYRAMID, false>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
    default: return lut_cached_method<MACT_TETRA, false>(h, d_cache, n, d_rgb, npix, out, d_sel, s);
    }
}

cudaError_t launch_lut_pack4(const float *d_lut, int n, float4 *d_lut4, cudaStream_t s)
{
    const int nodes = n * n * n;
    k_lut_pack4<<<(nodes + 255) / 256, 256, 0, s>>>(d_lut, nodes, d_lut4);
    return cudaGetLastError();
}

cudaError_t launch_lut_pack(const float *d_lut, int n, float *d_packed, cudaStream_t s)
{
    const int nodes = n * n * n;
    float4 *n4 = reinterpret_cast<float4 *>(d_packed);
    cudaError_t e = launch_lut_pack4(d_lut, n, n4, s);
    if (e != cudaSuccess) return e;
    const PackedLut pk = packed_lut(n4, n);   // the same offsets the kernels read
    k_lut_edges<<<(nodes + 255) / 256, 256, 0, s>>>(n4, n, const_cast<float4 *>(pk.bxy), const_cast<float2 *>(pk.bz),
                                                    const_cast<float4 *>(pk.rxy), const_cast<float2 *>(pk.rz),
                                                    const_cast<float2 *>(pk.pxy), const_cast<float *>(pk.pz));
    return cudaGetLastError();
}


}  // namespace mact
