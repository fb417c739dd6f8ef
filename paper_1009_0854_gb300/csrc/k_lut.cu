// k_lut.cu -- 3D-LUT packing and the trilinear / prism / pyramidal /
// tetrahedral interpolators (Section "Comparison with 3D Lookup Table
// Interpolation Methods"), on the streaming tile engine.
//
// Extraction is bit-identical to an integer implementation: along each axis
// s = v (n-1), idx = s div 255, rem = s mod 255, and the code v = 255 uses
// idx = n-2, rem = 255; the fraction is rem * fl(1/255).  It is computed per
// pixel in integer arithmetic (no extra shared loads: the interpolation's
// gathers already keep the shared/L1 data pipe busy).  Simplex choices
// compare fractions, which order exactly as the integer remainders do
// (rem -> rem * fl(1/255) is strictly increasing on 0..255 in FP32).
//
// LUT placement: for n <= 17 every CTA stages the whole LUT in shared memory
// as float4 nodes (17^3 x 16 B = 78.6 KB), so a node is one 16-byte shared
// load.  Larger LUTs (33^3: 575 KB as float4) are first repacked into float4
// nodes in a scratch buffer of the handle (one small kernel per call) and
// read from global memory (L1/L2 resident).  For n = 9, 17, 33 the node
// strides are compile-time constants, so node addresses are immediate
// offsets from the cell's base.
#include "engine.cuh"
#include <atomic>

#include "internal.h"

namespace mact {

constexpr int kLutSmemMaxN = 17;
// Threads per CTA of the shared-memory LUT kernels (two CTAs per SM, each
// with its own staged copy of the LUT).  The register cap this leaves (128
// at 256 threads, 85 at 384) keeps the interpolators from spilling; measured
// on the 2^24 cube, 256 threads suit trilinear, prism and pyramid and 384 the
// tetrahedral method (512 threads, 64 registers, spilled: 11-21% slower).
template <int METHOD>
struct SmemThreads {
    static constexpr int value = METHOD == MACT_TETRA ? 384 : 256;
};

// Launch shape of the global-memory LUT kernels (about 24 resident warps per
// SM, 80 registers): trilinear 256 threads x 3 CTAs; the other methods
// 128 x 6, which measured 2-6% faster for them and 4% slower for trilinear.
template <int METHOD>
struct GlobalShape {
    static constexpr int threads = METHOD == MACT_TRILINEAR ? 256 : 128;
    static constexpr int ctas = METHOD == MACT_TRILINEAR ? 3 : 6;
};

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

// ---------------------------------------------------------- interpolation

__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, 0.f); }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f); }
__device__ __forceinline__ float4 f4fma(float4 a, float s, float4 c)
{
    return make_float4(fmaf(a.x, s, c.x), fmaf(a.y, s, c.y), fmaf(a.z, s, c.z), 0.f);
}

// Node fetch: shared memory, or the read-only global path.  With NARROW a
// node's padding float is not read (an 8-byte and a 4-byte load instead of
// one 16-byte load): fewer live registers for the same values.  Measured on
// GB300 it pays only for the pyramid (5 nodes, the most register-hungry
// selection); the other methods keep the single 16-byte load.
template <bool SMEM, bool NARROW = false>
__device__ __forceinline__ float4 node(const float4 *p)
{
    if constexpr (!NARROW) {
        if constexpr (SMEM) return *p;
        else return __ldg(p);
    } else {
        const float *f = reinterpret_cast<const float *>(p);
        float2 xy;
        float z;
        if constexpr (SMEM) {
            xy = *reinterpret_cast<const float2 *>(f);
            z = f[2];
        } else {
            xy = __ldg(reinterpret_cast<const float2 *>(f));
            z = __ldg(f + 2);
        }
        return make_float4(xy.x, xy.y, z, 0.f);
    }
}

// Node strides: compile-time for N > 0, runtime otherwise.
template <int N>
struct Strides {
    int n;
    __device__ __forceinline__ int r() const { return N > 0 ? N * N : n * n; }
    __device__ __forceinline__ int g() const { return N > 0 ? N : n; }
};

// Nodes each method reads from its cell.
template <int METHOD>
struct NodeCount {
    static constexpr int K = METHOD == MACT_TRILINEAR ? 8 : METHOD == MACT_PRISM ? 6 : METHOD == MACT_PYRAMID ? 5 : 4;
};

// Extraction result of one pixel: the cell, the simplex, the offsets of the
// nodes to read (relative to the cell's lower corner) and the three weights
// the interpolation formula uses.
template <int METHOD>
struct Sel {
    int base;     // lower-corner node index
    int rec;      // cell record index (caching layout)
    int simplex;
    int off[NodeCount<METHOD>::K];
    float w0, w1, w2;
};

// CACHED: nodes come from the per-cell records of the caching layout (base
// is still the lower-corner node index, for the selection id; rec is the
// cell's record index; node offsets become record slots and the value is
// c000 + the interpolation of the differences).
template <int METHOD, int N, bool SMEM, bool CACHED = false>
struct OpLut {
    static constexpr int K = NodeCount<METHOD>::K;
    const float4 *lut;        // shared or global float4 nodes, or cell records
    Strides<N> st;

    __device__ __forceinline__ static void locate(uint32_t v, int n, int &idx, float &f)
    {
        const int s = (int)v * (n - 1);
        idx = s / 255;
        int rem = s - 255 * idx;
        if (idx == n - 1) { idx = n - 2; rem = 255; }
        // rem * fl(1/255): strictly increasing in rem, so comparing fractions
        // orders cells exactly as the integer remainders do
        f = (float)rem * (1.0f / 255.0f);
    }

    __device__ __forceinline__ Sel<METHOD> select(uint32_t r, uint32_t g, uint32_t b) const
    {
        // node strides, or record slot strides in the caching layout
        const int sR = CACHED ? 4 : st.r(), sG = CACHED ? 2 : st.g(), sB = 1;
        Sel<METHOD> q;
        float fr, fg, fb;
        const int n = st.g();
        int ir, ig, ib;
        locate(r, n, ir, fr);
        locate(g, n, ig, fg);
        locate(b, n, ib, fb);
        q.base = (ir * n + ig) * n + ib;
        if (CACHED) q.rec = (ir * (n - 1) + ig) * (n - 1) + ib;
        if (METHOD == MACT_TRILINEAR) {
            const int o[8] = {0, sB, sG, sG + sB, sR, sR + sB, sR + sG, sR + sG + sB};
#pragma unroll
            for (int k = 0; k < 8; ++k) q.off[k] = o[k];
            q.simplex = 0;
            q.w0 = fb; q.w1 = fg; q.w2 = fr;
        } else if (METHOD == MACT_PRISM) {
            // prism axis R; triangle in the G-B face chosen by rem_G >= rem_B
            const bool lo = fg >= fb;
            const int oe = lo ? sG : sB;   // c010 or c001
            const int o[6] = {0, sR, sG + sB, sR + sG + sB, oe, sR + oe};
#pragma unroll
            for (int k = 0; k < 6; ++k) q.off[k] = o[k];
            q.simplex = lo ? 0 : 1;
            q.w0 = lo ? fg : fb; q.w1 = lo ? fb : fg; q.w2 = fr;
        } else if (METHOD == MACT_PYRAMID) {
            // apex c111; base on the face of the smallest fraction (B, then G, then R)
            int oX, oY;
            if (fb <= fr && fb <= fg) { oX = sR; oY = sG; q.w0 = fr; q.w1 = fg; q.w2 = fb; q.simplex = 0; }
            else if (fg <= fr && fg <= fb) { oX = sR; oY = sB; q.w0 = fr; q.w1 = fb; q.w2 = fg; q.simplex = 1; }
            else { oX = sG; oY = sB; q.w0 = fg; q.w1 = fb; q.w2 = fr; q.simplex = 2; }
            const int o[5] = {0, sR + sG + sB, oX, oY, oX + oY};
#pragma unroll
            for (int k = 0; k < 5; ++k) q.off[k] = o[k];
        } else {
            // tetrahedral: path from c000 along the axes in decreasing fraction
            int o1, o2;
            if (fr >= fg && fg >= fb)      { o1 = sR; o2 = sR + sG; q.w0 = fr; q.w1 = fg; q.w2 = fb; q.simplex = 0; }
            else if (fr >= fb && fb > fg)  { o1 = sR; o2 = sR + sB; q.w0 = fr; q.w1 = fb; q.w2 = fg; q.simplex = 1; }
            else if (fb > fr && fr >= fg)  { o1 = sB; o2 = sR + sB; q.w0 = fb; q.w1 = fr; q.w2 = fg; q.simplex = 2; }
            else if (fg > fr && fr >= fb)  { o1 = sG; o2 = sR + sG; q.w0 = fg; q.w1 = fr; q.w2 = fb; q.simplex = 3; }
            else if (fg >= fb && fb > fr)  { o1 = sG; o2 = sG + sB; q.w0 = fg; q.w1 = fb; q.w2 = fr; q.simplex = 4; }
            else                           { o1 = sB; o2 = sG + sB; q.w0 = fb; q.w1 = fg; q.w2 = fr; q.simplex = 5; }
            const int o[4] = {0, o1, o2, sR + sG + sB};
#pragma unroll
            for (int k = 0; k < 4; ++k) q.off[k] = o[k];
        }
        return q;
    }

    __device__ __forceinline__ void load(const Sel<METHOD> &q, float4 (&nd)[K]) const
    {
        const float4 *cb = CACHED ? lut + (int64_t)q.rec * 8 : lut + q.base;
#pragma unroll
        for (int k = 0; k < K; ++k) nd[k] = node<SMEM, METHOD == MACT_PYRAMID>(cb + q.off[k]);
    }

    // value from the loaded nodes: directly, or c000 + interpolated differences
    __device__ __forceinline__ static float4 value(const float4 (&nd)[K], const Sel<METHOD> &q)
    {
        if (!CACHED) return interp(nd, q);
        float4 d[K];
        d[0] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 1; k < K; ++k) d[k] = nd[k];
        return f4add(nd[0], interp(d, q));
    }

    __device__ __forceinline__ static float4 interp(const float4 (&nd)[K], const Sel<METHOD> &q)
    {
        if (METHOD == MACT_TRILINEAR) {
            // repeated linear interpolation along B, then G, then R
            // nd: c000 c001 c010 c011 c100 c101 c110 c111
            const float4 c00 = f4fma(f4sub(nd[1], nd[0]), q.w0, nd[0]);
            const float4 c01 = f4fma(f4sub(nd[3], nd[2]), q.w0, nd[2]);
            const float4 c10 = f4fma(f4sub(nd[5], nd[4]), q.w0, nd[4]);
            const float4 c11 = f4fma(f4sub(nd[7], nd[6]), q.w0, nd[6]);
            const float4 c0 = f4fma(f4sub(c01, c00), q.w1, c00);
            const float4 c1 = f4fma(f4sub(c11, c10), q.w1, c10);
            return f4fma(f4sub(c1, c0), q.w2, c0);
        } else if (METHOD == MACT_PRISM) {
            // nd: c000 c100 c011 c111 ce0 ce1; triangle at R = 0 and R = 1, then linear in R
            const float4 t0 = f4fma(f4sub(nd[2], nd[4]), q.w1, f4fma(f4sub(nd[4], nd[0]), q.w0, nd[0]));
            const float4 t1 = f4fma(f4sub(nd[3], nd[5]), q.w1, f4fma(f4sub(nd[5], nd[1]), q.w0, nd[1]));
            return f4fma(f4sub(t1, t0), q.w2, t0);
        } else if (METHOD == MACT_PYRAMID) {
            // nd: c000 c111 cX cY cA;
            // c000 + (c111-cA) fZ + (cX-c000) fX + (cY-c000) fY + (cA-cX-cY+c000) fX fY
            const float4 cross = f4add(f4sub(f4sub(nd[4], nd[2]), nd[3]), nd[0]);
            float4 acc = f4fma(f4sub(nd[1], nd[4]), q.w2, nd[0]);
            acc = f4fma(f4sub(nd[2], nd[0]), q.w0, acc);
            acc = f4fma(f4sub(nd[3], nd[0]), q.w1, acc);
            return f4fma(cross, q.w0 * q.w1, acc);
        } else {
            // nd: c000 c1 c2 c111
            float4 acc = f4fma(f4sub(nd[1], nd[0]), q.w0, nd[0]);
            acc = f4fma(f4sub(nd[2], nd[1]), q.w1, acc);
            return f4fma(f4sub(nd[3], nd[2]), q.w2, acc);
        }
    }

    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        const Sel<METHOD> q = select(r, g, b);
        float4 nd[K];
        load(q, nd);
        const float4 v = value(nd, q);
        o0 = v.x;
        o1 = v.y;
        o2 = v.z;
        return q.base * 8 + q.simplex;
    }

};

// SMEM: stage the packed float3 LUT as float4 nodes in shared memory.
// Otherwise lut4 is the float4 copy in global memory.
template <int THREADS, int MINB, int METHOD, int N, bool SMEM, bool SEL, bool CACHED = false>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_interp(const __grid_constant__ ImageDesc im, const float *__restrict__ lut, const float4 *__restrict__ lut4,
             int n, int32_t *sel, int64_t ntiles)
{
    extern __shared__ float4 slut[];
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    OpLut<METHOD, N, SMEM, CACHED> op;
    if constexpr (SMEM) {
        const int nodes = n * n * n;
        for (int i = threadIdx.x; i < nodes; i += THREADS)
            slut[i] = make_float4(lut[3 * i], lut[3 * i + 1], lut[3 * i + 2], 0.0f);
        op.lut = slut;
    } else {
        op.lut = lut4;
    }
    op.st.n = n;
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

template <int THREADS, int MINB, int METHOD, int N, bool SMEM, bool SEL, bool CACHED = false>
static cudaError_t launch_interp(const mact_ctx &h, const ImageDesc &im, const float *lut, const float4 *lut4,
                                 int n, int32_t *sel, cudaStream_t s)
{
    const int64_t nt = tiles_of_t<THREADS>(im);
    if (nt == 0) return cudaSuccess;
    auto kern = k_lut_interp<THREADS, MINB, METHOD, N, SMEM, SEL, CACHED>;
    const size_t smem = SMEM ? (size_t)n * n * n * sizeof(float4) : 0;
    // The shared-memory attribute is per device: remember the devices it was
    // set on.  Occupancy per LUT size (it depends on the staged LUT's bytes).
    // Both caches are atomics: concurrent first launches compute the same value.
    static std::atomic<uint64_t> attr_devices{0};
    static std::atomic<int> occ_cache[kLutSmemMaxN + 1];
    if (SMEM) {
        const uint64_t bit = 1ull << (h.device & 63);
        if ((attr_devices.load(std::memory_order_acquire) & bit) == 0) {
            const int maxs = kLutSmemMaxN * kLutSmemMaxN * kLutSmemMaxN * (int)sizeof(float4);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
            if (e != cudaSuccess) return e;
            attr_devices.fetch_or(bit, std::memory_order_acq_rel);
        }
    }
    std::atomic<int> &slot = occ_cache[SMEM ? n : 0];
    int occ = slot.load(std::memory_order_relaxed);
    if (occ == 0) {
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, THREADS, smem);
        occ = (e != cudaSuccess || o <= 0) ? 1 : o;
        slot.store(occ, std::memory_order_relaxed);
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    const int64_t grid = nt < cap ? nt : cap;
    kern<<<(unsigned)grid, THREADS, smem, s>>>(im, lut, lut4, n, sel, nt);
    return cudaGetLastError();
}

template <int METHOD, int N, bool SMEM>
static cudaError_t launch_sel(const mact_ctx &h, const ImageDesc &im, const float *lut, const float4 *lut4, int n,
                              int32_t *sel, cudaStream_t s)
{
    constexpr int T = SMEM ? SmemThreads<METHOD>::value : GlobalShape<METHOD>::threads;
    // two CTAs per SM for the shared-memory LUT; for the global one a cap of
    // 80 registers, where 64 spilled and measured 5-8% slower
    constexpr int MINB = SMEM ? 2 : GlobalShape<METHOD>::ctas;
    ImageDesc imt = im;   // one long row of tiles of this launch shape
    imt.tiles_per_row = (im.width + TileShape<T>::px - 1) / TileShape<T>::px;
    if (sel) return launch_interp<T, MINB, METHOD, N, SMEM, true>(h, imt, lut, lut4, n, sel, s);
    return launch_interp<T, MINB, METHOD, N, SMEM, false>(h, imt, lut, lut4, n, sel, s);
}

template <int METHOD>
static cudaError_t interp_method(const mact_ctx &h, const ImageDesc &im, const float *lut, const float4 *lut4,
                                 int n, int32_t *sel, cudaStream_t s)
{
    if (n == 9) return launch_sel<METHOD, 9, true>(h, im, lut, lut4, n, sel, s);
    if (n == 17) return launch_sel<METHOD, 17, true>(h, im, lut, lut4, n, sel, s);
    if (n == 33) return launch_sel<METHOD, 33, false>(h, im, lut, lut4, n, sel, s);
    if (n <= kLutSmemMaxN) return launch_sel<METHOD, 0, true>(h, im, lut, lut4, n, sel, s);
    return launch_sel<METHOD, 0, false>(h, im, lut, lut4, n, sel, s);
}

cudaError_t launch_lut_interp(const mact_ctx &h, int method, const float *d_lut, int n, const uint8_t *d_rgb,
                              int64_t npix, float *const out[3], int32_t *d_sel, const float4 *d_lut4,
                              cudaStream_t s)
{
    ImageDesc im{};
    im.rgb = d_rgb;
    for (int c = 0; c < 3; ++c) im.out[c] = out[c];
    im.width = npix;
    im.height = 1;
    im.pitch = 3 * npix;
    im.opitch = npix;
    im.space = MACT_CIELAB;
    im.dtype = MACT_F32;
    switch (method) {
    case MACT_TRILINEAR: return interp_method<MACT_TRILINEAR>(h, im, d_lut, d_lut4, n, d_sel, s);
    case MACT_PRISM: return interp_method<MACT_PRISM>(h, im, d_lut, d_lut4, n, d_sel, s);
    case MACT_PYRAMID: return interp_method<MACT_PYRAMID>(h, im, d_lut, d_lut4, n, d_sel, s);
    default: return interp_method<MACT_TETRA>(h, im, d_lut, d_lut4, n, d_sel, s);
    }
}

template <int METHOD, int N>
static cudaError_t cached_sel(const mact_ctx &h, const ImageDesc &im, const float4 *cache, int n, int32_t *sel,
                              cudaStream_t s)
{
    if (sel) return launch_interp<kThreads, 4, METHOD, N, false, true, true>(h, im, nullptr, cache, n, sel, s);
    return launch_interp<kThreads, 4, METHOD, N, false, false, true>(h, im, nullptr, cache, n, sel, s);
}

template <int METHOD>
static cudaError_t cached_method(const mact_ctx &h, const ImageDesc &im, const float4 *cache, int n, int32_t *sel,
                                 cudaStream_t s)
{
    if (n == 17) return cached_sel<METHOD, 17>(h, im, cache, n, sel, s);
    if (n == 33) return cached_sel<METHOD, 33>(h, im, cache, n, sel, s);
    return cached_sel<METHOD, 0>(h, im, cache, n, sel, s);
}

cudaError_t launch_lut_interp_cached(const mact_ctx &h, int method, const float4 *d_cache, int n,
                                     const uint8_t *d_rgb, int64_t npix, float *const out[3], int32_t *d_sel,
                                     cudaStream_t s)
{
    ImageDesc im{};
    im.rgb = d_rgb;
    for (int c = 0; c < 3; ++c) im.out[c] = out[c];
    im.width = npix;
    im.height = 1;
    im.pitch = 3 * npix;
    im.opitch = npix;
    im.space = MACT_CIELAB;
    im.dtype = MACT_F32;
    const int P = TileShape<kThreads>::px;
    im.tiles_per_row = (npix + P - 1) / P;
    switch (method) {
    case MACT_TRILINEAR: return cached_method<MACT_TRILINEAR>(h, im, d_cache, n, d_sel, s);
    case MACT_PRISM: return cached_method<MACT_PRISM>(h, im, d_cache, n, d_sel, s);
    case MACT_PYRAMID: return cached_method<MACT_PYRAMID>(h, im, d_cache, n, d_sel, s);
    default: return cached_method<MACT_TETRA>(h, im, d_cache, n, d_sel, s);
    }
}

cudaError_t launch_lut_pack4(const float *d_lut, int n, float4 *d_lut4, cudaStream_t s)
{
    const int nodes = n * n * n;
    k_lut_pack4<<<(nodes + 255) / 256, 256, 0, s>>>(d_lut, nodes, d_lut4);
    return cudaGetLastError();
}

bool lut_needs_pack(int n) { return n > kLutSmemMaxN; }

}  // namespace mact
