// k_lut.cu -- 3D-LUT packing and the trilinear / prism / pyramidal /
// tetrahedral interpolators (Section "Comparison with 3D Lookup Table
// Interpolation Methods"), on the streaming tile engine.
//
// Extraction is integer-only so that the cell and simplex chosen are
// bit-identical to any exact implementation: along each axis
// s = v (n-1), idx = s div 255, rem = s mod 255, and the code v = 255 uses
// idx = n-2, rem = 255; the fraction is rem/255.  Simplex choices compare the
// integer remainders.
//
// LUT placement: for n <= 17 every CTA stages the whole LUT in shared memory
// as float4 nodes (17^3 x 16 B = 78.6 KB), so each node is one 16-byte
// shared load; larger LUTs (33^3 = 431 KB) stay in global memory, read
// through the read-only path (they stay resident in L2 and partly in L1).
#include "engine.cuh"
#include "internal.h"

namespace mact {

constexpr int kLutSmemMaxN = 17;
constexpr int kLutThreadsSmem = 512;

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

// ---------------------------------------------------------- interpolation

__device__ __forceinline__ void locate(uint32_t v, int n, int &idx, int &rem)
{
    const int s = (int)v * (n - 1);
    idx = s / 255;
    rem = s - 255 * idx;
    if (idx == n - 1) { idx = n - 2; rem = 255; }
}

// Node fetch from shared (float4) or global (packed float3) storage.
template <bool SMEM>
struct Nodes;
template <>
struct Nodes<true> {
    const float4 *p;
    __device__ __forceinline__ float4 operator[](int i) const { return p[i]; }
};
template <>
struct Nodes<false> {
    const float *p;
    __device__ __forceinline__ float4 operator[](int i) const
    {
        return make_float4(__ldg(p + 3 * i), __ldg(p + 3 * i + 1), __ldg(p + 3 * i + 2), 0.0f);
    }
};

__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f); }
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, 0.f); }
__device__ __forceinline__ float4 f4fma(float4 a, float s, float4 c)
{
    return make_float4(fmaf(a.x, s, c.x), fmaf(a.y, s, c.y), fmaf(a.z, s, c.z), 0.f);
}

template <int METHOD, bool SMEM>
struct OpLut {
    Nodes<SMEM> lut;
    int n;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        int ir, ig, ib, rr, rg, rb;
        locate(r, n, ir, rr);
        locate(g, n, ig, rg);
        locate(b, n, ib, rb);
        const float fr = (float)rr * (1.0f / 255.0f);
        const float fg = (float)rg * (1.0f / 255.0f);
        const float fb = (float)rb * (1.0f / 255.0f);
        const int base = (ir * n + ig) * n + ib;
        const int sR = n * n, sG = n, sB = 1;   // node strides
        float4 v;
        int simplex;
        if (METHOD == MACT_TRILINEAR) {
            const float4 c000 = lut[base], c001 = lut[base + sB], c010 = lut[base + sG],
                         c011 = lut[base + sG + sB], c100 = lut[base + sR], c101 = lut[base + sR + sB],
                         c110 = lut[base + sR + sG], c111 = lut[base + sR + sG + sB];
            // repeated linear interpolation along B, then G, then R
            const float4 c00 = f4fma(f4sub(c001, c000), fb, c000);
            const float4 c01 = f4fma(f4sub(c011, c010), fb, c010);
            const float4 c10 = f4fma(f4sub(c101, c100), fb, c100);
            const float4 c11 = f4fma(f4sub(c111, c110), fb, c110);
            const float4 c0 = f4fma(f4sub(c01, c00), fg, c00);
            const float4 c1 = f4fma(f4sub(c11, c10), fg, c10);
            v = f4fma(f4sub(c1, c0), fr, c0);
            simplex = 0;
        } else if (METHOD == MACT_PRISM) {
            // prism axis R; triangle in the G-B face chosen by rem_G >= rem_B
            const bool lo = rg >= rb;
            const float4 c000 = lut[base], c100 = lut[base + sR];
            const float4 c011 = lut[base + sG + sB], c111 = lut[base + sR + sG + sB];
            const int oe = lo ? sG : sB;          // c010 or c001
            const float4 ce0 = lut[base + oe], ce1 = lut[base + sR + oe];
            // lo:  c000 + (c010-c000) fg + (c011-c010) fb + R-linear part
            // !lo: c000 + (c011-c001) fg + (c001-c000) fb + R-linear part
            const float fa = lo ? fg : fb, fc = lo ? fb : fg;
            const float4 t0 = f4fma(f4sub(c011, ce0), fc, f4fma(f4sub(ce0, c000), fa, c000));
            const float4 t1 = f4fma(f4sub(c111, ce1), fc, f4fma(f4sub(ce1, c100), fa, c100));
            v = f4fma(f4sub(t1, t0), fr, t0);
            simplex = lo ? 0 : 1;
        } else if (METHOD == MACT_PYRAMID) {
            // apex c111; base on the face of the smallest fraction (B, then G, then R)
            int oX, oY, oA;
            float fX, fY, fZ;
            if (rb <= rr && rb <= rg) { oX = sR; oY = sG; fX = fr; fY = fg; fZ = fb; simplex = 0; }
            else if (rg <= rr && rg <= rb) { oX = sR; oY = sB; fX = fr; fY = fb; fZ = fg; simplex = 1; }
            else { oX = sG; oY = sB; fX = fg; fY = fb; fZ = fr; simplex = 2; }
            oA = oX + oY;
            const float4 c000 = lut[base], c111 = lut[base + sR + sG + sB];
            const float4 cX = lut[base + oX], cY = lut[base + oY], cA = lut[base + oA];
            // c000 + (c111-cA) fZ + (cX-c000) fX + (cY-c000) fY + (cA-cX-cY+c000) fX fY
            const float4 cross = f4add(f4sub(f4sub(cA, cX), cY), c000);
            float4 acc = f4fma(f4sub(c111, cA), fZ, c000);
            acc = f4fma(f4sub(cX, c000), fX, acc);
            acc = f4fma(f4sub(cY, c000), fY, acc);
            v = f4fma(cross, fX * fY, acc);
        } else {
            // tetrahedral: path from c000 along the axes in decreasing fraction
            int o1, o2;
            float f1, f2, f3;
            if (rr >= rg && rg >= rb)      { o1 = sR; o2 = sR + sG; f1 = fr; f2 = fg; f3 = fb; simplex = 0; }
            else if (rr >= rb && rb > rg)  { o1 = sR; o2 = sR + sB; f1 = fr; f2 = fb; f3 = fg; simplex = 1; }
            else if (rb > rr && rr >= rg)  { o1 = sB; o2 = sR + sB; f1 = fb; f2 = fr; f3 = fg; simplex = 2; }
            else if (rg > rr && rr >= rb)  { o1 = sG; o2 = sR + sG; f1 = fg; f2 = fr; f3 = fb; simplex = 3; }
            else if (rg >= rb && rb > rr)  { o1 = sG; o2 = sG + sB; f1 = fg; f2 = fb; f3 = fr; simplex = 4; }
            else                           { o1 = sB; o2 = sG + sB; f1 = fb; f2 = fg; f3 = fr; simplex = 5; }
            const float4 c000 = lut[base], c1 = lut[base + o1], c2 = lut[base + o2],
                         c111 = lut[base + sR + sG + sB];
            float4 acc = f4fma(f4sub(c1, c000), f1, c000);
            acc = f4fma(f4sub(c2, c1), f2, acc);
            v = f4fma(f4sub(c111, c2), f3, acc);
        }
        o0 = v.x;
        o1 = v.y;
        o2 = v.z;
        return base * 8 + simplex;
    }
};

template <int THREADS, int METHOD, bool SMEM, bool SEL>
__global__ void __launch_bounds__(THREADS)
k_lut_interp(const __grid_constant__ ImageDesc im, const float *__restrict__ lut, int n, int32_t *sel,
             int64_t ntiles)
{
    extern __shared__ float4 slut[];
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    OpLut<METHOD, SMEM> op;
    if constexpr (SMEM) {
        const int nodes = n * n * n;
        for (int i = threadIdx.x; i < nodes; i += THREADS)
            slut[i] = make_float4(lut[3 * i], lut[3 * i + 1], lut[3 * i + 2], 0.0f);
        op.lut.p = slut;
    } else {
        op.lut.p = lut;
    }
    op.n = n;
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

template <int THREADS, int METHOD, bool SMEM, bool SEL>
static cudaError_t launch_interp(const mact_ctx &h, const ImageDesc &im, const float *lut, int n,
                                 int32_t *sel, cudaStream_t s)
{
    const int64_t nt = tiles_of_t<THREADS>(im);
    if (nt == 0) return cudaSuccess;
    auto kern = k_lut_interp<THREADS, METHOD, SMEM, SEL>;
    const size_t smem = SMEM ? (size_t)kLutSmemMaxN * kLutSmemMaxN * kLutSmemMaxN * sizeof(float4) : 0;
    static int occ = 0;
    if (occ == 0) {
        if (SMEM) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, THREADS, smem);
        occ = (e != cudaSuccess || o <= 0) ? 1 : o;
    }
    const int64_t cap = (int64_t)h.num_sms * occ;
    const int64_t grid = nt < cap ? nt : cap;
    kern<<<(unsigned)grid, THREADS, smem, s>>>(im, lut, n, sel, nt);
    return cudaGetLastError();
}

template <int METHOD>
static cudaError_t interp_method(const mact_ctx &h, const ImageDesc &im, const float *lut, int n,
                                 int32_t *sel, cudaStream_t s)
{
    if (n <= kLutSmemMaxN) {
        if (sel) return launch_interp<kLutThreadsSmem, METHOD, true, true>(h, im, lut, n, sel, s);
        return launch_interp<kLutThreadsSmem, METHOD, true, false>(h, im, lut, n, sel, s);
    }
    if (sel) return launch_interp<kThreads, METHOD, false, true>(h, im, lut, n, sel, s);
    return launch_interp<kThreads, METHOD, false, false>(h, im, lut, n, sel, s);
}

cudaError_t launch_lut_interp(const mact_ctx &h, int method, const float *d_lut, int n, const uint8_t *d_rgb,
                              int64_t npix, float *const out[3], int32_t *d_sel, cudaStream_t s)
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
    const int P = n <= kLutSmemMaxN ? TileShape<kLutThreadsSmem>::px : TileShape<kThreads>::px;
    im.tiles_per_row = (npix + P - 1) / P;
    switch (method) {
    case MACT_TRILINEAR: return interp_method<MACT_TRILINEAR>(h, im, d_lut, n, d_sel, s);
    case MACT_PRISM: return interp_method<MACT_PRISM>(h, im, d_lut, n, d_sel, s);
    case MACT_PYRAMID: return interp_method<MACT_PYRAMID>(h, im, d_lut, n, d_sel, s);
    default: return interp_method<MACT_TETRA>(h, im, d_lut, n, d_sel, s);
    }
}

}  // namespace mact
