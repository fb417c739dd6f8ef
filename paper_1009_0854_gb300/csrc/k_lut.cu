// k_lut.cu -- 3D-LUT packing and the trilinear / prism / pyramidal /
// tetrahedral interpolators (Section "Comparison with 3D Lookup Table
// Interpolation Methods"), on the streaming tile engine.
//
// Extraction is bit-identical to an integer implementation: along each axis
// s = v (n-1), idx = s div 255, rem = s mod 255, and the code v = 255 uses
// idx = n-2, rem = 255; the fraction is rem/255.  Every CTA tabulates, per
// 8-bit code and axis, the node offset idx * stride and the fraction, so a
// pixel's cell costs three shared loads; simplex choices compare fractions,
// which order exactly as the integer remainders do (x -> x/255 is strictly
// increasing on the integers 0..255 in FP32).
//
// LUT placement: for n <= 17 every CTA stages the whole LUT in shared memory
// as float4 nodes (17^3 x 16 B = 78.6 KB), so a node is one 16-byte shared
// load.  Larger LUTs (33^3: 575 KB as float4) are first repacked into float4
// nodes in a scratch buffer of the handle (one small kernel per call) and
// read from global memory (L1/L2 resident).  For n = 9, 17, 33 the node
// strides are compile-time constants, so node addresses are immediate
// offsets from the cell's base.
#include "engine.cuh"
#include "internal.h"

namespace mact {

constexpr int kLutSmemMaxN = 17;
constexpr int kLutThreadsSmem = 512;
// Cell extraction: false = integer arithmetic per pixel (div by 255 as a
// multiply-shift), true = per-code tables in shared memory.  The gathers of
// the interpolation already saturate the shared/L1 data pipe, so the
// arithmetic form (no extra shared loads) is the default.
constexpr bool kLocateByTable = false;

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

// ---------------------------------------------------------- interpolation

// Per-code extraction table entry: node offset along the axis and fraction.
struct AxisEntry {
    int off;
    float f;
};

__device__ __forceinline__ void fill_axis_tables(AxisEntry *tab, int n)
{
    // tab[axis * 256 + v], axis 0 = R (stride n^2), 1 = G (n), 2 = B (1)
    for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) {
        const int axis = i >> 8, v = i & 255;
        const int s = v * (n - 1);
        int idx = s / 255, rem = s - 255 * idx;
        if (idx == n - 1) { idx = n - 2; rem = 255; }
        const int stride = axis == 0 ? n * n : (axis == 1 ? n : 1);
        tab[i].off = idx * stride;
        tab[i].f = (float)rem * (1.0f / 255.0f);
    }
}

__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, 0.f); }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f); }
__device__ __forceinline__ float4 f4fma(float4 a, float s, float4 c)
{
    return make_float4(fmaf(a.x, s, c.x), fmaf(a.y, s, c.y), fmaf(a.z, s, c.z), 0.f);
}

// Node fetch: shared memory, or the read-only global path.
template <bool SMEM>
__device__ __forceinline__ float4 node(const float4 *p)
{
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

// Node strides: compile-time for N > 0, runtime otherwise.
template <int N>
struct Strides {
    int n;
    __device__ __forceinline__ int r() const { return N > 0 ? N * N : n * n; }
    __device__ __forceinline__ int g() const { return N > 0 ? N : n; }
};

template <int METHOD, int N, bool SMEM>
struct OpLut {
    const float4 *lut;        // shared or global float4 nodes
    const AxisEntry *tab;     // shared extraction table
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

    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        const int sR = st.r(), sG = st.g(), sB = 1;
        int base;
        float fr, fg, fb;
        if (kLocateByTable) {
            const AxisEntry er = tab[r], eg = tab[256 + g], eb = tab[512 + b];
            base = er.off + eg.off + eb.off;
            fr = er.f; fg = eg.f; fb = eb.f;
        } else {
            const int n = st.g();
            int ir, ig, ib;
            locate(r, n, ir, fr);
            locate(g, n, ig, fg);
            locate(b, n, ib, fb);
            base = ir * sR + ig * sG + ib;
        }
        const float4 *cb = lut + base;
        auto c = [cb](int k) { return node<SMEM>(cb + k); };
        float4 v;
        int simplex;
        if (METHOD == MACT_TRILINEAR) {
            const float4 c000 = c(0), c001 = c(sB), c010 = c(sG), c011 = c(sG + sB), c100 = c(sR),
                         c101 = c(sR + sB), c110 = c(sR + sG), c111 = c(sR + sG + sB);
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
            const bool lo = fg >= fb;
            const int oe = lo ? sG : sB;   // c010 or c001
            const float4 c000 = c(0), c100 = c(sR), c011 = c(sG + sB), c111 = c(sR + sG + sB);
            const float4 ce0 = c(oe), ce1 = c(sR + oe);
            const float fa = lo ? fg : fb, fc = lo ? fb : fg;
            const float4 t0 = f4fma(f4sub(c011, ce0), fc, f4fma(f4sub(ce0, c000), fa, c000));
            const float4 t1 = f4fma(f4sub(c111, ce1), fc, f4fma(f4sub(ce1, c100), fa, c100));
            v = f4fma(f4sub(t1, t0), fr, t0);
            simplex = lo ? 0 : 1;
        } else if (METHOD == MACT_PYRAMID) {
            // apex c111; base on the face of the smallest fraction (B, then G, then R)
            int oX, oY;
            float fX, fY, fZ;
            if (fb <= fr && fb <= fg) { oX = sR; oY = sG; fX = fr; fY = fg; fZ = fb; simplex = 0; }
            else if (fg <= fr && fg <= fb) { oX = sR; oY = sB; fX = fr; fY = fb; fZ = fg; simplex = 1; }
            else { oX = sG; oY = sB; fX = fg; fY = fb; fZ = fr; simplex = 2; }
            const float4 c000 = c(0), c111 = c(sR + sG + sB);
            const float4 cX = c(oX), cY = c(oY), cA = c(oX + oY);
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
            if (fr >= fg && fg >= fb)      { o1 = sR; o2 = sR + sG; f1 = fr; f2 = fg; f3 = fb; simplex = 0; }
            else if (fr >= fb && fb > fg)  { o1 = sR; o2 = sR + sB; f1 = fr; f2 = fb; f3 = fg; simplex = 1; }
            else if (fb > fr && fr >= fg)  { o1 = sB; o2 = sR + sB; f1 = fb; f2 = fr; f3 = fg; simplex = 2; }
            else if (fg > fr && fr >= fb)  { o1 = sG; o2 = sR + sG; f1 = fg; f2 = fr; f3 = fb; simplex = 3; }
            else if (fg >= fb && fb > fr)  { o1 = sG; o2 = sG + sB; f1 = fg; f2 = fb; f3 = fr; simplex = 4; }
            else                           { o1 = sB; o2 = sG + sB; f1 = fb; f2 = fg; f3 = fr; simplex = 5; }
            const float4 c000 = c(0), c1 = c(o1), c2 = c(o2), c111 = c(sR + sG + sB);
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

// SMEM: stage the packed float3 LUT as float4 nodes in shared memory.
// Otherwise lut4 is the float4 copy in global memory.
template <int THREADS, int MINB, int METHOD, int N, bool SMEM, bool SEL>
__global__ void __launch_bounds__(THREADS, MINB)
k_lut_interp(const __grid_constant__ ImageDesc im, const float *__restrict__ lut, const float4 *__restrict__ lut4,
             int n, int32_t *sel, int64_t ntiles)
{
    extern __shared__ float4 slut[];
    __shared__ uint4 sbuf[TileShape<THREADS>::vecs];
    __shared__ AxisEntry stab[kLocateByTable ? 3 * 256 : 1];
    if (kLocateByTable) fill_axis_tables(stab, n);
    OpLut<METHOD, N, SMEM> op;
    if constexpr (SMEM) {
        const int nodes = n * n * n;
        for (int i = threadIdx.x; i < nodes; i += THREADS)
            slut[i] = make_float4(lut[3 * i], lut[3 * i + 1], lut[3 * i + 2], 0.0f);
        op.lut = slut;
    } else {
        op.lut = lut4;
    }
    op.tab = stab;
    op.st.n = n;
    run_image<THREADS, float, SEL>(im, ntiles, op, sbuf, sel);
}

template <int THREADS, int MINB, int METHOD, int N, bool SMEM, bool SEL>
static cudaError_t launch_interp(const mact_ctx &h, const ImageDesc &im, const float *lut, const float4 *lut4,
                                 int n, int32_t *sel, cudaStream_t s)
{
    const int64_t nt = tiles_of_t<THREADS>(im);
    if (nt == 0) return cudaSuccess;
    auto kern = k_lut_interp<THREADS, MINB, METHOD, N, SMEM, SEL>;
    const size_t smem = SMEM ? (size_t)n * n * n * sizeof(float4) : 0;
    static int occ_cache[kLutSmemMaxN + 1] = {0};
    int &occ = occ_cache[SMEM ? n : 0];
    if (occ == 0) {
        if (SMEM) {
            const int maxs = kLutSmemMaxN * kLutSmemMaxN * kLutSmemMaxN * (int)sizeof(float4);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
            if (e != cudaSuccess) return e;
        }
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, THREADS, smem);
        occ = (e != cudaSuccess || o <= 0) ? 1 : o;
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
    constexpr int T = SMEM ? kLutThreadsSmem : kThreads;
    constexpr int MINB = SMEM ? 2 : 4;   // cap registers at 64 so 1024+ threads stay resident
    if (sel) return launch_interp<T, MINB, METHOD, N, SMEM, true>(h, im, lut, lut4, n, sel, s);
    return launch_interp<T, MINB, METHOD, N, SMEM, false>(h, im, lut, lut4, n, sel, s);
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
    const int P = n <= kLutSmemMaxN ? TileShape<kLutThreadsSmem>::px : TileShape<kThreads>::px;
    im.tiles_per_row = (npix + P - 1) / P;
    switch (method) {
    case MACT_TRILINEAR: return interp_method<MACT_TRILINEAR>(h, im, d_lut, d_lut4, n, d_sel, s);
    case MACT_PRISM: return interp_method<MACT_PRISM>(h, im, d_lut, d_lut4, n, d_sel, s);
    case MACT_PYRAMID: return interp_method<MACT_PYRAMID>(h, im, d_lut, d_lut4, n, d_sel, s);
    default: return interp_method<MACT_TETRA>(h, im, d_lut, d_lut4, n, d_sel, s);
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
