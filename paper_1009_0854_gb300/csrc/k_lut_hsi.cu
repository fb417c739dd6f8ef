// k_lut_hsi.cu -- a 3D LUT of the HSI transform with angular interpolation of
// the hue (Eq. equ_angular, in the closing paragraphs of Section "Comparison
// with 3D Lookup Table Interpolation Methods"), trilinear.
//
// The paper gives the pairwise mix of two angles,
//   theta = atan2((1 - a) sin t0 + a sin t1, (1 - a) cos t0 + a cos t1),
// and reports trilinear HSI interpolation built on it.  Reading: S and I
// take the trilinear weights; H is mixed pairwise along B, then G, then R
// (the order of repeated linear interpolation); a gray node (S = 0, hue
// undefined) has no hue, so a pair with one gray member takes the other's
// angle and a pair of grays stays gray; a result with S = 0 takes H = 0, the
// exact transform's convention for grays.
//
// Nodes hold (cos H, sin H, S, I) in FP32, the unit hue vector precomputed
// at build time (gray nodes: the zero vector).  Since the sine and cosine of
// a mixed angle are its normalised mixed vector, the chain needs no
// per-pixel trigonometry: seven normalisations (rsqrt) and one atan2.  A
// pair whose mixed vector vanishes (antipodal hues at a ~ 0.5) has no
// direction; it is treated as gray.
#include "engine.cuh"
#include "internal.h"

namespace mact {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Eq. equ_rgb_kender (exact) in FP64 on real-valued codes.
__device__ void hsi_exact64(double r, double g, double b, double &h, double &s, double &i)
{
    const double sum = r + g + b;
    const double mn = fmin(fmin(r, g), b);
    const double s3 = 1.7320508075688772;
    if (r > b && g > b) h = kPi / 3.0 + atan(s3 * (g - r) / (g - b + r - b));
    else if (g > r) h = kPi + atan(s3 * (b - g) / (b - r + g - r));
    else if (b > g) h = 5.0 * kPi / 3.0 + atan(s3 * (r - b) / (r - g + b - g));
    else h = 0.0;   // r > g = b (hue 0), or gray (convention)
    s = sum > 0.0 ? 1.0 - 3.0 * mn / sum : 0.0;
    i = sum / 765.0;
}

__global__ void k_lut_build_hsi(int n, float4 *__restrict__ lut)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= n * n * n) return;
    const int k = node % n, j = (node / n) % n, i = node / (n * n);
    const double step = 255.0 / (double)(n - 1);
    double h, s, v;
    hsi_exact64(i * step, j * step, k * step, h, s, v);
    const float hf = (float)h, sf = (float)s, vf = (float)v;
    if (sf == 0.0f) lut[node] = make_float4(0.0f, 0.0f, 0.0f, vf);
    else lut[node] = make_float4((float)cos((double)hf), (float)sin((double)hf), sf, vf);
}

// Integer cell extraction, as for the other LUT interpolators: s = v (n-1),
// idx = s div 255, rem = s mod 255; v = 255 uses idx = n-2, rem = 255.
__device__ __forceinline__ void locate(uint32_t v, int n, int &idx, float &f)
{
    const int s = (int)v * (n - 1);
    idx = s / 255;
    int rem = s - 255 * idx;
    if (idx == n - 1) { idx = n - 2; rem = 255; }
    f = (float)rem * (1.0f / 255.0f);
}

// Eq. equ_angular on unit vectors, gray (zero) members skipped.  The gray
// rule only changes the result when the mixed vector vanishes (a = 0 or 1
// against a gray member, both gray, or antipodal hues), so it is tested on
// that path alone; elsewhere normalising the mix gives the other member's
// direction to rounding.
__device__ __forceinline__ float2 angle_mix(float2 u0, float2 u1, float a)
{
    const float x = fmaf(a, u1.x - u0.x, u0.x);
    const float y = fmaf(a, u1.y - u0.y, u0.y);
    const float m2 = fmaf(x, x, y * y);
    if (m2 > 1e-30f) {
        const float r = rsqrtf(m2);
        return make_float2(x * r, y * r);
    }
    const bool g0 = u0.x == 0.0f && u0.y == 0.0f;
    const bool g1 = u1.x == 0.0f && u1.y == 0.0f;
    if (g0) return u1;
    if (g1) return u0;
    return make_float2(0.0f, 0.0f);
}

template <int N>
struct OpLutHsiAngular {
    const float4 *lut;
    int n;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        const int nn = N > 0 ? N : n;
        int ir, ig, ib;
        float fr, fg, fb;
        locate(r, nn, ir, fr);
        locate(g, nn, ig, fg);
        locate(b, nn, ib, fb);
        const float4 *c = lut + ((ir * nn + ig) * nn + ib);
        const int sG = nn, sR = nn * nn;
        // corner k = 4 dR + 2 dG + dB
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldg(c + ((k >> 2) & 1) * sR + ((k >> 1) & 1) * sG + (k & 1));
        // S and I: repeated linear interpolation along B, G, R (the trilinear weights)
        float s2[4], i2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s2[k] = fmaf(fb, v[2 * k + 1].z - v[2 * k].z, v[2 * k].z);
            i2[k] = fmaf(fb, v[2 * k + 1].w - v[2 * k].w, v[2 * k].w);
        }
        const float s0 = fmaf(fg, s2[1] - s2[0], s2[0]), s1 = fmaf(fg, s2[3] - s2[2], s2[2]);
        const float i0 = fmaf(fg, i2[1] - i2[0], i2[0]), i1 = fmaf(fg, i2[3] - i2[2], i2[2]);
        const float S = fmaf(fr, s1 - s0, s0);
        const float I = fmaf(fr, i1 - i0, i0);
        // H: the pairwise chain along B, G, R
        float2 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 a = v[2 * k], b1 = v[2 * k + 1];
            u[k] = angle_mix(make_float2(a.x, a.y), make_float2(b1.x, b1.y), fb);
        }
        const float2 w0 = angle_mix(u[0], u[1], fg), w1 = angle_mix(u[2], u[3], fg);
        const float2 hv = angle_mix(w0, w1, fr);
        float H = atan2f(hv.y, hv.x);
        if (H < 0.0f) H += 6.28318530717958648f;
        if (H >= 6.28318530717958648f) H -= 6.28318530717958648f;
        if (S == 0.0f) H = 0.0f;
        o0 = H;
        o1 = S;
        o2 = I;
        return 0;
    }
};

constexpr int kHsiLutThreads = 256;

template <int N>
__global__ void __launch_bounds__(kHsiLutThreads, 3)
k_lut_hsi_interp(const __grid_constant__ ImageDesc im, const float4 *__restrict__ lut, int n, int64_t ntiles)
{
    __shared__ uint4 sbuf[TileShape<kHsiLutThreads>::vecs];
    OpLutHsiAngular<N> op{lut, n};
    run_image<kHsiLutThreads, float, false>(im, ntiles, op, sbuf, nullptr);
}

template <int N>
cudaError_t launch_hsi_interp(const mact_ctx &h, const ImageDesc &im, const float4 *lut, int n, cudaStream_t s)
{
    const int64_t nt = tiles_of_t<kHsiLutThreads>(im);
    if (nt == 0) return cudaSuccess;
    static const int occ = [] {   // thread-safe one-time init
        int o = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_lut_hsi_interp<N>, kHsiLutThreads, 0);
        return (e != cudaSuccess || o <= 0) ? 1 : o;
    }();
    const int64_t cap = (int64_t)h.num_sms * occ;
    const int64_t grid = nt < cap ? nt : cap;
    k_lut_hsi_interp<N><<<(unsigned)grid, kHsiLutThreads, 0, s>>>(im, lut, n, nt);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lut_build_hsi(int n, float4 *d_lut4, cudaStream_t s)
{
    const int nodes = n * n * n;
    k_lut_build_hsi<<<(nodes + 255) / 256, 256, 0, s>>>(n, d_lut4);
    return cudaGetLastError();
}

cudaError_t launch_lut_interp_hsi(const mact_ctx &h, const float4 *d_lut4, int n, const uint8_t *d_rgb,
                                  int64_t npix, float *const out[3], cudaStream_t s)
{
    ImageDesc im{};
    im.rgb = d_rgb;
    for (int c = 0; c < 3; ++c) im.out[c] = out[c];
    im.width = npix;
    im.height = 1;
    im.pitch = 3 * npix;
    im.opitch = npix;
    im.space = MACT_HSI;
    im.dtype = MACT_F32;
    im.tiles_per_row = (npix + TileShape<kHsiLutThreads>::px - 1) / TileShape<kHsiLutThreads>::px;
    if (n == 17) return launch_hsi_interp<17>(h, im, d_lut4, n, s);
    if (n == 33) return launch_hsi_interp<33>(h, im, d_lut4, n, s);
    return launch_hsi_interp<0>(h, im, d_lut4, n, s);
}

}  // namespace mact
