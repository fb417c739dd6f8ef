// k_eps.cu -- transformation error over every 24-bit colour, on the GPU.
//
// Section "Calculation of the Color Space Transformation Errors": the paper
// reports, over all 2^24 colours, the average and maximum distance between
// the approximate and the exact transform -- Delta E*ab (Eq. equ_cielab_dist)
// for CIELAB and for SCT (after the inverse SCT, Eq. equ_sct_rgb, and
// conversion to CIELAB), D_HSI (Eq. equ_hsi_dist) for HSI -- and the same
// Delta E*ab for the LUT interpolators (Table tab_lut).  Here each colour is
// generated from its index (no input buffer), pushed through the production
// FP32 per-pixel operator, and compared with the exact transform evaluated
// in FP64 on the device.  Sums and maxima are reduced per CTA in FP64 and
// then in a fixed order, so the result is deterministic.
#include "internal.h"
#include "pixel.cuh"

namespace mact {

constexpr int kEpsThreads = 256;

struct Exact64 {
    const double *g64;   // FP64 linearisation table (256)
    const double *m;     // rgb_to_xyz / white, FP64
    double gt, gs, go, ge;   // gamma parameters for non-integer codes
};

__device__ __forceinline__ double lin_of_real(double code, const Exact64 &x)
{
    const double kp = code / 255.0;
    if (kp < x.gt) return kp / x.gs;
    return pow((kp + x.go) / (1.0 + x.go), x.ge);
}

__device__ __forceinline__ void lab_from_lin(double k0, double k1, double k2, const Exact64 &x, double lab[3])
{
    double f[3];
    for (int c = 0; c < 3; ++c) {
        const double t = x.m[3 * c] * k0 + x.m[3 * c + 1] * k1 + x.m[3 * c + 2] * k2;
        f[c] = t > 0.008856 ? cbrt(t) : 7.787 * t + 16.0 / 116.0;
    }
    lab[0] = 116.0 * f[1] - 16.0;
    lab[1] = 500.0 * (f[0] - f[1]);
    lab[2] = 200.0 * (f[1] - f[2]);
}

__device__ __forceinline__ double dist3(const double a[3], double b0, double b1, double b2)
{
    const double d0 = a[0] - b0, d1 = a[1] - b1, d2 = a[2] - b2;
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

// error of one colour; KIND 0 CIELAB, 1 HSI, 2 SCT, 3 LUT (values are Lab)
template <int KIND>
__device__ __forceinline__ double colour_error(uint32_t r, uint32_t g, uint32_t b, float o0, float o1, float o2,
                                               const Exact64 &x)
{
    if (KIND == 1) {
        // exact Kender hue (Eq. equ_rgb_kender), S, I; D_HSI (Eq. equ_hsi_dist)
        const double R = r, G = g, B = b, pi = 3.14159265358979323846;
        double H = 0.0;
        if (R > B && G > B) H = pi / 3.0 + atan(sqrt(3.0) * (G - R) / (G - B + R - B));
        else if (G > R) H = pi + atan(sqrt(3.0) * (B - G) / (B - R + G - R));
        else if (B > G) H = 5.0 * pi / 3.0 + atan(sqrt(3.0) * (R - B) / (R - G + B - G));
        const double sum = R + G + B, mn = fmin(R, fmin(G, B));
        const double S = sum > 0.0 ? 1.0 - 3.0 * mn / sum : 0.0;
        const double I = sum / 765.0;
        double dh = fabs(H - (double)o0);
        const double th = dh <= pi ? dh : 2.0 * pi - dh;
        const double si = (double)o1, ii = (double)o2;
        const double v = S * S + si * si - 2.0 * S * si * cos(th) + (I - ii) * (I - ii);
        return sqrt(v > 0.0 ? v : 0.0);
    }
    double ref[3];
    lab_from_lin(x.g64[r], x.g64[g], x.g64[b], x, ref);
    if (KIND == 2) {
        // inverse SCT (Eq. equ_sct_rgb) to real-valued codes, then exact CIELAB
        const double L = o0, A = o1, Bg = o2;
        const double rr = L * sin(A) * cos(Bg), gg = L * sin(A) * sin(Bg), bb = L * cos(A);
        double lab[3];
        lab_from_lin(lin_of_real(rr, x), lin_of_real(gg, x), lin_of_real(bb, x), x, lab);
        return dist3(ref, lab[0], lab[1], lab[2]);
    }
    return dist3(ref, o0, o1, o2);
}

template <int KIND, class Op>
__device__ __forceinline__ void eps_body(const Op &op, const Exact64 &x, double2 *partial)
{
    double sum = 0.0, mx = 0.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (1u << 24); k += gridDim.x * blockDim.x) {
        const uint32_t r = k >> 16, g = (k >> 8) & 255u, b = k & 255u;
        float o0, o1, o2;
        op(r, g, b, o0, o1, o2);
        const double e = colour_error<KIND>(r, g, b, o0, o1, o2, x);
        sum += e;
        mx = fmax(mx, e);
    }
    __shared__ double rs[kEpsThreads], rm[kEpsThreads];
    rs[threadIdx.x] = sum;
    rm[threadIdx.x] = mx;
    __syncthreads();
    for (int s = kEpsThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            rs[threadIdx.x] += rs[threadIdx.x + s];
            rm[threadIdx.x] = fmax(rm[threadIdx.x], rm[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = make_double2(rs[0], rm[0]);
}

template <int KIND, bool EXACT, int RDEG>
__global__ void __launch_bounds__(kEpsThreads)
k_eps_space(const __grid_constant__ Coeffs co, const float *__restrict__ gamma, Exact64 x, double2 *partial)
{
    __shared__ float sgam[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sgam[i] = gamma[i];
    __syncthreads();
    if (KIND == 0) {
        const OpCielab<EXACT, RDEG> op{RDEG != 0 || EXACT ? sgam : reinterpret_cast<const float *>(x.g64), co};
        eps_body<0>(op, x, partial);
    } else if (KIND == 1) {
        const OpHsi<EXACT> op{co};
        eps_body<1>(op, x, partial);
    } else {
        const OpSct<EXACT> op{co};
        eps_body<2>(op, x, partial);
    }
}

// LUT interpolation with the same integer extraction as k_lut.cu (global
// float4 nodes, runtime strides): Lab values
struct LutEval {
    const float4 *lut;
    int n;
    int method;
    __device__ __forceinline__ static void locate(uint32_t v, int n, int &idx, float &f)
    {
        const int s = (int)v * (n - 1);
        idx = s / 255;
        int rem = s - 255 * idx;
        if (idx == n - 1) { idx = n - 2; rem = 255; }
        f = (float)rem * (1.0f / 255.0f);
    }
    __device__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1, float &o2) const;
};

__device__ __forceinline__ float4 l4(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ float4 s4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, 0.f); }
__device__ __forceinline__ float4 a4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, 0.f); }
__device__ __forceinline__ float4 m4(float4 a, float s, float4 c)
{
    return make_float4(fmaf(a.x, s, c.x), fmaf(a.y, s, c.y), fmaf(a.z, s, c.z), 0.f);
}

__device__ int LutEval::operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1, float &o2) const
{
    int ir, ig, ib;
    float fr, fg, fb;
    locate(r, n, ir, fr);
    locate(g, n, ig, fg);
    locate(b, n, ib, fb);
    const int sR = n * n, sG = n, sB = 1;
    const float4 *c = lut + (ir * sR + ig * sG + ib);
    float4 v;
    if (method == MACT_TRILINEAR) {
        const float4 c00 = m4(s4(l4(c + sB), l4(c)), fb, l4(c));
        const float4 c01 = m4(s4(l4(c + sG + sB), l4(c + sG)), fb, l4(c + sG));
        const float4 c10 = m4(s4(l4(c + sR + sB), l4(c + sR)), fb, l4(c + sR));
        const float4 c11 = m4(s4(l4(c + sR + sG + sB), l4(c + sR + sG)), fb, l4(c + sR + sG));
        const float4 c0 = m4(s4(c01, c00), fg, c00), c1 = m4(s4(c11, c10), fg, c10);
        v = m4(s4(c1, c0), fr, c0);
    } else if (method == MACT_PRISM) {
        const bool lo = fg >= fb;
        const int oe = lo ? sG : sB;
        const float fa = lo ? fg : fb, fc = lo ? fb : fg;
        const float4 c000 = l4(c), c100 = l4(c + sR), c011 = l4(c + sG + sB), c111 = l4(c + sR + sG + sB);
        const float4 ce0 = l4(c + oe), ce1 = l4(c + sR + oe);
        const float4 t0 = m4(s4(c011, ce0), fc, m4(s4(ce0, c000), fa, c000));
        const float4 t1 = m4(s4(c111, ce1), fc, m4(s4(ce1, c100), fa, c100));
        v = m4(s4(t1, t0), fr, t0);
    } else if (method == MACT_PYRAMID) {
        int oX, oY;
        float fX, fY, fZ;
        if (fb <= fr && fb <= fg) { oX = sR; oY = sG; fX = fr; fY = fg; fZ = fb; }
        else if (fg <= fr && fg <= fb) { oX = sR; oY = sB; fX = fr; fY = fb; fZ = fg; }
        else { oX = sG; oY = sB; fX = fg; fY = fb; fZ = fr; }
        const float4 c000 = l4(c), c111 = l4(c + sR + sG + sB), cX = l4(c + oX), cY = l4(c + oY),
                     cA = l4(c + oX + oY);
        const float4 cross = a4(s4(s4(cA, cX), cY), c000);
        float4 acc = m4(s4(c111, cA), fZ, c000);
        acc = m4(s4(cX, c000), fX, acc);
        acc = m4(s4(cY, c000), fY, acc);
        v = m4(cross, fX * fY, acc);
    } else {
        int p1, p2;
        float f1, f2, f3;
        if (fr >= fg && fg >= fb)      { p1 = sR; p2 = sR + sG; f1 = fr; f2 = fg; f3 = fb; }
        else if (fr >= fb && fb > fg)  { p1 = sR; p2 = sR + sB; f1 = fr; f2 = fb; f3 = fg; }
        else if (fb > fr && fr >= fg)  { p1 = sB; p2 = sR + sB; f1 = fb; f2 = fr; f3 = fg; }
        else if (fg > fr && fr >= fb)  { p1 = sG; p2 = sR + sG; f1 = fg; f2 = fr; f3 = fb; }
        else if (fg >= fb && fb > fr)  { p1 = sG; p2 = sG + sB; f1 = fg; f2 = fb; f3 = fr; }
        else                           { p1 = sB; p2 = sG + sB; f1 = fb; f2 = fg; f3 = fr; }
        const float4 c000 = l4(c), c1 = l4(c + p1), c2 = l4(c + p2), c111 = l4(c + sR + sG + sB);
        float4 acc = m4(s4(c1, c000), f1, c000);
        acc = m4(s4(c2, c1), f2, acc);
        v = m4(s4(c111, c2), f3, acc);
    }
    o0 = v.x;
    o1 = v.y;
    o2 = v.z;
    return 0;
}

__global__ void __launch_bounds__(kEpsThreads) k_eps_lut(LutEval op, Exact64 x, double2 *partial)
{
    eps_body<3>(op, x, partial);
}

__global__ void k_eps_reduce(const double2 *__restrict__ partial, int n, double *out)
{
    __shared__ double rs[kEpsThreads], rm[kEpsThreads];
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        s += partial[i].x;
        m = fmax(m, partial[i].y);
    }
    rs[threadIdx.x] = s;
    rm[threadIdx.x] = m;
    __syncthreads();
    for (int st = kEpsThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            rs[threadIdx.x] += rs[threadIdx.x + st];
            rm[threadIdx.x] = fmax(rm[threadIdx.x], rm[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = rs[0] / 16777216.0;
        out[1] = rm[0];
    }
}

static Exact64 exact_of(const mact_ctx &h, const double *d_m64)
{
    Exact64 x;
    x.g64 = reinterpret_cast<const double *>(h.d_gamma + 256);
    x.m = d_m64;
    x.gt = h.cfg.rgb.gamma_threshold;
    x.gs = h.cfg.rgb.gamma_slope;
    x.go = h.cfg.rgb.gamma_offset;
    x.ge = h.cfg.rgb.gamma_exponent;
    return x;
}

template <int KIND>
static void launch_space(const mact_ctx &h, int grid, const Exact64 &x, double2 *partial, cudaStream_t s)
{
    if (h.cfg.exact) {
        k_eps_space<KIND, true, 4><<<grid, kEpsThreads, 0, s>>>(h.co, h.d_gamma, x, partial);
    } else if constexpr (KIND != 0) {   // the cube-root form matters to CIELAB only
        k_eps_space<KIND, false, 4><<<grid, kEpsThreads, 0, s>>>(h.co, h.d_gamma, x, partial);
    } else {
        if (!h.co.lab_rational) k_eps_space<0, false, 0><<<grid, kEpsThreads, 0, s>>>(h.co, h.d_gamma, x, partial);
        else if (h.co.lab_deg == 6) k_eps_space<0, false, 6><<<grid, kEpsThreads, 0, s>>>(h.co, h.d_gamma, x, partial);
        else k_eps_space<0, false, 4><<<grid, kEpsThreads, 0, s>>>(h.co, h.d_gamma, x, partial);
    }
}

// target: 0..2 = space of the handle's transform; 3 = LUT (method, d_lut4, n)
cudaError_t run_cube_error(const mact_ctx &h, int target, int method, const float4 *d_lut4, int n,
                           double out[2], cudaStream_t s)
{
    const int grid = h.num_sms * 4;
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, grid * sizeof(double2) + 9 * sizeof(double) + 2 * sizeof(double));
    if (e != cudaSuccess) return e;
    double2 *partial = static_cast<double2 *>(buf);
    double *d_m = reinterpret_cast<double *>(partial + grid);
    double *d_out = d_m + 9;
    e = cudaMemcpyAsync(d_m, h.co.m64, 9 * sizeof(double), cudaMemcpyHostToDevice, s);
    const Exact64 x = exact_of(h, d_m);
    if (e == cudaSuccess) {
        if (target == 0) launch_space<0>(h, grid, x, partial, s);
        else if (target == 1) launch_space<1>(h, grid, x, partial, s);
        else if (target == 2) launch_space<2>(h, grid, x, partial, s);
        else k_eps_lut<<<grid, kEpsThreads, 0, s>>>(LutEval{d_lut4, n, method}, x, partial);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_eps_reduce<<<1, kEpsThreads, 0, s>>>(partial, grid, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    return e;
}

}  // namespace mact
