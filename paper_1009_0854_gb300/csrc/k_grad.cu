// k_grad.cu -- differentiable RGB -> CIELAB on linear RGB input.
//
// Input x is linear RGB (the output of Eq. equ_rgb_lin) as planar FP32
// (N, 3, HW).  Forward: t = (M / white) x (Eq. equ_rgb_xyz), f(t) with the
// cube root replaced by the handle's rational approximant (or cbrtf in the
// exact configuration), Lab from Eq. equ_xyz_lab.  Backward applies the
// chain rule with the derivative of what the forward evaluates:
//   f'(t) = (d'(t) q(t) - d(t) q'(t)) / q(t)^2   for f = 1 + d/q (t > 0.008856)
//   f'(t) = f(t) / (3 t)                           exact cube root
//   f'(t) = 7.787                                  linear segment t <= 0.008856
//   dL/df_y = 116, da/df_x = 500, da/df_y = -500, db/df_y = 200, db/df_z = -200
// and dt/dx = M / white.  The fused loss kernel computes the mean Delta E*ab
// against a target Lab image and its gradient in one pass (reads x and the
// target, writes the gradient: 36 bytes per pixel); per-CTA partial sums are
// reduced in a fixed order by a second one-CTA kernel, so the loss is
// deterministic.
#include <initializer_list>

#include "internal.h"
#include "pixel.cuh"

namespace mact {

constexpr int kGradThreads = 256;

// FORM: 0 = the exact cube root; 4 or 6 = the rational with chains of that
// degree (derivative chains one lower).
template <int FORM>
__device__ __forceinline__ void f_df(float t, const Coeffs &co, float &f, float &df)
{
    if (t <= kKnee) {
        f = fmaf(kLinSlope, t, kLinOffset);
        df = kLinSlope;
        return;
    }
    if (FORM == 0) {
        f = cbrtf(t);
        df = f * rcp_nr(3.0f * t);
    } else {
        constexpr int D = FORM == 0 ? 4 : FORM;
        const float d = horner<D>(co.lab_d, t);
        const float q = horner<D>(co.lab_q, t);
        const float r = rcp_nr(q);
        f = fmaf(d, r, 1.0f);
        const float dd = horner<D - 1>(co.lab_dd, t);
        const float dq = horner<D - 1>(co.lab_dq, t);
        df = fmaf(dd, q, -d * dq) * (r * r);
    }
}

struct PixelLab {
    float lab[3];
    float df[3];
};

template <int FORM>
__device__ __forceinline__ PixelLab lab_of(float x0, float x1, float x2, const Coeffs &co)
{
    PixelLab p;
    float f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t = fmaf(co.m[3 * c + 2], x2, fmaf(co.m[3 * c + 1], x1, co.m[3 * c] * x0));
        f_df<FORM>(t, co, f[c], p.df[c]);
    }
    p.lab[0] = fmaf(116.0f, f[1], -16.0f);
    p.lab[1] = 500.0f * (f[0] - f[1]);
    p.lab[2] = 200.0f * (f[1] - f[2]);
    return p;
}

// gradient w.r.t. x of <gLab, Lab(x)>
__device__ __forceinline__ void back(const PixelLab &p, float gL, float ga, float gb, const Coeffs &co,
                                     float &g0, float &g1, float &g2)
{
    const float gfx = 500.0f * ga;
    const float gfy = fmaf(116.0f, gL, fmaf(-500.0f, ga, 200.0f * gb));
    const float gfz = -200.0f * gb;
    const float gt0 = gfx * p.df[0], gt1 = gfy * p.df[1], gt2 = gfz * p.df[2];
    g0 = fmaf(co.m[0], gt0, fmaf(co.m[3], gt1, co.m[6] * gt2));
    g1 = fmaf(co.m[1], gt0, fmaf(co.m[4], gt1, co.m[7] * gt2));
    g2 = fmaf(co.m[2], gt0, fmaf(co.m[5], gt1, co.m[8] * gt2));
}

// Work split: quads of 4 consecutive pixels of one image plane when
// hw % 4 == 0 and the pointers are 16-byte aligned (16-byte loads and
// stores); single pixels otherwise.  Index math is 32-bit: the entry points
// admit at most 2^31 pixels, so a grid-stride index never wraps.
struct Geometry {
    int64_t hw;
    uint32_t per_img;     // work items per image (quads or pixels)
    uint32_t items;       // total work items
};

template <bool VEC>
__device__ __forceinline__ int64_t item_base(const Geometry &g, uint32_t u)
{
    const uint32_t b = u / g.per_img, i = u - b * g.per_img;
    return (int64_t)b * 3 * g.hw + (VEC ? 4 * (int64_t)i : (int64_t)i);
}

template <bool VEC>
__device__ __forceinline__ void load_item(const float *p, int64_t o, float (&v)[4])
{
    if (VEC) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p + o));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        v[0] = __ldcs(p + o);
    }
}

template <bool VEC>
__device__ __forceinline__ void store_item(float *p, int64_t o, const float (&v)[4])
{
    if (VEC) __stcs(reinterpret_cast<float4 *>(p + o), make_float4(v[0], v[1], v[2], v[3]));
    else __stcs(p + o, v[0]);
}

template <int FORM, bool VEC>
__global__ void __launch_bounds__(kGradThreads)
k_lab_forward(const float *__restrict__ x, Geometry g, float *__restrict__ lab, const __grid_constant__ Coeffs co)
{
    constexpr int W = VEC ? 4 : 1;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.items; u += gridDim.x * blockDim.x) {
        const int64_t o = item_base<VEC>(g, u);
        float x0[4], x1[4], x2[4], l0[4], l1[4], l2[4];
        load_item<VEC>(x, o, x0);
        load_item<VEC>(x, o + g.hw, x1);
        load_item<VEC>(x, o + 2 * g.hw, x2);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const PixelLab p = lab_of<FORM>(x0[j], x1[j], x2[j], co);
            l0[j] = p.lab[0]; l1[j] = p.lab[1]; l2[j] = p.lab[2];
        }
        store_item<VEC>(lab, o, l0);
        store_item<VEC>(lab, o + g.hw, l1);
        store_item<VEC>(lab, o + 2 * g.hw, l2);
    }
}

template <int FORM, bool VEC>
__global__ void __launch_bounds__(kGradThreads)
k_lab_backward(const float *__restrict__ x, const float *__restrict__ glab, Geometry g, float *__restrict__ gx,
               const __grid_constant__ Coeffs co)
{
    constexpr int W = VEC ? 4 : 1;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.items; u += gridDim.x * blockDim.x) {
        const int64_t o = item_base<VEC>(g, u);
        float x0[4], x1[4], x2[4], a0[4], a1[4], a2[4];
        load_item<VEC>(x, o, x0);
        load_item<VEC>(x, o + g.hw, x1);
        load_item<VEC>(x, o + 2 * g.hw, x2);
        load_item<VEC>(glab, o, a0);
        load_item<VEC>(glab, o + g.hw, a1);
        load_item<VEC>(glab, o + 2 * g.hw, a2);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const PixelLab p = lab_of<FORM>(x0[j], x1[j], x2[j], co);
            back(p, a0[j], a1[j], a2[j], co, x0[j], x1[j], x2[j]);
        }
        store_item<VEC>(gx, o, x0);
        store_item<VEC>(gx, o + g.hw, x1);
        store_item<VEC>(gx, o + 2 * g.hw, x2);
    }
}

template <int FORM, bool GRAD, bool VEC>
__global__ void __launch_bounds__(kGradThreads)
k_lab_delta_e(const float *__restrict__ x, const float *__restrict__ tgt, Geometry g, float inv_npix,
              float *__restrict__ gx, double *__restrict__ partial, const __grid_constant__ Coeffs co)
{
    constexpr int W = VEC ? 4 : 1;
    double acc = 0.0;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < g.items; u += gridDim.x * blockDim.x) {
        const int64_t o = item_base<VEC>(g, u);
        float x0[4], x1[4], x2[4], t0[4], t1[4], t2[4];
        load_item<VEC>(x, o, x0);
        load_item<VEC>(x, o + g.hw, x1);
        load_item<VEC>(x, o + 2 * g.hw, x2);
        load_item<VEC>(tgt, o, t0);
        load_item<VEC>(tgt, o + g.hw, t1);
        load_item<VEC>(tgt, o + 2 * g.hw, t2);
        float sum = 0.0f;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const PixelLab p = lab_of<FORM>(x0[j], x1[j], x2[j], co);
            const float dl = p.lab[0] - t0[j], da = p.lab[1] - t1[j], db = p.lab[2] - t2[j];
            const float de = sqrtf(fmaf(dl, dl, fmaf(da, da, db * db)));
            sum += de;
            if (GRAD) {
                const float sc = de > 0.0f ? inv_npix / de : 0.0f;
                back(p, dl * sc, da * sc, db * sc, co, x0[j], x1[j], x2[j]);
            }
        }
        acc += (double)sum;
        if (GRAD) {
            store_item<VEC>(gx, o, x0);
            store_item<VEC>(gx, o + g.hw, x1);
            store_item<VEC>(gx, o + 2 * g.hw, x2);
        }
    }
    // block reduction in a fixed order
    __shared__ double red[kGradThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = kGradThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double *__restrict__ partial, int n, double scale, float *__restrict__ out)
{
    __shared__ double red[kGradThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += partial[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int st = kGradThreads / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(red[0] * scale);
}

// One wave of the kernel's resident CTAs (grid-stride loops inside): a grid
// larger than what fits leaves a second, partly empty wave.  occ <= 8, so the
// grid never exceeds the num_sms * 8 loss partials.
static int grad_grid(const mact_ctx &h, uint32_t items, int occ)
{
    const int64_t g = ((int64_t)items + kGradThreads - 1) / kGradThreads;
    const int64_t cap = (int64_t)h.num_sms * (occ < 8 ? occ : 8);
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

// resident CTAs per SM of one kernel instantiation (thread-safe one-time init)
template <class K>
static int occupancy(K kern)
{
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kGradThreads, 0);
    return (e != cudaSuccess || o <= 0) ? 1 : o;
}

template <int FORM, bool VEC>
static int occ_forward()
{
    static const int o = occupancy(k_lab_forward<FORM, VEC>);
    return o;
}

template <int FORM, bool VEC>
static int occ_backward()
{
    static const int o = occupancy(k_lab_backward<FORM, VEC>);
    return o;
}

template <int FORM, bool GRAD, bool VEC>
static int occ_delta_e()
{
    static const int o = occupancy(k_lab_delta_e<FORM, GRAD, VEC>);
    return o;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Work geometry; VEC when every pointer given is 16-byte aligned and hw % 4 == 0.
static Geometry geometry(int64_t nb, int64_t hw, bool vec)
{
    Geometry g;
    g.hw = hw;
    g.per_img = (uint32_t)(vec ? hw / 4 : hw);
    g.items = (uint32_t)(nb * (int64_t)g.per_img);
    return g;
}

static bool use_vec(int64_t hw, std::initializer_list<const void *> ptrs)
{
    if (hw % 4 != 0) return false;
    for (const void *p : ptrs)
        if (p && !aligned16(p)) return false;
    return true;
}

// 0: exact cube root; 4 or 6: the rational's chain degree (the polynomial
// cube root is refused by the entry points before launch)
static int grad_form(const mact_ctx &h) { return h.cfg.exact ? 0 : h.co.lab_deg; }

cudaError_t launch_lab_forward(const mact_ctx &h, const float *x, int64_t nb, int64_t hw, float *lab, cudaStream_t s)
{
    const bool v = use_vec(hw, {x, lab});
    const Geometry g = geometry(nb, hw, v);
#define MACT_FWD(F, V) \
    k_lab_forward<F, V><<<grad_grid(h, g.items, occ_forward<F, V>()), kGradThreads, 0, s>>>(x, g, lab, h.co)
    switch (grad_form(h)) {
    case 0:
        if (v) MACT_FWD(0, true);
        else MACT_FWD(0, false);
        break;
    case 6:
        if (v) MACT_FWD(6, true);
        else MACT_FWD(6, false);
        break;
    default:
        if (v) MACT_FWD(4, true);
        else MACT_FWD(4, false);
    }
#undef MACT_FWD
    return cudaGetLastError();
}

cudaError_t launch_lab_backward(const mact_ctx &h, const float *x, const float *glab, int64_t nb, int64_t hw,
                                float *gx, cudaStream_t s)
{
    const bool v = use_vec(hw, {x, glab, gx});
    const Geometry g = geometry(nb, hw, v);
#define MACT_BWD(F, V) \
    k_lab_backward<F, V><<<grad_grid(h, g.items, occ_backward<F, V>()), kGradThreads, 0, s>>>(x, glab, g, gx, h.co)
    switch (grad_form(h)) {
    case 0:
        if (v) MACT_BWD(0, true);
        else MACT_BWD(0, false);
        break;
    case 6:
        if (v) MACT_BWD(6, true);
        else MACT_BWD(6, false);
        break;
    default:
        if (v) MACT_BWD(4, true);
        else MACT_BWD(4, false);
    }
#undef MACT_BWD
    return cudaGetLastError();
}

// returns the grid it launched (the number of loss partials written)
template <int FORM>
static int delta_e_launch(const mact_ctx &h, bool grad, bool v, cudaStream_t s, const float *x, const float *tgt,
                          const Geometry &g, float inv, float *gx, double *partial, const Coeffs &co)
{
    int grid;
#define MACT_DE(G, V)                                                                          \
    grid = grad_grid(h, g.items, occ_delta_e<FORM, G, V>());                                   \
    k_lab_delta_e<FORM, G, V><<<grid, kGradThreads, 0, s>>>(x, tgt, g, inv, gx, partial, co)
    if (grad && v) { MACT_DE(true, true); }
    else if (grad) { MACT_DE(true, false); }
    else if (v) { MACT_DE(false, true); }
    else { MACT_DE(false, false); }
#undef MACT_DE
    return grid;
}

cudaError_t launch_lab_delta_e(const mact_ctx &h, const float *x, const float *tgt, int64_t nb, int64_t hw,
                               float *loss, float *gx, double *partial, cudaStream_t s)
{
    // partial holds num_sms * 8 entries, the largest grid grad_grid returns
    const bool v = use_vec(hw, {x, tgt, gx});
    const Geometry g = geometry(nb, hw, v);
    const float inv = (float)(1.0 / (double)(nb * hw));
    int grid;
    switch (grad_form(h)) {
    case 0: grid = delta_e_launch<0>(h, gx != nullptr, v, s, x, tgt, g, inv, gx, partial, h.co); break;
    case 6: grid = delta_e_launch<6>(h, gx != nullptr, v, s, x, tgt, g, inv, gx, partial, h.co); break;
    default: grid = delta_e_launch<4>(h, gx != nullptr, v, s, x, tgt, g, inv, gx, partial, h.co);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<1, kGradThreads, 0, s>>>(partial, grid, 1.0 / (double)(nb * hw), loss);
    return cudaGetLastError();
}

}  // namespace mact
