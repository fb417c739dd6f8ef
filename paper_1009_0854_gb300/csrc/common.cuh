// common.cuh -- internal types and device helpers shared by the libmact
// kernels.  Nothing here is exported; the public interface is include/mact.h.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mact.h"

namespace mact {

// Streaming engine geometry: 256 threads per CTA, 4 pixels per thread per
// sub-block, 4 sub-blocks per tile -> 4096 pixels (12 KB of input) per tile.
constexpr int kThreads = 256;
constexpr int kPxPerThread = 4;
constexpr int kTile = kThreads * kPxPerThread * 4;

// Coefficients travel by value in the kernel parameter block, so every
// uniform coefficient is a constant-bank operand of its FFMA.  Arrays are
// ascending powers, zero-padded to the fixed evaluation degree (padding with
// leading zeros leaves every Horner step bit-identical).
struct Coeffs {
    double m64[9];       // rgb_to_xyz / white in FP64 (polynomial cube-root path)
    double lab_p64[6];   // polynomial cube root in FP64, degree 5 (zero-padded)
    float m[9];          // rgb_to_xyz row c divided by white[c]
    float lab_d[8];      // rational: p - q (degree <= 6); polynomial: p (degree 5); zero-padded
    float lab_q[8];      // rational: q (degree <= 6)
    float lab_dd[7];     // rational: d' = (p - q)' (degree <= 5)
    float lab_dq[7];     // rational: q' (degree <= 5)
    int32_t lab_rational;
    int32_t lab_deg;     // Horner degree of the rational's chains: 4 (n, m <= 4) or 6
    float hsi[6];        // arctan(sqrt(3) x) on |x| <= 1, degree 5
    float sct_p[6];      // 2 arcsin(y/sqrt 2), y = sqrt(1 - B/L), degree 5
    float sct_q[6];      // arccos(x) on [0, 0.5], degree 5
    float sct_f[6];      // arctan(x) on [0, 254/255], degree 5
    float sct_g[6];      // pi/2 - arctan(w) on [1/255, 1], degree 5
    // CIELUV on white-normalised t = (X/Xn, Y/Yn, Z/Zn): denominator
    // weights (Xn, 15 Yn, 3 Zn) and, with dn = Xn + 15 Yn + 3 Zn, the
    // difference-form weights (4 Xn 15 Yn, 9 Yn Xn, 4 Xn 3 Zn, 9 Yn 3 Zn) / dn;
    // FP64 numerators 4 Xn, 9 Yn and the white's u'n, v'n for the
    // polynomial cube-root path
    float luv_den[3];
    float luv_c[4];
    double luv_den64[3];
    double luv_u64, luv_v64, luv_un64, luv_vn64;
    // pairs for the packed FP32 instructions of the FP16-plane kernels, each
    // one 8-byte operand: (lab_d[i], lab_q[i]) and column j of matrix rows 0
    // and 1, (m[j], m[3 + j])
    float2 lab_dqp[8];
    float2 mp[3];
};

// One image (or a contiguous run treated as one row) for the tile engine.
struct ImageDesc {
    const uint8_t *rgb;
    void *out[3];
    int64_t width;        // pixels per row (the whole image if contiguous)
    int64_t height;       // rows
    int64_t pitch;        // input row pitch in bytes
    int64_t opitch;       // output row pitch in elements
    int64_t tiles_per_row;
    int64_t tile_begin;   // prefix sum of tiles over a batch
    int32_t space;
    int32_t dtype;
};

// A short work list carried in a kernel's parameter block (with the Coeffs
// block it stays under the 4 KB classic parameter limit).
constexpr int kParamImages = 32;
struct ParamList {
    ImageDesc img[kParamImages];
};
static_assert(sizeof(ParamList) + sizeof(Coeffs) + 64 <= 4096, "kernel parameters exceed 4 KB");

// Horner evaluation a0 + x (a1 + x (a2 + ...)) with FMA, degree D.
template <int D>
__device__ __forceinline__ float horner(const float *a, float x)
{
    float s = a[D];
#pragma unroll
    for (int i = D - 1; i >= 0; --i) s = fmaf(s, x, a[i]);
    return s;
}

// Reciprocal: hardware approximation (rcp.approx.ftz.f32) refined by one
// Newton-Raphson step r' = r + r (1 - q r) (the classical iteration for 1/q,
// quadratic convergence).  Used only on arguments in [4e-4, 4].
__device__ __forceinline__ float rcp_nr(float q)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
    float e = fmaf(-q, r, 1.0f);
    return fmaf(r, e, r);
}

// Fast quotient a / b via rcp.approx (about 2 ulp); used where the tolerance
// allows it (HSI hue argument, saturation; SCT ratios).
__device__ __forceinline__ float rcp_approx(float b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    return r;
}
__device__ __forceinline__ float div_approx(float a, float b) { return a * rcp_approx(b); }

// Hardware reciprocal square root and square root approximations
// (rsqrt.approx / sqrt.approx, a few ulp): no special-case branches.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (the sm_100-family f32x2 instructions, through CUDA's
// __ffma2_rn / __fadd2_rn / __fmul2_rn): one instruction computes both lanes,
// each rounded to nearest exactly as the scalar fmaf, a + b, a - b or a * b
// would be, so results are bit-identical to the scalar forms while the
// instruction count halves.  (Measured against the same operations written as
// inline PTX: the intrinsics left the compiler more freedom and gave 3% more
// on FP16 MACT CIELAB planes.)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Streaming (evict-first) stores of 4 consecutive results.
__device__ __forceinline__ void store4(float *p, float a, float b, float c, float d)
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(a, b, c, d));
}
__device__ __forceinline__ void store4(__half *p, float a, float b, float c, float d)
{
    __half2 lo = __floats2half2_rn(a, b);
    __half2 hi = __floats2half2_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t *>(&lo);
    v.y = *reinterpret_cast<uint32_t *>(&hi);
    __stcs(reinterpret_cast<uint2 *>(p), v);
}
__device__ __forceinline__ void store1(float *p, float a) { __stcs(p, a); }
__device__ __forceinline__ void store1(__half *p, float a) { *p = __float2half_rn(a); }

}  // namespace mact
