// pixel.cuh -- per-pixel transforms of MACT, FP32.
//
// Each operator maps one 8-bit R'G'B' triplet to three outputs.  The
// approximant operators follow the paper's formulas; where the FP32 form
// differs from the literal formula it is an algebraically identical
// rewrite chosen for rounding behaviour, stated at the site.
#pragma once

#include "common.cuh"

namespace mact {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kKnee = 0.008856f;             // Eq. equ_xyz_lab branch point
constexpr float kLinSlope = 7.787f;            // linear segment of f(t)
constexpr float kLinOffset = 16.0f / 116.0f;

// ------------------------------------------------------------------ CIELAB
// Eq. equ_rgb_lin (table lookup, as the paper suggests), Eq. equ_rgb_xyz with
// the rows pre-divided by the white point, Eq. equ_xyz_lab with the cube root
// replaced by the minimax rational of Table tab_cbrt_rat.  The
// linearisation table holds FP32 entries, or FP64 entries for the polynomial
// (lab_m = 0) variant.
//
// FP32 form of the rational: f = 1 + d(t)/q(t) with d = p - q.  Identical to
// p/q in exact arithmetic; near t = 1, where f ~ 1 and a*, b* amplify
// absolute errors by 500 and 200, d is small and its rounding error scales
// with it, so the worst a* error over the 2^24 colours drops from ~2.2e-4
// (p/q) to ~1.2e-4.
// DEG: Horner degree of both chains (4 for the printed rationals, 6 for the
// library's fits up to (6, 6); higher coefficients are zero).
template <int DEG>
__device__ __forceinline__ float f_mact(float t, const Coeffs &co)
{
    float d = horner<DEG>(co.lab_d, t);
    float q = horner<DEG>(co.lab_q, t);
    float fa = fmaf(d, rcp_nr(q), 1.0f);
    float fl = fmaf(kLinSlope, t, kLinOffset);
    return t > kKnee ? fa : fl;
}

// The cube-root polynomials of Table tab_cbrt_poly (lab_m = 0) have slopes up
// to ~4.4 at t = 1 (t^(1/3) has 1/3), so the FP32 rounding of t alone moves
// a* by more than 2e-4.  That option (which the paper rejects for its error)
// is evaluated in FP64: t from an FP64 linearisation table and matrix, then
// the polynomial.
__device__ __forceinline__ double f_mact_poly64(double t, const Coeffs &co)
{
    double s = co.lab_p64[5];
#pragma unroll
    for (int i = 4; i >= 0; --i) s = fma(s, t, co.lab_p64[i]);
    return t > 0.008856 ? s : 7.787 * t + 16.0 / 116.0;
}

__device__ __forceinline__ float f_exact(float t)
{
    float fl = fmaf(kLinSlope, t, kLinOffset);
    return t > kKnee ? cbrtf(t) : fl;
}

// RDEG: 0 = the FP64 cube-root polynomial; 4 or 6 = the rational with
// chains of that degree (ignored when EXACT).
template <bool EXACT, int RDEG>
struct OpCielab {
    const float *gam;   // 256-entry linearisation table in shared memory
    const Coeffs &co;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        if (!EXACT && RDEG == 0) {
            const double *g64 = reinterpret_cast<const double *>(gam);
            const double k0 = g64[r], k1 = g64[g], k2 = g64[b];
            const double *m = co.m64;
            const double fx = f_mact_poly64(fma(m[2], k2, fma(m[1], k1, m[0] * k0)), co);
            const double fy = f_mact_poly64(fma(m[5], k2, fma(m[4], k1, m[3] * k0)), co);
            const double fz = f_mact_poly64(fma(m[8], k2, fma(m[7], k1, m[6] * k0)), co);
            o0 = (float)(116.0 * fy - 16.0);
            o1 = (float)(500.0 * (fx - fy));
            o2 = (float)(200.0 * (fy - fz));
            return 0;
        }
        float k0 = gam[r], k1 = gam[g], k2 = gam[b];
        float tx = fmaf(co.m[2], k2, fmaf(co.m[1], k1, co.m[0] * k0));
        float ty = fmaf(co.m[5], k2, fmaf(co.m[4], k1, co.m[3] * k0));
        float tz = fmaf(co.m[8], k2, fmaf(co.m[7], k1, co.m[6] * k0));
        float fx, fy, fz;
        if (EXACT) {
            fx = f_exact(tx); fy = f_exact(ty); fz = f_exact(tz);
        } else {
            constexpr int D = RDEG == 0 ? 4 : RDEG;   // (RDEG 0 returned above)
            fx = f_mact<D>(tx, co); fy = f_mact<D>(ty, co); fz = f_mact<D>(tz, co);
        }
        o0 = fmaf(116.0f, fy, -16.0f);
        o1 = 500.0f * (fx - fy);
        o2 = 200.0f * (fy - fz);
        return 0;
    }
};

// --------------------------------------------------------------------- HSI
// Kender's case chain (Eq. equ_rgb_kender) on integer codes, in the printed
// order with strict comparisons.  Approximant: arctan(sqrt(3) x) ->
// sgn(x) P_n(|x|) (Table tab_arctan, odd symmetry).  Exact: atanf.
// The "R > B" case and grays (hue undefined) give H = 0.
template <bool EXACT>
struct OpHsi {
    const Coeffs &co;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        int R = (int)r, G = (int)g, B = (int)b;
        int num, den;
        float base;
        bool zero = false;
        if (R > B && G > B) { num = G - R; den = G - B + R - B; base = kPi / 3.0f; }
        else if (G > R)     { num = B - G; den = B - R + G - R; base = kPi; }
        else if (B > G)     { num = R - B; den = R - G + B - G; base = 5.0f * kPi / 3.0f; }
        else                { num = 0; den = 1; base = 0.0f; zero = true; }
        float x = div_approx((float)num, (float)den);
        float h;
        if (EXACT) {
            h = base + atanf(1.7320508075688772f * x);
        } else {
            float v = horner<5>(co.hsi, fabsf(x));
            h = base + (x < 0.0f ? -v : v);
        }
        o0 = zero ? 0.0f : h;
        int sum = R + G + B;
        int mn = min(R, min(G, B));
        // S = 1 - 3 min / sum, formed as (sum - 3 min) / sum: the numerator is
        // an exact integer, so grays give exactly 0
        o1 = sum > 0 ? div_approx((float)(sum - 3 * mn), (float)sum) : 0.0f;
        o2 = (float)sum * (1.0f / 765.0f);
        return 0;
    }
};

// --------------------------------------------------------------------- SCT
// Eq. equ_rgb_sct with Eq. equ_sct_b.  Angle A: x = B/L; if x >= 0.5 the
// arcsin form (Eq. equ_arccos_cheap) with y = sqrt(1 - x), else the arccos
// polynomial.  The test x >= 0.5 is taken exactly on integers
// (2B >= L  <=>  3 B^2 >= R^2 + G^2), and 1 - x is formed as
// (R^2 + G^2) / (L (L + B)), which avoids the cancellation of 1 - B/L when
// B ~ L (exactly equal in real arithmetic).  Angle B (Eq. arctan_split):
// f(G/R) if G < R, else g(R/G); R = 0 < G gives pi/2, R = G = 0 gives 0.
// Exact form: atan2f for both angles (well conditioned at every pixel).
template <bool EXACT>
struct OpSct {
    const Coeffs &co;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        int R = (int)r, G = (int)g, B = (int)b;
        int rg2 = R * R + G * G;
        int s2 = rg2 + B * B;
        float L = sqrtf((float)s2);
        float A, Bang;
        if (EXACT) {
            A = atan2f(sqrtf((float)rg2), (float)B);
            Bang = atan2f((float)G, (float)R);
        } else {
            // branch-free: hardware rsqrt / sqrt / rcp approximations (a few
            // ulp, far inside the 1e-5 tolerance) and selects
            const float s2f = (float)max(s2, 1);
            const float rl = rsqrt_approx(s2f);          // 1/L
            L = s2f * rl;
            const bool arcs = 3 * B * B >= rg2;          // B/L >= 0.5, exactly
            const float x = (float)B * rl;
            const float y = sqrt_approx((float)rg2 * rcp_approx(L * (L + (float)B)));
            const float pa = horner<5>(co.sct_p, y);
            const float qa = horner<5>(co.sct_q, x);
            A = arcs ? pa : qa;
            const bool useF = G < R;
            const int nn = useF ? G : R, dd = useF ? R : G;
            const float w = (float)nn * rcp_approx((float)max(dd, 1));
            float c[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) c[i] = useF ? co.sct_f[i] : co.sct_g[i];
            Bang = horner<5>(c, w);
            Bang = (R == 0) ? ((G > 0) ? kPi / 2.0f : 0.0f) : Bang;
            L = (s2 == 0) ? 0.0f : L;
        }
        if (s2 == 0) { A = 0.0f; Bang = 0.0f; }
        o0 = L;
        o1 = A;
        o2 = Bang;
        return 0;
    }
};

}  // namespace mact
