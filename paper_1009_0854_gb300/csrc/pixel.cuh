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
// library's fits up to (6, 6); higher coefficients are zero).  The two
// chains run together on one packed FP32 pair (lane x: d, lane y: q), one
// f32x2 FMA per degree; each lane rounds exactly like the scalar fmaf chain.
// NR: refine the reciprocal with a Newton step (FP32 planes); FP16 planes
// round far more coarsely than the step's correction, so they skip it.
template <int DEG, bool NR = true>
__device__ __forceinline__ float f_mact(float t, const Coeffs &co)
{
    const float2 tt = make_float2(t, t);
    float2 s;
    if constexpr (NR) {
        s = make_float2(co.lab_d[DEG], co.lab_q[DEG]);
#pragma unroll
        for (int i = DEG - 1; i >= 0; --i) s = fma2(s, tt, make_float2(co.lab_d[i], co.lab_q[i]));
    } else {   // FP16 planes: the coefficient pairs stored as pairs
        s = co.lab_dqp[DEG];
#pragma unroll
        for (int i = DEG - 1; i >= 0; --i) s = fma2(s, tt, co.lab_dqp[i]);
    }
    float fa = fmaf(s.x, NR ? rcp_nr(s.y) : rcp_approx(s.y), 1.0f);
    float fl = fmaf(kLinSlope, t, kLinOffset);
    return t > kKnee ? fa : fl;
}

// The same for the X and Y channels at once, t = (tx, ty): lanes are
// channels here (chains (dx, dy) and (qx, qy) with broadcast coefficients,
// the reciprocal's Newton step and the two branches as pairs), each lane
// rounded exactly as f_mact's scalar operations.
template <int DEG, bool NR = true>
__device__ __forceinline__ float2 f_mact_xy(float2 t, const Coeffs &co)
{
    float2 d = make_float2(co.lab_d[DEG], co.lab_d[DEG]);
    float2 q = make_float2(co.lab_q[DEG], co.lab_q[DEG]);
#pragma unroll
    for (int i = DEG - 1; i >= 0; --i) {
        d = fma2(d, t, make_float2(co.lab_d[i], co.lab_d[i]));
        q = fma2(q, t, make_float2(co.lab_q[i], co.lab_q[i]));
    }
    float2 r = make_float2(rcp_approx(q.x), rcp_approx(q.y));
    const float2 one = make_float2(1.0f, 1.0f);
    if (NR) r = fma2(r, fma2(make_float2(-q.x, -q.y), r, one), r);   // r + r (1 - q r)
    const float2 fa = fma2(d, r, one);
    const float2 fl = fma2(make_float2(kLinSlope, kLinSlope), t, make_float2(kLinOffset, kLinOffset));
    return make_float2(t.x > kKnee ? fa.x : fl.x, t.y > kKnee ? fa.y : fl.y);
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

// Rows 0 and 1 of the white-divided matrix times the linearised code as one
// FP32 pair; NR = false (FP16 planes) takes each coefficient pair as one
// stored 8-byte operand.
template <bool NR>
__device__ __forceinline__ float2 rows01(const Coeffs &co, float k0, float k1, float k2)
{
    if constexpr (NR)
        return fma2(make_float2(co.m[2], co.m[5]), make_float2(k2, k2),
                    fma2(make_float2(co.m[1], co.m[4]), make_float2(k1, k1),
                         mul2(make_float2(co.m[0], co.m[3]), make_float2(k0, k0))));
    else
        return fma2(co.mp[2], make_float2(k2, k2), fma2(co.mp[1], make_float2(k1, k1), mul2(co.mp[0], make_float2(k0, k0))));
}

// RDEG: 0 = the FP64 cube-root polynomial; 4 or 6 = the rational with
// chains of that degree (ignored when EXACT).  NR: Newton step on the
// rational's reciprocal (off for FP16 planes).  The X and Y rows of the
// matrix and a* and b* run as packed FP32 pairs, and so does the cube-root
// rational: for FP32 planes each channel's (d, q) chains (66 instructions
// per pixel, 75 registers; the kernel is HBM-bound there, and this form
// measured 3% faster on a 16384^2 image), for FP16 planes the X and Y
// channels together (f_mact_xy), with the matrix and Z-chain coefficient
// pairs read as stored 8-byte pairs (52 instructions per pixel; issue-bound).
// Stored pairs for FP32 planes cut them to 60 instructions per pixel but
// measured 2-4% slower on a 16384^2 image.  All forms are bit-identical to
// the scalar ones.
template <bool EXACT, int RDEG, bool NR = true>
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
        // (tx, ty) = rows 0 and 1 of the matrix, tz = row 2
        const float2 txy = rows01<NR>(co, k0, k1, k2);
        float tz = fmaf(co.m[8], k2, fmaf(co.m[7], k1, co.m[6] * k0));
        float fx, fy, fz;
        if (EXACT) {
            fx = f_exact(txy.x); fy = f_exact(txy.y); fz = f_exact(tz);
        } else {
            constexpr int D = RDEG == 0 ? 4 : RDEG;   // (RDEG 0 returned above)
            if (NR) {   // FP32 planes: each channel's d and q chains as one pair
                fx = f_mact<D, NR>(txy.x, co); fy = f_mact<D, NR>(txy.y, co);
            } else {    // FP16 planes: the X and Y channels as pairs
                const float2 fxy = f_mact_xy<D, NR>(txy, co);
                fx = fxy.x; fy = fxy.y;
            }
            fz = f_mact<D, NR>(tz, co);
        }
        o0 = fmaf(116.0f, fy, -16.0f);
        const float2 ab = mul2(make_float2(500.0f, 200.0f), sub2(make_float2(fx, fy), make_float2(fy, fz)));
        o1 = ab.x;
        o2 = ab.y;
        return 0;
    }
};

// ------------------------------------------------------------------ CIELUV
// CIE 1976 L*u*v*, the variant the Conclusions name: L* exactly as in CIELAB
// (the same cube-root approximant, or cbrtf when EXACT), and on the
// white-normalised t the chromaticity terms u' - u'n = 4 Xn tx / D - u'n and
// v' - v'n = 9 Yn ty / D - v'n with D = Xn tx + 15 Yn ty + 3 Zn tz;
// u* = 13 L* (u' - u'n), v* = 13 L* (v' - v'n).  Black (D = 0) gives
// u* = v* = 0.  FP32 form: with dn = Xn + 15 Yn + 3 Zn, identically
//   u' - u'n = 4 Xn (15 Yn (tx - ty) + 3 Zn (tx - tz)) / (dn D),
//   v' - v'n = 9 Yn (Xn (ty - tx) + 3 Zn (ty - tz)) / (dn D),
// which has no cancellation near the neutral axis (the differences of t are
// small there and exact), like the 1 + d/q form of the cube root.  The
// quotient uses the refined reciprocal; the u and v terms run as packed FP32
// pairs.  RDEG 0 (the FP64 cube-root polynomial) runs in FP64, direct form.
template <bool EXACT, int RDEG, bool NR = true>
struct OpCieluv {
    const float *gam;   // 256-entry linearisation table in shared memory
    const Coeffs &co;
    __device__ __forceinline__ int operator()(uint32_t r, uint32_t g, uint32_t b, float &o0, float &o1,
                                              float &o2) const
    {
        if (!EXACT && RDEG == 0) {
            const double *g64 = reinterpret_cast<const double *>(gam);
            const double k0 = g64[r], k1 = g64[g], k2 = g64[b];
            const double *m = co.m64;
            const double tx = fma(m[2], k2, fma(m[1], k1, m[0] * k0));
            const double ty = fma(m[5], k2, fma(m[4], k1, m[3] * k0));
            const double tz = fma(m[8], k2, fma(m[7], k1, m[6] * k0));
            const double L = 116.0 * f_mact_poly64(ty, co) - 16.0;
            const double D = co.luv_den64[0] * tx + co.luv_den64[1] * ty + co.luv_den64[2] * tz;
            o0 = D > 0.0 ? (float)L : 0.0f;
            o1 = D > 0.0 ? (float)(13.0 * L * (co.luv_u64 * tx / D - co.luv_un64)) : 0.0f;
            o2 = D > 0.0 ? (float)(13.0 * L * (co.luv_v64 * ty / D - co.luv_vn64)) : 0.0f;
            return 0;
        }
        float k0 = gam[r], k1 = gam[g], k2 = gam[b];
        const float2 txy = rows01<NR>(co, k0, k1, k2);
        float tz = fmaf(co.m[8], k2, fmaf(co.m[7], k1, co.m[6] * k0));
        float fy;
        if (EXACT) {
            fy = f_exact(txy.y);
        } else {
            constexpr int D = RDEG == 0 ? 4 : RDEG;
            fy = f_mact<D, NR>(txy.y, co);
        }
        const float L = fmaf(116.0f, fy, -16.0f);
        const float den = fmaf(co.luv_den[2], tz, fmaf(co.luv_den[1], txy.y, co.luv_den[0] * txy.x));
        const float rd = den > 0.0f ? rcp_nr(den) : 0.0f;
        // (u' - u'n, v' - v'n) in the difference form, then times 13 L*
        const float2 d1 = sub2(txy, make_float2(txy.y, txy.x));     // (tx - ty, ty - tx)
        const float2 d2 = sub2(txy, make_float2(tz, tz));           // (tx - tz, ty - tz)
        const float2 num = fma2(make_float2(co.luv_c[0], co.luv_c[1]), d1,
                                mul2(make_float2(co.luv_c[2], co.luv_c[3]), d2));
        const float2 uv = mul2(num, make_float2(rd, rd));
        const float l13 = 13.0f * L;
        const float2 o = mul2(make_float2(l13, l13), uv);
        o0 = den > 0.0f ? L : 0.0f;      // black: exactly (0, 0, 0)
        o1 = den > 0.0f ? o.x : 0.0f;
        o2 = den > 0.0f ? o.y : 0.0f;
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
