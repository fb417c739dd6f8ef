/*
 * mact_oracle.c -- plain FP64 CPU oracle for the MACT per-pixel transforms.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this library.  It shares no code,
 * header or table with the CUDA library; it is the slow, obviously correct
 * statement of what the paper computes, against which the kernels are checked.
 *
 * Everything is double precision, one pixel at a time, in the order the paper
 * writes the formulas.  Polynomials are evaluated as the plain sum
 * a0 + a1 x + a2 x^2 + ... (no Horner restructuring, no fusion).  The only
 * concession to speed is an OpenMP "parallel for" over independent pixels
 * (and a reduction for the error statistics), which changes no per-pixel
 * arithmetic.
 *
 * Readings of the paper taken here (each one is pinned by a test):
 *  - CIELAB, HSI and SCT take 8-bit codes.  CIELAB linearises k' = code/255
 *    with the BT.709 inverse gamma (Eq. equ_rgb_lin); HSI and SCT work on the
 *    gamma-encoded codes directly.
 *  - f(t) uses the approximant only for t > 0.008856 (Eq. equ_xyz_lab); the
 *    linear segment 7.787 t + 16/116 is kept exactly.  No clamp of t to 1.
 *  - CIELUV (named in the Conclusions, defined by the CIE, not printed):
 *    L* as in CIELAB, u* = 13 L* (u' - u'n), v* = 13 L* (v' - v'n); black
 *    gives u* = v* = 0.
 *  - HSI hue: Kender's case chain (Eq. equ_rgb_kender) evaluated in the
 *    printed order with strict comparisons; hue 0 when max-min (chroma) is 0
 *    (the "undefined" case); S = 0 for black.
 *  - SCT: x = B/L; arcsin form when x >= 0.5 (Eq. equ_arccos_stable /
 *    equ_arccos_cheap), arccos polynomial otherwise; angle B uses f(G/R)
 *    when G < R and g(R/G) otherwise (Eq. arctan_split); R=0,G>0 gives pi/2;
 *    R=G=0 gives 0; black gives L = A = B = 0.
 *  - LUT nodes sit at k' = i/(N-1) on each axis (R outermost); the cell of a
 *    code v is idx = v(N-1) div 255 with remainder rem = v(N-1) mod 255,
 *    except v = 255 which uses idx = N-2, rem = 255.  Simplex choice compares
 *    the integer remainders.
 *
 * Parity unpinned: the HSI average cube error (orc_cube_eps_hsi; 1-3% from
 * the printed averages) and the angular HSI LUT's maximum cube error
 * (orc_cube_eps_hsi_lut).  Parity partial: the pyramidal LUT's average cube
 * error (within 0.07%; its maxima are exact).  Everything else is pinned.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* Source RGB definition: BT.709 inverse gamma parameters, the RGB->XYZ
 * matrix (row-major) and the reference white (Eq. equ_rgb_lin, equ_rgb_xyz
 * and the D65 white point of Section "Color Space Description"). */
typedef struct {
    double threshold, slope, offset, exponent;
    double m[9];
    double white[3];
} orc_rgbdef;

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------- helpers */

/* p(x) = a[0] + a[1] x + ... + a[n] x^n, written as the plain sum. */
static double orc_poly(const double *a, int n, double x)
{
    double s = 0.0, xp = 1.0;
    for (int i = 0; i <= n; ++i) {
        s += a[i] * xp;
        xp *= x;
    }
    return s;
}

static void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

ORC_API int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ CIELAB */

/* Eq. equ_rgb_lin: nonlinear k' in [0,1] -> linear k (BT.709). */
ORC_API double orc_gamma_inverse(const orc_rgbdef *d, double kp)
{
    if (kp < d->threshold) return kp / d->slope;
    return pow((kp + d->offset) / (1.0 + d->offset), d->exponent);
}

/* Eq. equ_rgb_xyz followed by the division by the reference white:
 * t = (X/X0, Y/Y0, Z/Z0) for 8-bit codes (r, g, b). */
ORC_API void orc_rgb_to_t(const orc_rgbdef *d, double r, double g, double b, double t[3])
{
    double k[3];
    k[0] = orc_gamma_inverse(d, r / 255.0);
    k[1] = orc_gamma_inverse(d, g / 255.0);
    k[2] = orc_gamma_inverse(d, b / 255.0);
    for (int c = 0; c < 3; ++c) {
        double xyz = d->m[3 * c + 0] * k[0] + d->m[3 * c + 1] * k[1] + d->m[3 * c + 2] * k[2];
        t[c] = xyz / d->white[c];
    }
}

/* Eq. equ_xyz_lab, exact f(t). */
static double orc_f_exact(double t)
{
    if (t > 0.008856) return cbrt(t);
    return 7.787 * t + 16.0 / 116.0;
}

/* f(t) with the cube root replaced by p_n(t)/q_m(t) (Tables tab_cbrt_rat,
 * tab_cbrt_poly; m < 0 means a polynomial, i.e. q = 1). */
static double orc_f_approx(double t, const double *p, int n, const double *q, int m)
{
    if (t > 0.008856) {
        double num = orc_poly(p, n, t);
        double den = (m >= 0) ? orc_poly(q, m, t) : 1.0;
        return num / den;
    }
    return 7.787 * t + 16.0 / 116.0;
}

/* L*, a*, b* from f values (Eq. equ_xyz_lab). */
static void orc_lab_from_f(double fx, double fy, double fz, double lab[3])
{
    lab[0] = 116.0 * fy - 16.0;
    lab[1] = 500.0 * (fx - fy);
    lab[2] = 200.0 * (fy - fz);
}

/* One pixel of RGB -> CIELAB.  mode 0: exact; mode 1: MACT approximant. */
ORC_API void orc_cielab_pixel(const orc_rgbdef *d, int mode,
                              const double *p, int n, const double *q, int m,
                              double r, double g, double b, double lab[3])
{
    double t[3], f[3];
    orc_rgb_to_t(d, r, g, b, t);
    for (int c = 0; c < 3; ++c)
        f[c] = mode ? orc_f_approx(t[c], p, n, q, m) : orc_f_exact(t[c]);
    orc_lab_from_f(f[0], f[1], f[2], lab);
}

ORC_API void orc_cielab(const orc_rgbdef *d, int mode,
                        const double *p, int n, const double *q, int m,
                        const uint8_t *rgb, int64_t npix,
                        double *L, double *A, double *B, int nthreads)
{
    orc_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npix; ++i) {
        double lab[3];
        orc_cielab_pixel(d, mode, p, n, q, m, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], lab);
        L[i] = lab[0];
        A[i] = lab[1];
        B[i] = lab[2];
    }
}

/* Eq. equ_cielab_dist. */
ORC_API double orc_delta_e(const double x[3], const double y[3])
{
    double dl = x[0] - y[0], da = x[1] - y[1], db = x[2] - y[2];
    return sqrt(dl * dl + da * da + db * db);
}

/* ------------------------------------------------------------------ CIELUV */
/* The paper's Conclusions note that the method carries over to CIELUV,
 * whose only costly step is the same cube root in L*.  CIE 1976 L*u*v*
 * (the standard definition, not printed in the paper):
 *   L* = 116 f(Y/Yn) - 16, with f the Eq. equ_xyz_lab function (exact, or the
 *        MACT approximant for t > 0.008856);
 *   u' = 4X / (X + 15Y + 3Z), v' = 9Y / (X + 15Y + 3Z), and u'n, v'n the same
 *        of the reference white;
 *   u* = 13 L* (u' - u'n), v* = 13 L* (v' - v'n).
 * Black (X + 15Y + 3Z = 0) has no chromaticity: u* = v* = 0 there.  XYZ are
 * the un-normalised tristimulus values t_c * white_c. */
ORC_API void orc_cieluv_pixel(const orc_rgbdef *d, int mode,
                              const double *p, int n, const double *q, int m,
                              double r, double g, double b, double luv[3])
{
    double t[3];
    orc_rgb_to_t(d, r, g, b, t);
    const double X = t[0] * d->white[0], Y = t[1] * d->white[1], Z = t[2] * d->white[2];
    const double fy = mode ? orc_f_approx(t[1], p, n, q, m) : orc_f_exact(t[1]);
    const double L = 116.0 * fy - 16.0;
    const double Xn = d->white[0], Yn = d->white[1], Zn = d->white[2];
    const double dn = Xn + 15.0 * Yn + 3.0 * Zn;
    const double un = 4.0 * Xn / dn, vn = 9.0 * Yn / dn;
    const double den = X + 15.0 * Y + 3.0 * Z;
    luv[0] = L;
    if (den > 0.0) {
        luv[1] = 13.0 * L * (4.0 * X / den - un);
        luv[2] = 13.0 * L * (9.0 * Y / den - vn);
    } else {
        luv[1] = 0.0;
        luv[2] = 0.0;
    }
}

ORC_API void orc_cieluv(const orc_rgbdef *d, int mode,
                        const double *p, int n, const double *q, int m,
                        const uint8_t *rgb, int64_t npix,
                        double *L, double *U, double *V, int nthreads)
{
    orc_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npix; ++i) {
        double luv[3];
        orc_cieluv_pixel(d, mode, p, n, q, m, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], luv);
        L[i] = luv[0];
        U[i] = luv[1];
        V[i] = luv[2];
    }
}

/* Delta E*uv (the Euclidean distance in L*u*v*) between the MACT and the
 * exact CIELUV, average and maximum over the 2^24 cube. */
ORC_API void orc_cube_eps_cieluv(const orc_rgbdef *d, const double *p, int n,
                                 const double *q, int m, double out[2])
{
    double sum = 0.0, mx = 0.0;
#pragma omp parallel for reduction(+:sum) reduction(max:mx) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double e[3], a[3];
                orc_cieluv_pixel(d, 0, NULL, 0, NULL, 0, r, g, b, e);
                orc_cieluv_pixel(d, 1, p, n, q, m, r, g, b, a);
                double de = orc_delta_e(e, a);
                sum += de;
                if (de > mx) mx = de;
            }
    out[0] = sum / 16777216.0;
    out[1] = mx;
}

/* --------------------------------------------------------------------- HSI */

/* arctan(sqrt(3) x) -- exact, or sgn(x) P_n(|x|) (Table tab_arctan and the
 * odd-symmetry identity of Section "Approximation of the Inverse Tangent
 * Function"). */
static double orc_atan_sqrt3(double x, const double *c, int n)
{
    if (!c) return atan(sqrt(3.0) * x);
    if (x < 0.0) return -orc_poly(c, n, -x);
    return orc_poly(c, n, x);
}

/* Eq. equ_rgb_kender hue (radians) on codes r, g, b; c == NULL is exact. */
static double orc_hue_kender(double r, double g, double b, const double *c, int n)
{
    if (r > b && g > b) return ORC_PI / 3.0 + orc_atan_sqrt3((g - r) / (g - b + r - b), c, n);
    if (g > r) return ORC_PI + orc_atan_sqrt3((b - g) / (b - r + g - r), c, n);
    if (b > g) return 5.0 * ORC_PI / 3.0 + orc_atan_sqrt3((r - b) / (r - g + b - g), c, n);
    if (r > b) return 0.0;
    return 0.0; /* undefined (gray): convention H = 0 */
}

/* Eq. equ_rgb_hsi hue via arccos (the original form), for cross-checking. */
static double orc_hue_arccos(double r, double g, double b)
{
    double den = sqrt((r - g) * (r - g) + (r - b) * (g - b));
    if (den == 0.0) return 0.0;
    double c = 0.5 * (r - g + r - b) / den;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double h = acos(c);
    if (b > g) h = 2.0 * ORC_PI - h;
    return h;
}

/* One pixel of RGB -> HSI.  mode 0: Kender exact, 1: Kender with P_n,
 * 2: arccos form.  H in radians, S and I in [0,1] with R = R'/255. */
ORC_API void orc_hsi_pixel(int mode, const double *c, int n,
                           double r, double g, double b, double hsi[3])
{
    double sum = r + g + b;
    double mn = r < g ? (r < b ? r : b) : (g < b ? g : b);
    if (mode == 2)
        hsi[0] = orc_hue_arccos(r, g, b);
    else
        hsi[0] = orc_hue_kender(r, g, b, mode == 1 ? c : NULL, n);
    hsi[1] = sum > 0.0 ? 1.0 - 3.0 * mn / sum : 0.0;
    hsi[2] = (sum / 255.0) / 3.0;
}

ORC_API void orc_hsi(int mode, const double *c, int n,
                     const uint8_t *rgb, int64_t npix,
                     double *H, double *S, double *I, int nthreads)
{
    orc_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npix; ++i) {
        double hsi[3];
        orc_hsi_pixel(mode, c, n, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], hsi);
        H[i] = hsi[0];
        S[i] = hsi[1];
        I[i] = hsi[2];
    }
}

/* Eq. equ_hsi_dist. */
ORC_API double orc_d_hsi(const double x[3], const double y[3])
{
    double dh = fabs(x[0] - y[0]);
    double th = dh <= ORC_PI ? dh : 2.0 * ORC_PI - dh;
    double di = x[2] - y[2];
    double v = x[1] * x[1] + y[1] * y[1] - 2.0 * x[1] * y[1] * cos(th) + di * di;
    return sqrt(v > 0.0 ? v : 0.0);
}

/* --------------------------------------------------------------------- SCT */

typedef struct {
    const double *p; int n;   /* Table tab_arcsin: 2 arcsin(y/sqrt2), y = sqrt(1-x) */
    const double *q; int m;   /* Table tab_arccos: arccos(x) on [0, 0.5]           */
    const double *f; int rf;  /* Table tab_f: arctan(x) on [0, 254/255]            */
    const double *g; int rg;  /* Table tab_g: pi/2 - arctan(w) on [1/255, 1]       */
} orc_sct_coeffs;

/* One pixel of RGB -> SCT (Eq. equ_rgb_sct with Eq. equ_sct_b).
 * co == NULL: exact.  Output (L, angle A, angle B), L in code units. */
ORC_API void orc_sct_pixel(const orc_sct_coeffs *co, double r, double g, double b, double out[3])
{
    double L = sqrt(r * r + g * g + b * b);
    double A, B;
    if (L == 0.0) {
        out[0] = 0.0; out[1] = 0.0; out[2] = 0.0;
        return;
    }
    double x = b / L;
    if (!co) {
        A = acos(x);
    } else if (x >= 0.5) {
        double y = sqrt(1.0 - x);                 /* Eq. equ_arccos_cheap */
        A = orc_poly(co->p, co->n, y);
    } else {
        A = orc_poly(co->q, co->m, x);
    }
    if (r == 0.0 && g == 0.0) {
        B = 0.0;                                  /* undefined: convention 0 */
    } else if (!co) {
        B = atan2(g, r);
    } else if (r == 0.0) {
        B = ORC_PI / 2.0;                         /* R = 0, G > 0 */
    } else if (g < r) {
        B = orc_poly(co->f, co->rf, g / r);       /* f(G/R) */
    } else {
        B = orc_poly(co->g, co->rg, r / g);       /* g: pi/2 - arctan(R/G) */
    }
    out[0] = L;
    out[1] = A;
    out[2] = B;
}

ORC_API void orc_sct(const orc_sct_coeffs *co, const uint8_t *rgb, int64_t npix,
                     double *Lo, double *Ao, double *Bo, int nthreads)
{
    orc_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npix; ++i) {
        double s[3];
        orc_sct_pixel(co, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], s);
        Lo[i] = s[0];
        Ao[i] = s[1];
        Bo[i] = s[2];
    }
}

/* Eq. equ_sct_rgb: SCT -> RGB codes (real valued, not clamped). */
ORC_API void orc_sct_inverse(const double s[3], double rgb[3])
{
    rgb[0] = s[0] * sin(s[1]) * cos(s[2]);
    rgb[1] = s[0] * sin(s[1]) * sin(s[2]);
    rgb[2] = s[0] * cos(s[1]);
}

/* ---------------------------------------------------------------- 3D LUTs */

/* Packing (Section "Comparison with 3D Lookup Table Interpolation Methods"):
 * node (i, j, k) holds the exact CIELAB of k' = (i, j, k)/(N-1), rounded to
 * FP32.  Layout lut[((i*N + j)*N + k)*3 + c], R outermost. */
ORC_API void orc_lut_build(const orc_rgbdef *d, int N, float *lut)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                double lab[3];
                double s = 255.0 / (double)(N - 1);
                orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, i * s, j * s, k * s, lab);
                for (int c = 0; c < 3; ++c)
                    lut[((int64_t)(i * N + j) * N + k) * 3 + c] = (float)lab[c];
            }
}

/* Extraction: integer cell index and remainder of a code along one axis. */
static void orc_lut_locate(int v, int N, int *idx, int *rem)
{
    int s = v * (N - 1);
    *idx = s / 255;
    *rem = s % 255;
    if (*idx == N - 1) {   /* v = 255 */
        *idx = N - 2;
        *rem = 255;
    }
}

enum { ORC_TRILINEAR = 0, ORC_PRISM = 1, ORC_PYRAMID = 2, ORC_TETRA = 3 };

/* Interpolation of one pixel.  Writes the three values and returns the
 * selection id: (node index of the cell's lower corner) * 8 + simplex id.
 * Corner cXYZ has X = R offset, Y = G offset, Z = B offset.  Weights are the
 * classic forms of each method (Kang 2006, as the paper cites). */
ORC_API int orc_lut_interp_pixel(int method, const float *lut, int N,
                                 int r, int g, int b, double out[3])
{
    int ir, ig, ib, rr, rg, rb;
    orc_lut_locate(r, N, &ir, &rr);
    orc_lut_locate(g, N, &ig, &rg);
    orc_lut_locate(b, N, &ib, &rb);
    double fr = rr / 255.0, fg = rg / 255.0, fb = rb / 255.0;
    int base = (ir * N + ig) * N + ib;
    int simplex = 0;
    for (int ch = 0; ch < 3; ++ch) {
#define C(x, y, z) ((double)lut[((int64_t)base + (int64_t)(x) * N * N + (int64_t)(y) * N + (z)) * 3 + ch])
        double c000 = C(0, 0, 0), c001 = C(0, 0, 1), c010 = C(0, 1, 0), c011 = C(0, 1, 1);
        double c100 = C(1, 0, 0), c101 = C(1, 0, 1), c110 = C(1, 1, 0), c111 = C(1, 1, 1);
#undef C
        double v;
        if (method == ORC_TRILINEAR) {
            v = c000 * (1 - fr) * (1 - fg) * (1 - fb) + c001 * (1 - fr) * (1 - fg) * fb
              + c010 * (1 - fr) * fg * (1 - fb) + c011 * (1 - fr) * fg * fb
              + c100 * fr * (1 - fg) * (1 - fb) + c101 * fr * (1 - fg) * fb
              + c110 * fr * fg * (1 - fb) + c111 * fr * fg * fb;
            simplex = 0;
        } else if (method == ORC_PRISM) {
            /* prism axis along R; the G-B face is split on its diagonal */
            if (rg >= rb) {
                v = c000 + (c010 - c000) * fg + (c011 - c010) * fb + (c100 - c000) * fr
                  + (c110 - c100 - c010 + c000) * fg * fr + (c111 - c110 - c011 + c010) * fb * fr;
                simplex = 0;
            } else {
                v = c000 + (c011 - c001) * fg + (c001 - c000) * fb + (c100 - c000) * fr
                  + (c111 - c101 - c011 + c001) * fg * fr + (c101 - c100 - c001 + c000) * fb * fr;
                simplex = 1;
            }
        } else if (method == ORC_PYRAMID) {
            /* apex c111; the base is the cube face of the smallest fraction */
            if (rb <= rr && rb <= rg) {          /* base B = 0 */
                v = c000 + (c111 - c110) * fb + (c100 - c000) * fr + (c010 - c000) * fg
                  + (c110 - c100 - c010 + c000) * fr * fg;
                simplex = 0;
            } else if (rg <= rr && rg <= rb) {   /* base G = 0 */
                v = c000 + (c111 - c101) * fg + (c100 - c000) * fr + (c001 - c000) * fb
                  + (c101 - c100 - c001 + c000) * fr * fb;
                simplex = 1;
            } else {                             /* base R = 0 */
                v = c000 + (c111 - c011) * fr + (c010 - c000) * fg + (c001 - c000) * fb
                  + (c011 - c001 - c010 + c000) * fg * fb;
                simplex = 2;
            }
        } else {
            /* tetrahedral: six orderings of (rem_R, rem_G, rem_B) */
            if (rr >= rg && rg >= rb) {
                v = c000 + (c100 - c000) * fr + (c110 - c100) * fg + (c111 - c110) * fb;
                simplex = 0;
            } else if (rr >= rb && rb > rg) {
                v = c000 + (c100 - c000) * fr + (c111 - c101) * fg + (c101 - c100) * fb;
                simplex = 1;
            } else if (rb > rr && rr >= rg) {
                v = c000 + (c101 - c001) * fr + (c111 - c101) * fg + (c001 - c000) * fb;
                simplex = 2;
            } else if (rg > rr && rr >= rb) {
                v = c000 + (c110 - c010) * fr + (c010 - c000) * fg + (c111 - c110) * fb;
                simplex = 3;
            } else if (rg >= rb && rb > rr) {
                v = c000 + (c111 - c011) * fr + (c010 - c000) * fg + (c011 - c010) * fb;
                simplex = 4;
            } else {
                v = c000 + (c111 - c011) * fr + (c011 - c001) * fg + (c001 - c000) * fb;
                simplex = 5;
            }
        }
        out[ch] = v;
    }
    return base * 8 + simplex;
}

ORC_API void orc_lut_interp(int method, const float *lut, int N,
                            const uint8_t *rgb, int64_t npix,
                            double *o0, double *o1, double *o2, int32_t *sel, int nthreads)
{
    orc_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npix; ++i) {
        double v[3];
        int s = orc_lut_interp_pixel(method, lut, N, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], v);
        o0[i] = v[0];
        o1[i] = v[1];
        o2[i] = v[2];
        if (sel) sel[i] = s;
    }
}

/* ------------------------------------------- statistics over the RGB cube */
/* Section "Calculation of the Color Space Transformation Errors": average and
 * maximum transformation error over every 24-bit colour. */

/* Fractions of the cube with t_c > 0.008856 (Eq. equ_cbrt_prob). */
ORC_API void orc_cube_cbrt_probs(const orc_rgbdef *d, double probs[3])
{
    int64_t cnt[3] = {0, 0, 0};
    int64_t c0 = 0, c1 = 0, c2 = 0;
#pragma omp parallel for reduction(+:c0, c1, c2) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double t[3];
                orc_rgb_to_t(d, r, g, b, t);
                c0 += t[0] > 0.008856;
                c1 += t[1] > 0.008856;
                c2 += t[2] > 0.008856;
            }
    cnt[0] = c0; cnt[1] = c1; cnt[2] = c2;
    for (int c = 0; c < 3; ++c) probs[c] = (double)cnt[c] / 16777216.0;
}

/* P(B/L >= 0.5) and P(not (R = G = 0)) (Eq. equ_sct_arcsin_arccos_prob,
 * equ_sct_b_prob), on the codes. */
ORC_API void orc_cube_sct_probs(double probs[2])
{
    int64_t na = 0, nb = 0;
#pragma omp parallel for reduction(+:na, nb) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double L = sqrt((double)(r * r + g * g + b * b));
                if (L > 0.0 && b / L >= 0.5) na++;
                if (!(r == 0 && g == 0)) nb++;
            }
    probs[0] = (double)na / 16777216.0;
    probs[1] = (double)nb / 16777216.0;
}

/* CIELAB: Delta E*ab between the MACT and the exact transform. */
ORC_API void orc_cube_eps_cielab(const orc_rgbdef *d, const double *p, int n,
                                 const double *q, int m, double out[2])
{
    double sum = 0.0, mx = 0.0;
#pragma omp parallel for reduction(+:sum) reduction(max:mx) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double e[3], a[3];
                orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, r, g, b, e);
                orc_cielab_pixel(d, 1, p, n, q, m, r, g, b, a);
                double de = orc_delta_e(e, a);
                sum += de;
                if (de > mx) mx = de;
            }
    out[0] = sum / 16777216.0;
    out[1] = mx;
}

/* HSI: D_HSI between Kender-with-P_n and the exact transform. */
ORC_API void orc_cube_eps_hsi(const double *c, int n, double out[2])
{
    double sum = 0.0, mx = 0.0;
#pragma omp parallel for reduction(+:sum) reduction(max:mx) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double e[3], a[3];
                orc_hsi_pixel(0, NULL, 0, r, g, b, e);
                orc_hsi_pixel(1, c, n, r, g, b, a);
                double dd = orc_d_hsi(e, a);
                sum += dd;
                if (dd > mx) mx = dd;
            }
    out[0] = sum / 16777216.0;
    out[1] = mx;
}

/* SCT: approximate SCT -> inverse SCT -> exact CIELAB, Delta E*ab against
 * the exact CIELAB of the pixel (Section "Color Space Description" of SCT). */
ORC_API void orc_cube_eps_sct(const orc_rgbdef *d, const orc_sct_coeffs *co, double out[2])
{
    double sum = 0.0, mx = 0.0;
#pragma omp parallel for reduction(+:sum) reduction(max:mx) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double s[3], back[3], e[3], a[3];
                orc_sct_pixel(co, r, g, b, s);
                orc_sct_inverse(s, back);
                orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, back[0], back[1], back[2], a);
                orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, r, g, b, e);
                double de = orc_delta_e(e, a);
                sum += de;
                if (de > mx) mx = de;
            }
    out[0] = sum / 16777216.0;
    out[1] = mx;
}

/* LUT interpolation: Delta E*ab against the exact CIELAB. */
ORC_API void orc_cube_eps_lut(const orc_rgbdef *d, int method, const float *lut, int N, double out[2])
{
    double sum = 0.0, mx = 0.0;
#pragma omp parallel for reduction(+:sum) reduction(max:mx) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double e[3], a[3];
                orc_lut_interp_pixel(method, lut, N, r, g, b, a);
                orc_cielab_pixel(d, 0, NULL, 0, NULL, 0, r, g, b, e);
                double de = orc_delta_e(e, a);
                sum += de;
                if (de > mx) mx = de;
            }
    out[0] = sum / 16777216.0;
    out[1] = mx;
}

/* -------------------------------------- HSI LUT with angular interpolation */
/* Section "Comparison with 3D Lookup Table Interpolation Methods" (the
 * closing paragraphs, Eq. equ_angular): interpolating a LUT of an angular
 * space must mix hues as angles.  Reading (the paper gives the pairwise
 * formula only): trilinear interpolation where S and I take the trilinear
 * weights and H is mixed pairwise by Eq. equ_angular along B, then G, then
 * R, the order of repeated linear interpolation; a gray node (S = 0, hue
 * undefined) has no hue, so a pair with one gray member takes the other's
 * angle and a pair of grays stays gray; a result with S = 0 takes H = 0,
 * the exact transform's convention for grays.  Parity of eps_max unpinned: the
 * printed maximum comes from antipodal hue pairs mixed at alpha ~ 0.5,
 * where the formula is ill-conditioned; eps_avg is pinned within 0.5%
 * (it lands 0.3% away).
 *
 * LUT: node (i, j, k) holds the exact HSI (Eq. equ_rgb_kender) of codes
 * 255 (i, j, k)/(N-1), each of H, S, I rounded to FP32 (H = 0 at grays).
 * Layout lut[((i*N + j)*N + k)*3 + c], R outermost. */
ORC_API void orc_lut_build_hsi(int N, float *lut)
{
    double s = 255.0 / (double)(N - 1);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                double hsi[3];
                orc_hsi_pixel(0, NULL, 0, i * s, j * s, k * s, hsi);
                for (int c = 0; c < 3; ++c)
                    lut[((int64_t)(i * N + j) * N + k) * 3 + c] = (float)hsi[c];
            }
}

/* Eq. equ_angular for the pair (h0, h1) at coefficient a, gray members
 * skipped; *mod receives the modulus of the mixed (cos, sin) sum, the
 * conditioning of the mix (1 when a member is skipped). */
static void orc_angle_mix(double h0, int g0, double h1, int g1, double a, double *h, int *g, double *mod)
{
    *mod = 1.0;
    if (g0 && g1) { *h = 0.0; *g = 1; return; }
    *g = 0;
    if (g0) { *h = h1; return; }
    if (g1) { *h = h0; return; }
    double y = (1.0 - a) * sin(h0) + a * sin(h1);
    double x = (1.0 - a) * cos(h0) + a * cos(h1);
    *h = atan2(y, x);
    *mod = sqrt(x * x + y * y);
}

/* One pixel: out = (H in [0, 2pi), S, I); returns the smallest mix modulus
 * met along the chain (small = the hue is ill-conditioned there). */
ORC_API double orc_lut_interp_hsi_pixel(const float *lut, int N, int r, int g, int b, double out[3])
{
    int ir, ig, ib, rr, rg, rb;
    orc_lut_locate(r, N, &ir, &rr);
    orc_lut_locate(g, N, &ig, &rg);
    orc_lut_locate(b, N, &ib, &rb);
    double f[3] = {rr / 255.0, rg / 255.0, rb / 255.0};   /* R, G, B */
    int64_t base = ((int64_t)ir * N + ig) * N + ib;
    double hv[8], sv[8], iv[8];
    int gv[8];
    for (int c = 0; c < 8; ++c) {   /* corner c = 4 dR + 2 dG + dB */
        int64_t node = base + (int64_t)((c >> 2) & 1) * N * N + (int64_t)((c >> 1) & 1) * N + (c & 1);
        hv[c] = lut[node * 3 + 0];
        sv[c] = lut[node * 3 + 1];
        iv[c] = lut[node * 3 + 2];
        gv[c] = sv[c] == 0.0;
    }
    double S = 0.0, I = 0.0;
    for (int c = 0; c < 8; ++c) {
        double w = (((c >> 2) & 1) ? f[0] : 1.0 - f[0]) * (((c >> 1) & 1) ? f[1] : 1.0 - f[1]) *
                   ((c & 1) ? f[2] : 1.0 - f[2]);
        S += w * sv[c];
        I += w * iv[c];
    }
    double cond = 1.0, m;
    int n = 8;
    for (int axis = 2; axis >= 0; --axis) {   /* B (bit 0), then G (bit 1), then R (bit 2) */
        for (int k = 0; k < n / 2; ++k) {     /* after each pass the survivors are packed */
            double h;
            int gg;
            orc_angle_mix(hv[2 * k], gv[2 * k], hv[2 * k + 1], gv[2 * k + 1], f[axis], &h, &gg, &m);
            hv[k] = h;
            gv[k] = gg;
            if (m < cond) cond = m;
        }
        n /= 2;
    }
    double H = hv[0];
    if (H < 0.0) H += 2.0 * ORC_PI;
    if (H >= 2.0 * ORC_PI) H -= 2.0 * ORC_PI;
    if (S == 0.0) H = 0.0;   /* a gray result: the exact transform's convention */
    out[0] = H;
    out[1] = S;
    out[2] = I;
    return cond;
}

ORC_API void orc_lut_interp_hsi(const float *lut, int N, const uint8_t *rgb, int64_t npix,
                                double *H, double *S, double *I, double *cond, int nthreads)
{
    orc_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npix; ++i) {
        double o[3];
        double c = orc_lut_interp_hsi_pixel(lut, N, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], o);
        H[i] = o[0];
        S[i] = o[1];
        I[i] = o[2];
        if (cond) cond[i] = c;
    }
}

/* eps^T of the angular HSI LUT: D_HSI (Eq. equ_hsi_dist) against the exact
 * HSI over every 24-bit colour. */
ORC_API void orc_cube_eps_hsi_lut(const float *lut, int N, double out[2])
{
    double sum = 0.0, mx = 0.0;
#pragma omp parallel for reduction(+:sum) reduction(max:mx) schedule(static)
    for (int r = 0; r < 256; ++r)
        for (int g = 0; g < 256; ++g)
            for (int b = 0; b < 256; ++b) {
                double e[3], a[3];
                orc_lut_interp_hsi_pixel(lut, N, r, g, b, a);
                orc_hsi_pixel(0, NULL, 0, r, g, b, e);
                double d = orc_d_hsi(e, a);
                sum += d;
                if (d > mx) mx = d;
            }
    out[0] = sum / 16777216.0;
    out[1] = mx;
}

/* ------------------------------------------- differentiable RGB -> CIELAB */
/* Input is LINEAR RGB (the output of Eq. equ_rgb_lin), planar (N, 3, HW).
 * Lab follows Eq. equ_rgb_xyz and equ_xyz_lab; the loss is the mean over
 * pixels of Delta E*ab (Eq. equ_cielab_dist) against a target Lab image
 * (N, 3, HW).  The gradient is the analytic derivative of that loss:
 *   dLoss/dLab = (Lab - target) / (npix * Delta E)   (0 where Delta E = 0)
 *   dLab/df:     L = 116 f_y - 16, a = 500 (f_x - f_y), b = 200 (f_y - f_z)
 *   df/dt:       exact 1/(3 t^(2/3)); approximant (p'q - p q')/q^2;
 *                7.787 on the linear segment t <= 0.008856
 *   dt/dRGB:     rows of the matrix divided by the white point. */

static double orc_dpoly(const double *a, int n, double x)
{
    double s = 0.0, xp = 1.0;
    for (int i = 1; i <= n; ++i) {
        s += i * a[i] * xp;
        xp *= x;
    }
    return s;
}

/* f(t) and f'(t); mode 0 exact, 1 approximant p/q (m < 0: polynomial). */
static void orc_f_and_df(int mode, const double *p, int n, const double *q, int m, double t, double *f, double *df)
{
    if (t <= 0.008856) {
        *f = 7.787 * t + 16.0 / 116.0;
        *df = 7.787;
        return;
    }
    if (!mode) {
        *f = cbrt(t);
        *df = 1.0 / (3.0 * cbrt(t * t));
        return;
    }
    double pv = orc_poly(p, n, t), dp = orc_dpoly(p, n, t);
    double qv = m >= 0 ? orc_poly(q, m, t) : 1.0, dq = m >= 0 ? orc_dpoly(q, m, t) : 0.0;
    *f = pv / qv;
    *df = (dp * qv - pv * dq) / (qv * qv);
}

/* Lab of linear RGB (N, 3, HW) -> (N, 3, HW). */
ORC_API void orc_lab_linear(const orc_rgbdef *d, int mode, const double *p, int n, const double *q, int m,
                            const double *x, int64_t nb, int64_t hw, double *lab)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nb * hw; ++k) {
        int64_t b = k / hw, i = k % hw;
        const double *xb = x + b * 3 * hw;
        double f[3], df;
        for (int c = 0; c < 3; ++c) {
            double xyz = d->m[3 * c] * xb[i] + d->m[3 * c + 1] * xb[hw + i] + d->m[3 * c + 2] * xb[2 * hw + i];
            orc_f_and_df(mode, p, n, q, m, xyz / d->white[c], &f[c], &df);
        }
        double lab3[3];
        orc_lab_from_f(f[0], f[1], f[2], lab3);
        for (int c = 0; c < 3; ++c) lab[b * 3 * hw + c * hw + i] = lab3[c];
    }
}

/* Mean Delta E*ab loss against target Lab and its gradient w.r.t. x. */
ORC_API double orc_lab_loss_grad(const orc_rgbdef *d, int mode, const double *p, int n, const double *q, int m,
                                 const double *x, const double *target, int64_t nb, int64_t hw, double *grad)
{
    const double npix = (double)(nb * hw);
    double total = 0.0;
#pragma omp parallel for reduction(+:total) schedule(static)
    for (int64_t k = 0; k < nb * hw; ++k) {
        int64_t b = k / hw, i = k % hw;
        const double *xb = x + b * 3 * hw;
        const double *tb = target + b * 3 * hw;
        double f[3], df[3];
        for (int c = 0; c < 3; ++c) {
            double xyz = d->m[3 * c] * xb[i] + d->m[3 * c + 1] * xb[hw + i] + d->m[3 * c + 2] * xb[2 * hw + i];
            orc_f_and_df(mode, p, n, q, m, xyz / d->white[c], &f[c], &df[c]);
        }
        double lab3[3];
        orc_lab_from_f(f[0], f[1], f[2], lab3);
        double dl = lab3[0] - tb[i], da = lab3[1] - tb[hw + i], dbb = lab3[2] - tb[2 * hw + i];
        double de = sqrt(dl * dl + da * da + dbb * dbb);
        total += de;
        if (!grad) continue;
        double gL = 0.0, ga = 0.0, gb = 0.0;
        if (de > 0.0) {
            gL = dl / (de * npix);
            ga = da / (de * npix);
            gb = dbb / (de * npix);
        }
        double gf[3] = {500.0 * ga, 116.0 * gL - 500.0 * ga + 200.0 * gb, -200.0 * gb};
        double gt[3];
        for (int c = 0; c < 3; ++c) gt[c] = gf[c] * df[c] / d->white[c];
        for (int j = 0; j < 3; ++j)
            grad[b * 3 * hw + j * hw + i] = d->m[j] * gt[0] + d->m[3 + j] * gt[1] + d->m[6 + j] * gt[2];
    }
    return total / npix;
}
