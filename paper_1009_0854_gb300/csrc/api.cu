// api.cu -- the exported C ABI of libmact.so (include/mact.h): argument
// validation, handle state, work lists, and dispatch to the kernels.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace mact {

bool hsi_unit_interval_fit(int n, double *coef6, double *err);
bool cbrt_rational_fit(int n, int m, double *p7, double *q7, double *err);

// ---- coefficient tables of the paper (ascending powers) -------------------

// Table tab_cbrt_poly: t^(1/3) ~ p_n(t).
static const double kCbrtPoly[4][6] = {
    {1.268979e-01, 2.393873, -1.647669, 0, 0, 0},
    {9.787826e-02, 4.057495, -7.388864, 4.331370, 0, 0},
    {8.111133e-02, 5.926004, -2.017165e+01, 2.833070e+01, -1.324728e+01, 0},
    {7.002910e-02, 7.961214, -4.329352e+01, 1.063182e+02, -1.135685e+02, 4.358268e+01},
};

// Table tab_cbrt_rat: t^(1/3) ~ p_n(t)/q_m(t) on [0.008856, 1].
struct RatRow { int n, m; double p[5], q[5]; };
static const RatRow kCbrtRat[9] = {
    {2, 2, {6.309655e-03, 5.785782e-01, 1.591005}, {4.482646e-02, 1.175862, 9.596879e-01}},
    {2, 3, {2.500705e-03, 3.447113e-01, 1.942708}, {1.978701e-02, 8.542797e-01, 1.664540, -2.503267e-01}},
    {3, 2, {1.776519e-03, 2.632323e-01, 1.751297, 3.836709e-01}, {1.432256e-02, 6.779998e-01, 1.706260}},
    {2, 4, {1.317899e-03, 2.390113e-01, 2.099395},
     {1.124254e-02, 6.726679e-01, 2.184656, -7.511150e-01, 2.229717e-01}},
    {3, 3, {4.370889e-04, 9.526952e-02, 1.252009, 1.302733}, {3.912364e-03, 2.954084e-01, 1.717143, 6.343408e-01}},
    {4, 2, {7.589302e-04, 1.519784e-01, 1.663584, 8.368075e-01, -1.657269e-01},
     {6.644723e-03, 4.506424e-01, 2.030622}},
    {3, 4, {1.683667e-04, 4.667675e-02, 9.106812e-01, 1.810577},
     {1.610864e-03, 1.617974e-01, 1.494070, 1.218468, -1.079451e-01}},
    {4, 3, {1.349673e-04, 3.832079e-02, 7.870174e-01, 1.799062, 2.071170e-01},
     {1.299250e-03, 1.345420e-01, 1.330358, 1.365369}},
    {4, 4, {3.927283e-05, 1.392318e-02, 4.114739e-01, 1.734853, 8.679223e-01},
     {4.022100e-04, 5.414536e-02, 8.221526e-01, 1.800167, 3.513617e-01}},
};

// Table tab_arctan as printed (n = 2 with a2 negative: the printed plus sign
// gives an error of 1.5 at x = 1 and is read as a typesetting slip).
static const double kHsiPrinted[4][6] = {
    {5.959793e-03, 1.782975, -7.497879e-01, 0, 0, 0},
    {-3.654076e-03, 1.884080, -9.805583e-01, 1.430580e-01, 0, 0},
    {-1.286369e-03, 1.796716, -4.958969e-01, -6.927404e-01, 4.421541e-01, 0},
    {-1.801283e-04, 1.739333, -2.039848e-02, -2.065512, 2.052837, -6.591729e-01},
};

// Tables tab_arcsin, tab_arccos, tab_f, tab_g (degrees 4 and 5).
static const double kSctArcsin[2][6] = {
    {2.097797e-05, 1.412840, 1.429881e-02, 6.704361e-02, 6.909677e-02, 0},
    {-2.370048e-06, 1.414434, -3.300037e-03, 1.354670e-01, -3.994259e-02, 6.099502e-02},
};
static const double kSctArccos[2][6] = {
    {1.570786, -9.990285e-01, -1.429899e-02, -9.481335e-02, -1.381942e-01, 0},
    {1.570798, -1.000156, 3.299810e-03, -1.915780e-01, 7.988231e-02, -1.725177e-01},
};
static const double kSctF[2][6] = {
    {-1.036508e-04, 1.003740, -1.773538e-02, -3.390563e-01, 1.386796e-01, 0},
    {2.073866e-05, 9.982666e-01, 2.352573e-02, -4.506862e-01, 2.635050e-01, -4.920822e-02},
};
static const double kSctG[2][6] = {
    {1.570917, -1.004004, 1.885694e-02, 3.373159e-01, -1.377930e-01, 0},
    {1.570769, -9.981253e-01, -2.440212e-02, 4.528921e-01, -2.659181e-01, 5.016228e-02},
};

// ---- errors ----------------------------------------------------------------

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

mact_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return MACT_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MACT_E_NOMEM : MACT_E_CUDA;
}

static mact_status inval(const char *msg)
{
    set_error(msg);
    return MACT_E_INVAL;
}

// ---- configuration ---------------------------------------------------------

static void build_gamma(const mact_rgb_def &d, float *g32, double *g64);

static mact_status build_coeffs(const mact_config &cfg, Coeffs &co)
{
    std::memset(&co, 0, sizeof(co));
    const mact_rgb_def &d = cfg.rgb;
    for (int c = 0; c < 3; ++c) {
        if (!(d.white[c] > 0.0) || !std::isfinite(d.white[c])) return inval("white point must be positive");
        double rowsum = 0.0;
        for (int j = 0; j < 3; ++j) {
            if (!std::isfinite(d.rgb_to_xyz[3 * c + j])) return inval("rgb_to_xyz must be finite");
            co.m64[3 * c + j] = d.rgb_to_xyz[3 * c + j] / d.white[c];
            co.m[3 * c + j] = (float)co.m64[3 * c + j];
            rowsum += d.rgb_to_xyz[3 * c + j];
        }
        // white (k = 1,1,1) must map to t <= 1: the cube-root fits live on [0.008856, 1]
        if (rowsum / d.white[c] > 1.0 + 1e-6) return inval("RGB definition maps white above the reference white");
    }
    {
        // CIE 1976 u', v' terms (the CIELUV variant)
        const double Xn = d.white[0], Yn = d.white[1], Zn = d.white[2];
        const double dn = Xn + 15.0 * Yn + 3.0 * Zn;
        const double den[3] = {Xn, 15.0 * Yn, 3.0 * Zn};
        for (int c = 0; c < 3; ++c) {
            co.luv_den64[c] = den[c];
            co.luv_den[c] = (float)den[c];
        }
        co.luv_u64 = 4.0 * Xn;
        co.luv_v64 = 9.0 * Yn;
        co.luv_un64 = 4.0 * Xn / dn;
        co.luv_vn64 = 9.0 * Yn / dn;
        co.luv_c[0] = (float)(4.0 * Xn * 15.0 * Yn / dn);
        co.luv_c[1] = (float)(9.0 * Yn * Xn / dn);
        co.luv_c[2] = (float)(4.0 * Xn * 3.0 * Zn / dn);
        co.luv_c[3] = (float)(9.0 * Yn * 3.0 * Zn / dn);
    }
    if (!(d.gamma_slope > 0.0) || !(d.gamma_exponent > 0.0) || !(d.gamma_offset > -1.0) ||
        !std::isfinite(d.gamma_threshold))
        return inval("invalid gamma parameters");
    {
        // the linearised codes must be finite, non-decreasing and within
        // [0, 1]: above 1, white leaves the cube-root fits' domain
        float g32[256];
        double g64[256];
        build_gamma(d, g32, g64);
        for (int v = 0; v < 256; ++v)
            if (!std::isfinite(g64[v]) || g64[v] < 0.0 || g64[v] > 1.0 + 1e-6 || (v > 0 && g64[v] < g64[v - 1]))
                return inval("gamma parameters give a linearised code outside [0, 1] or a decreasing curve");
    }

    // cube root
    if (cfg.lab_coeffs != 0 && cfg.lab_coeffs != 1) return inval("lab_coeffs must be 0 or 1");
    co.lab_deg = 4;
    if (cfg.lab_coeffs == 1) {
        // the library's own minimax rational of t^(1/3) on [0.008856, 1]
        if (cfg.lab_n < 1 || cfg.lab_n > 6 || cfg.lab_m < 1 || cfg.lab_m > 6)
            return inval("lab_coeffs = 1 needs 1 <= lab_n, lab_m <= 6");
        double p[7], q[7], e = 0.0;
        if (!cbrt_rational_fit(cfg.lab_n, cfg.lab_m, p, q, &e)) {
            set_error("Remez exchange for the cube-root rational did not converge");
            return MACT_E_UNSUPPORTED;
        }
        for (int i = 0; i < 7; ++i) {
            co.lab_d[i] = (float)(p[i] - q[i]);   // f = 1 + (p - q)/q
            co.lab_q[i] = (float)q[i];
        }
        for (int i = 0; i < 6; ++i) {             // derivatives, for the backward
            co.lab_dd[i] = (float)((i + 1) * (p[i + 1] - q[i + 1]));
            co.lab_dq[i] = (float)((i + 1) * q[i + 1]);
        }
        co.lab_rational = 1;
        co.lab_deg = (cfg.lab_n <= 4 && cfg.lab_m <= 4) ? 4 : 6;
    } else if (cfg.lab_m == 0) {
        if (cfg.lab_n < 2 || cfg.lab_n > 5) return inval("lab_n must be 2..5 for the polynomial (lab_m = 0)");
        for (int i = 0; i < 6; ++i) {
            co.lab_d[i] = (float)kCbrtPoly[cfg.lab_n - 2][i];
            co.lab_p64[i] = kCbrtPoly[cfg.lab_n - 2][i];
        }
        co.lab_rational = 0;
    } else {
        const RatRow *row = nullptr;
        for (const RatRow &r : kCbrtRat)
            if (r.n == cfg.lab_n && r.m == cfg.lab_m) row = &r;
        if (!row) return inval("(lab_n, lab_m) is not one of the nine rationals of the cube-root table");
        double p[5] = {0, 0, 0, 0, 0}, q[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i <= row->n; ++i) p[i] = row->p[i];
        for (int i = 0; i <= row->m; ++i) q[i] = row->q[i];
        for (int i = 0; i < 5; ++i) {
            co.lab_d[i] = (float)(p[i] - q[i]);   // f = 1 + (p - q)/q
            co.lab_q[i] = (float)q[i];
        }
        for (int i = 0; i < 4; ++i) {             // derivatives, for the backward
            co.lab_dd[i] = (float)((i + 1) * (p[i + 1] - q[i + 1]));
            co.lab_dq[i] = (float)((i + 1) * q[i + 1]);
        }
        co.lab_rational = 1;
    }

    for (int i = 0; i < 8; ++i) co.lab_dqp[i] = make_float2(co.lab_d[i], co.lab_q[i]);
    for (int j = 0; j < 3; ++j) co.mp[j] = make_float2(co.m[j], co.m[3 + j]);

    // HSI
    if (cfg.hsi_n < 2 || cfg.hsi_n > 5) return inval("hsi_n must be 2..5");
    if (cfg.hsi_coeffs == 0) {
        double c[6], e = 0.0;
        if (!hsi_unit_interval_fit(cfg.hsi_n, c, &e)) return inval("Remez fit of arctan(sqrt(3)x) failed");
        for (int i = 0; i < 6; ++i) co.hsi[i] = (float)c[i];
    } else if (cfg.hsi_coeffs == 1) {
        for (int i = 0; i < 6; ++i) co.hsi[i] = (float)kHsiPrinted[cfg.hsi_n - 2][i];
    } else {
        return inval("hsi_coeffs must be 0 (fit on [0,1]) or 1 (as printed)");
    }

    // SCT
    auto deg45 = [](int v) { return v == 4 || v == 5; };
    if (!deg45(cfg.sct_n) || !deg45(cfg.sct_m) || !deg45(cfg.sct_r)) return inval("sct degrees must be 4 or 5");
    for (int i = 0; i < 6; ++i) {
        co.sct_p[i] = (float)kSctArcsin[cfg.sct_n - 4][i];
        co.sct_q[i] = (float)kSctArccos[cfg.sct_m - 4][i];
        co.sct_f[i] = (float)kSctF[cfg.sct_r - 4][i];
        co.sct_g[i] = (float)kSctG[cfg.sct_r - 4][i];
    }
    return MACT_OK;
}

// Eq. equ_rgb_lin for the 256 codes, in double; g32 gets it rounded once to
// FP32, g64 keeps it in FP64.
static void build_gamma(const mact_rgb_def &d, float *g32, double *g64)
{
    for (int v = 0; v < 256; ++v) {
        double kp = v / 255.0;
        double k = kp < d.gamma_threshold ? kp / d.gamma_slope
                                          : std::pow((kp + d.gamma_offset) / (1.0 + d.gamma_offset), d.gamma_exponent);
        g32[v] = (float)k;
        g64[v] = k;
    }
}

mact_status check_image(const mact_image *img)
{
    if (!img) return inval("image is NULL");
    if (img->width < 0 || img->height < 0) return inval("negative image size");
    if (img->space < MACT_CIELAB || img->space > MACT_CIELUV) return inval("unknown space");
    if (img->dtype != MACT_F32 && img->dtype != MACT_F16) return inval("unknown dtype");
    if (img->width == 0 || img->height == 0) return MACT_OK;
    // at most 2^42 pixels: tile indices stay below 2^31
    if (img->width > (int64_t(1) << 42) || img->height > ((int64_t(1) << 42) / img->width))
        return inval("image too large (more than 2^42 pixels)");
    if (!img->rgb || !img->out[0] || !img->out[1] || !img->out[2]) return inval("NULL image pointer");
    const uintptr_t esz = img->dtype == MACT_F16 ? 2 : 4;   // the kernels store whole elements
    for (int c = 0; c < 3; ++c)
        if (reinterpret_cast<uintptr_t>(img->out[c]) % esz != 0) return inval("out[c] not aligned to its element size");
    if (img->height > 1 && img->pitch_bytes < 3 * img->width) return inval("pitch_bytes < 3*width");
    if (img->height > 1 && img->out_pitch_elems < img->width) return inval("out_pitch_elems < width");
    return MACT_OK;
}

// Typed arrays the kernels read or write element by element must be aligned
// to their element size (4 bytes: float, int32).
static bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

mact_status check_access(const mact_ctx &h, const void *p, const char *what)
{
    if (h.any_host || !p) return MACT_OK;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // an unknown pointer leaves an error behind: clear it
        a.type = cudaMemoryTypeUnregistered;
    }
    if (a.type == cudaMemoryTypeUnregistered) {
        set_error(std::string(what) + ": host memory the device cannot address (pin or register it)");
        return MACT_E_INVAL;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer != p) {
        set_error(std::string(what) + ": registered host memory with a different device address");
        return MACT_E_INVAL;
    }
    return MACT_OK;
}

mact_status check_image_access(const mact_ctx &h, const mact_image &img)
{
    if (h.any_host || img.width == 0 || img.height == 0) return MACT_OK;
    mact_status st = check_access(h, img.rgb, "image rgb");
    for (int c = 0; c < 3 && st == MACT_OK; ++c) st = check_access(h, img.out[c], "image out");
    return st;
}

ImageDesc make_desc(const mact_image &img, int64_t tile_px)
{
    ImageDesc d{};
    d.rgb = img.rgb;
    for (int c = 0; c < 3; ++c) d.out[c] = img.out[c];
    d.space = img.space;
    d.dtype = img.dtype;
    const bool contiguous = img.height == 1 || (img.pitch_bytes == 3 * img.width && img.out_pitch_elems == img.width);
    if (contiguous) {   // one long row: full tiles straddle image rows
        d.width = img.width * img.height;
        d.height = (d.width > 0) ? 1 : 0;
        d.pitch = 3 * d.width;
        d.opitch = d.width;
    } else {
        d.width = img.width;
        d.height = img.height;
        d.pitch = img.pitch_bytes;
        d.opitch = img.out_pitch_elems;
    }
    d.tiles_per_row = (d.width + tile_px - 1) / tile_px;
    return d;
}

}  // namespace mact

using namespace mact;

extern "C" {

void mact_config_default(mact_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->rgb.gamma_threshold = 0.081;
    cfg->rgb.gamma_slope = 4.5;
    cfg->rgb.gamma_offset = 0.099;
    cfg->rgb.gamma_exponent = 1.0 / 0.45;
    const double m[9] = {0.412391, 0.357584, 0.180481, 0.212639, 0.715169, 0.072192, 0.019331, 0.119195, 0.950532};
    std::memcpy(cfg->rgb.rgb_to_xyz, m, sizeof(m));
    cfg->rgb.white[0] = 0.950456;
    cfg->rgb.white[1] = 1.0;
    cfg->rgb.white[2] = 1.089058;
    cfg->exact = 0;
    cfg->lab_n = 4;
    cfg->lab_m = 4;
    cfg->hsi_n = 5;
    cfg->hsi_coeffs = 0;
    cfg->sct_n = cfg->sct_m = cfg->sct_r = 5;
    cfg->lab_coeffs = 0;
}

mact_status mact_create(const mact_config *cfg, mact_handle *out)
{
    if (!cfg || !out) return inval("mact_create: NULL argument");
    if (cfg->exact != 0 && cfg->exact != 1) return inval("exact must be 0 or 1");
    mact_ctx *h = new (std::nothrow) mact_ctx();
    if (!h) return MACT_E_NOMEM;
    h->cfg = *cfg;
    mact_status st = build_coeffs(*cfg, h->co);
    if (st != MACT_OK) { delete h; return st; }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->any_host, cudaDevAttrPageableMemoryAccess, h->device);
    if (const char *force = std::getenv("MACT_CHECK_HOST_POINTERS"))
        if (force[0] != '\0' && force[0] != '0') h->any_host = 0;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_gamma, 256 * (sizeof(float) + sizeof(double)));
    if (e == cudaSuccess) {
        struct { float g32[256]; double g64[256]; } tab;
        build_gamma(cfg->rgb, tab.g32, tab.g64);
        e = cudaMemcpy(h->d_gamma, &tab, sizeof(tab), cudaMemcpyHostToDevice);
    }
    for (auto &sl : h->batch_slots) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_copy, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev_kernel, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_lut, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_grad, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        st = cuda_status(e, "mact_create");
        mact_destroy(h);
        return st;
    }
    *out = h;
    return MACT_OK;
}

mact_status mact_destroy(mact_handle h)
{
    if (!h) return inval("mact_destroy: NULL handle");
    cudaDeviceSynchronize();
    if (h->d_gamma) cudaFree(h->d_gamma);
    for (auto &sl : h->batch_slots) {
        if (sl.d_work) cudaFree(sl.d_work);
        if (sl.h_work) cudaFreeHost(sl.h_work);
        if (sl.ev_copy) cudaEventDestroy(sl.ev_copy);
        if (sl.ev_kernel) cudaEventDestroy(sl.ev_kernel);
    }
    if (h->d_lut4) cudaFree(h->d_lut4);
    if (h->ev_lut) cudaEventDestroy(h->ev_lut);
    if (h->d_partial) cudaFree(h->d_partial);
    if (h->ev_grad) cudaEventDestroy(h->ev_grad);
    delete h;
    return MACT_OK;
}

mact_status mact_convert(mact_handle h, const mact_image *img, mact_stream stream)
{
    if (!h) return inval("mact_convert: NULL handle");
    mact_status st = check_image(img);
    if (st != MACT_OK) return st;
    if (img->width == 0 || img->height == 0) return MACT_OK;
    st = check_image_access(*h, *img);
    if (st != MACT_OK) return st;
    ImageDesc d = make_desc(*img);
    return cuda_status(launch_convert(*h, d, (cudaStream_t)stream), "mact_convert launch");
}

mact_status mact_convert_batch(mact_handle h, const mact_image *imgs, int32_t count, mact_stream stream)
{
    if (!h) return inval("mact_convert_batch: NULL handle");
    if (count < 0) return inval("negative image count");
    if (count > 0 && !imgs) return inval("imgs is NULL");
    for (int32_t i = 0; i < count; ++i) {
        mact_status st = check_image(&imgs[i]);
        if (st == MACT_OK) st = check_image_access(*h, imgs[i]);
        if (st != MACT_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int32_t nonempty = 0;
    for (int32_t i = 0; i < count; ++i) nonempty += (imgs[i].width != 0 && imgs[i].height != 0);
    if (nonempty == 0) return MACT_OK;
    if (nonempty <= kParamImages) {   // short list: by value in the kernel parameters
        BatchCfg cfg;
        {
            std::lock_guard<std::mutex> lock(h->batch_mu);
            cfg = h->batch_cfg;
        }
        ParamList list{};
        int64_t total = 0;
        int32_t n = 0;
        for (int32_t i = 0; i < count; ++i) {
            if (imgs[i].width == 0 || imgs[i].height == 0) continue;
            ImageDesc d = make_desc(imgs[i], cfg.tile_px());
            d.tile_begin = total;
            total += tiles_of(d);
            list.img[n++] = d;
        }
        int per_sm = batch_blocks_per_sm(*h, cfg, true);
        if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
        int64_t grid = (int64_t)h->num_sms * per_sm;
        if (grid > total) grid = total;
        return cuda_status(launch_batch_param(*h, list, n, total, (int)grid, s, cfg), "mact_convert_batch launch");
    }
    std::lock_guard<std::mutex> lock(h->batch_mu);
    mact_ctx::BatchSlot &sl = h->batch_slots[h->batch_next];
    h->batch_next = (h->batch_next + 1) % mact_ctx::kBatchSlots;
    // this slot's staging buffer and device list were used kBatchSlots calls
    // ago: wait for that call's copy (host side) and kernel (stream side)
    cudaError_t e = cudaEventSynchronize(sl.ev_copy);
    if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch: previous copy");
    if (count > sl.cap) {
        e = cudaEventSynchronize(sl.ev_kernel);
        if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch: previous kernel");
        int64_t cap = count < 64 ? 64 : count;
        if (sl.d_work) cudaFree(sl.d_work);
        if (sl.h_work) cudaFreeHost(sl.h_work);
        sl.d_work = nullptr;
        sl.h_work = nullptr;
        sl.cap = 0;
        e = cudaMalloc(&sl.d_work, 256 + cap * sizeof(ImageDesc));
        if (e == cudaSuccess) e = cudaMemset(sl.d_work, 0, 256);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_work, cap * sizeof(ImageDesc));
        if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch: work list allocation");
        sl.cap = cap;
    }
    const BatchCfg cfg = h->batch_cfg;
    int64_t total = 0;
    int32_t n = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (imgs[i].width == 0 || imgs[i].height == 0) continue;
        ImageDesc d = make_desc(imgs[i], cfg.tile_px());
        d.tile_begin = total;
        total += tiles_of(d);
        sl.h_work[n++] = d;
    }
    if (total == 0) return MACT_OK;
    unsigned long long *d_ctr = reinterpret_cast<unsigned long long *>(sl.d_work);
    ImageDesc *d_imgs = reinterpret_cast<ImageDesc *>(reinterpret_cast<char *>(sl.d_work) + 256);
    e = cudaStreamWaitEvent(s, sl.ev_kernel, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_imgs, sl.h_work, n * sizeof(ImageDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_copy, s);
    if (e != cudaSuccess) return cuda_status(e, "mact_convert_batch: work list copy");
    int per_sm = batch_blocks_per_sm(*h, cfg);
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    int64_t grid = (int64_t)h->num_sms * per_sm;
    if (grid > total) grid = total;
    e = launch_batch(*h, d_imgs, n, total, d_ctr, (int)grid, s, cfg);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_kernel, s);
    return cuda_status(e, "mact_convert_batch launch");
}

mact_status mact_lut_build(mact_handle h, int32_t n, float *d_lut, mact_stream stream)
{
    if (!h) return inval("mact_lut_build: NULL handle");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (!d_lut) return inval("d_lut is NULL");
    if (!aligned4(d_lut)) return inval("d_lut not 4-byte aligned");
    mact_status st = check_access(*h, d_lut, "d_lut");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_build(*h, n, d_lut, (cudaStream_t)stream), "mact_lut_build launch");
}

mact_status mact_lut_interp(mact_handle h, int32_t method, const float *d_lut, int32_t n, const uint8_t *d_rgb,
                            int64_t npix, float *const d_out[3], int32_t *d_sel, mact_stream stream)
{
    if (!h) return inval("mact_lut_interp: NULL handle");
    if (method < MACT_TRILINEAR || method > MACT_TETRA) return inval("unknown interpolation method");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (npix < 0 || npix > (int64_t(1) << 42)) return inval("pixel count out of range");
    if (npix == 0) return MACT_OK;
    if (!d_lut || !d_rgb || !d_out || !d_out[0] || !d_out[1] || !d_out[2]) return inval("NULL pointer");
    if (!aligned4(d_lut) || !aligned4(d_out[0]) || !aligned4(d_out[1]) || !aligned4(d_out[2]) || !aligned4(d_sel))
        return inval("d_lut, d_out[] and d_sel must be 4-byte aligned");
    mact_status st = check_access(*h, d_lut, "d_lut");
    if (st == MACT_OK) st = check_access(*h, d_rgb, "d_rgb");
    for (int c = 0; c < 3 && st == MACT_OK; ++c) st = check_access(*h, d_out[c], "d_out");
    if (st == MACT_OK) st = check_access(*h, d_sel, "d_sel");
    if (st != MACT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!lut_needs_pack(n))
        return cuda_status(launch_lut_interp(*h, method, d_lut, nullptr, n, d_rgb, npix, d_out, d_sel, s),
                           "mact_lut_interp launch");
    // large LUT: repack into the handle's float4 buffer, read by the kernel
    std::lock_guard<std::mutex> lock(h->lut_mu);
    const int64_t nodes = (int64_t)n * n * n;
    cudaError_t e = cudaSuccess;
    if (nodes > h->lut4_cap) {
        e = cudaEventSynchronize(h->ev_lut);
        if (e == cudaSuccess && h->d_lut4) e = cudaFree(h->d_lut4);
        h->d_lut4 = nullptr;
        h->lut4_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&h->d_lut4, nodes * kLutPackedFloats * sizeof(float));
        if (e != cudaSuccess) return cuda_status(e, "mact_lut_interp: LUT buffer");
        h->lut4_cap = nodes;
    }
    e = cudaStreamWaitEvent(s, h->ev_lut, 0);   // previous reader of the buffer (any stream)
    if (e == cudaSuccess) e = launch_lut_pack(d_lut, n, h->d_lut4, s);
    if (e == cudaSuccess)
        e = launch_lut_interp(*h, method, nullptr, reinterpret_cast<const float4 *>(h->d_lut4), n, d_rgb, npix,
                              d_out, d_sel, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_lut, s);
    return cuda_status(e, "mact_lut_interp launch");
}

mact_status mact_lut_pack(mact_handle h, const float *d_lut, int32_t n, float *d_packed, mact_stream stream)
{
    if (!h) return inval("mact_lut_pack: NULL handle");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (!d_lut || !d_packed) return inval("NULL pointer");
    if (!aligned4(d_lut)) return inval("d_lut not 4-byte aligned");
    if ((reinterpret_cast<uintptr_t>(d_packed) & 15) != 0) return inval("d_packed must be 16-byte aligned");
    mact_status st = check_access(*h, d_lut, "d_lut");
    if (st == MACT_OK) st = check_access(*h, d_packed, "d_packed");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_pack(d_lut, n, d_packed, (cudaStream_t)stream), "mact_lut_pack launch");
}

mact_status mact_lut_interp_packed(mact_handle h, int32_t method, const float *d_lut4, int32_t n,
                                   const uint8_t *d_rgb, int64_t npix, float *const d_out[3], int32_t *d_sel,
                                   mact_stream stream)
{
    if (!h) return inval("mact_lut_interp_packed: NULL handle");
    if (method < MACT_TRILINEAR || method > MACT_TETRA) return inval("unknown interpolation method");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (npix < 0 || npix > (int64_t(1) << 42)) return inval("pixel count out of range");
    if (npix == 0) return MACT_OK;
    if (!d_lut4 || !d_rgb || !d_out || !d_out[0] || !d_out[1] || !d_out[2]) return inval("NULL pointer");
    if ((reinterpret_cast<uintptr_t>(d_lut4) & 15) != 0) return inval("d_packed must be 16-byte aligned");
    if (!aligned4(d_out[0]) || !aligned4(d_out[1]) || !aligned4(d_out[2]) || !aligned4(d_sel))
        return inval("d_out[] and d_sel must be 4-byte aligned");
    mact_status st = check_access(*h, d_lut4, "d_packed");
    if (st == MACT_OK) st = check_access(*h, d_rgb, "d_rgb");
    for (int c = 0; c < 3 && st == MACT_OK; ++c) st = check_access(*h, d_out[c], "d_out");
    if (st == MACT_OK) st = check_access(*h, d_sel, "d_sel");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_interp(*h, method, nullptr, reinterpret_cast<const float4 *>(d_lut4), n, d_rgb,
                                         npix, d_out, d_sel, (cudaStream_t)stream),
                       "mact_lut_interp_packed launch");
}

// ---- differentiable RGB -> CIELAB ------------------------------------------

static mact_status check_grad(mact_handle h, int64_t nbatch, int64_t hw, const char *who)
{
    // sizes first (they need no handle): the kernels walk 32-bit grid-stride
    // loops, and with at most 2^31 items index + stride stays below 2^32 and
    // cannot wrap; the factors are bounded before the product, so it cannot
    // overflow either
    if (nbatch < 0 || hw < 0) return inval("negative size");
    const int64_t kMax = int64_t(1) << 31;
    if (nbatch > kMax || hw > kMax || nbatch * hw > kMax) return inval("more than 2^31 pixels");
    if (!h) return inval(who);
    if (h->cfg.exact == 0 && h->co.lab_rational == 0) {
        set_error("gradients are provided for the rational cube-root approximants and the exact form");
        return MACT_E_UNSUPPORTED;
    }
    return MACT_OK;
}

mact_status mact_lab_forward(mact_handle h, const float *d_x, int64_t nbatch, int64_t hw, float *d_lab,
                             mact_stream stream)
{
    mact_status st = check_grad(h, nbatch, hw, "mact_lab_forward: NULL handle");
    if (st != MACT_OK) return st;
    if (nbatch * hw == 0) return MACT_OK;
    if (!d_x || !d_lab) return inval("NULL pointer");
    if (!aligned4(d_x) || !aligned4(d_lab)) return inval("d_x and d_lab must be 4-byte aligned");
    if ((st = check_access(*h, d_x, "d_x")) != MACT_OK || (st = check_access(*h, d_lab, "d_lab")) != MACT_OK)
        return st;
    return cuda_status(launch_lab_forward(*h, d_x, nbatch, hw, d_lab, (cudaStream_t)stream), "mact_lab_forward");
}

mact_status mact_lab_backward(mact_handle h, const float *d_x, const float *d_grad_lab, int64_t nbatch, int64_t hw,
                              float *d_grad_x, mact_stream stream)
{
    mact_status st = check_grad(h, nbatch, hw, "mact_lab_backward: NULL handle");
    if (st != MACT_OK) return st;
    if (nbatch * hw == 0) return MACT_OK;
    if (!d_x || !d_grad_lab || !d_grad_x) return inval("NULL pointer");
    if (!aligned4(d_x) || !aligned4(d_grad_lab) || !aligned4(d_grad_x))
        return inval("float arrays must be 4-byte aligned");
    if ((st = check_access(*h, d_x, "d_x")) != MACT_OK || (st = check_access(*h, d_grad_lab, "d_grad_lab")) != MACT_OK ||
        (st = check_access(*h, d_grad_x, "d_grad_x")) != MACT_OK)
        return st;
    return cuda_status(launch_lab_backward(*h, d_x, d_grad_lab, nbatch, hw, d_grad_x, (cudaStream_t)stream),
                       "mact_lab_backward");
}

mact_status mact_lab_delta_e_loss(mact_handle h, const float *d_x, const float *d_target_lab, int64_t nbatch,
                                  int64_t hw, float *d_loss, float *d_grad_x, mact_stream stream)
{
    mact_status st = check_grad(h, nbatch, hw, "mact_lab_delta_e_loss: NULL handle");
    if (st != MACT_OK) return st;
    if (nbatch * hw == 0) return inval("empty input: the mean is undefined");
    if (!d_x || !d_target_lab || !d_loss) return inval("NULL pointer");
    if (!aligned4(d_x) || !aligned4(d_target_lab) || !aligned4(d_loss) || !aligned4(d_grad_x))
        return inval("float arrays must be 4-byte aligned");
    if ((st = check_access(*h, d_x, "d_x")) != MACT_OK ||
        (st = check_access(*h, d_target_lab, "d_target_lab")) != MACT_OK ||
        (st = check_access(*h, d_loss, "d_loss")) != MACT_OK || (st = check_access(*h, d_grad_x, "d_grad_x")) != MACT_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(h->grad_mu);
    cudaError_t e = cudaSuccess;
    if (!h->d_partial) e = cudaMalloc(&h->d_partial, (size_t)h->num_sms * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_grad, 0);   // previous reader of the partials
    if (e == cudaSuccess) e = launch_lab_delta_e(*h, d_x, d_target_lab, nbatch, hw, d_loss, d_grad_x, h->d_partial, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_grad, s);
    return cuda_status(e, "mact_lab_delta_e_loss");
}

// ---- transformation error over the RGB cube --------------------------------

mact_status mact_cube_error(mact_handle h, int32_t space, double *eps_avg, double *eps_max)
{
    if (!h || !eps_avg || !eps_max) return inval("mact_cube_error: NULL argument");
    if (space < MACT_CIELAB || space > MACT_SCT) return inval("unknown space");
    double out[2] = {0.0, 0.0};
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = run_cube_error(*h, space, 0, nullptr, 0, out, s);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_status(e, "mact_cube_error");
    *eps_avg = out[0];
    *eps_max = out[1];
    return MACT_OK;
}

mact_status mact_cube_error_lut(mact_handle h, int32_t method, const float *d_lut, int32_t n, double *eps_avg,
                                double *eps_max)
{
    if (!h || !d_lut || !eps_avg || !eps_max) return inval("mact_cube_error_lut: NULL argument");
    if (method < MACT_TRILINEAR || method > MACT_TETRA) return inval("unknown interpolation method");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (!aligned4(d_lut)) return inval("d_lut not 4-byte aligned");
    mact_status st = check_access(*h, d_lut, "d_lut");
    if (st != MACT_OK) return st;
    double out[2] = {0.0, 0.0};
    cudaStream_t s = nullptr;
    float4 *lut4 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&lut4, (size_t)n * n * n * sizeof(float4));
    if (e == cudaSuccess) e = launch_lut_pack4(d_lut, n, lut4, s);
    if (e == cudaSuccess) e = run_cube_error(*h, 3, method, lut4, n, out, s);
    if (lut4) cudaFree(lut4);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_status(e, "mact_cube_error_lut");
    *eps_avg = out[0];
    *eps_max = out[1];
    return MACT_OK;
}

mact_status mact_lut_cache_build(mact_handle h, const float *d_lut, int32_t n, float *d_cache, mact_stream stream)
{
    if (!h) return inval("mact_lut_cache_build: NULL handle");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (!d_lut || !d_cache) return inval("NULL pointer");
    if ((reinterpret_cast<uintptr_t>(d_cache) & 15) != 0) return inval("d_cache must be 16-byte aligned");
    if (!aligned4(d_lut)) return inval("d_lut not 4-byte aligned");
    mact_status st = check_access(*h, d_lut, "d_lut");
    if (st == MACT_OK) st = check_access(*h, d_cache, "d_cache");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_cache_build(d_lut, n, reinterpret_cast<float4 *>(d_cache), (cudaStream_t)stream),
                       "mact_lut_cache_build");
}

mact_status mact_lut_interp_cached(mact_handle h, int32_t method, const float *d_cache, int32_t n,
                                   const uint8_t *d_rgb, int64_t npix, float *const d_out[3], int32_t *d_sel,
                                   mact_stream stream)
{
    if (!h) return inval("mact_lut_interp_cached: NULL handle");
    if (method < MACT_TRILINEAR || method > MACT_TETRA) return inval("unknown interpolation method");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (npix < 0 || npix > (int64_t(1) << 42)) return inval("pixel count out of range");
    if (npix == 0) return MACT_OK;
    if (!d_cache || !d_rgb || !d_out || !d_out[0] || !d_out[1] || !d_out[2]) return inval("NULL pointer");
    if ((reinterpret_cast<uintptr_t>(d_cache) & 15) != 0) return inval("d_cache must be 16-byte aligned");
    if (!aligned4(d_out[0]) || !aligned4(d_out[1]) || !aligned4(d_out[2]) || !aligned4(d_sel))
        return inval("d_out[] and d_sel must be 4-byte aligned");
    mact_status st = check_access(*h, d_cache, "d_cache");
    if (st == MACT_OK) st = check_access(*h, d_rgb, "d_rgb");
    for (int c = 0; c < 3 && st == MACT_OK; ++c) st = check_access(*h, d_out[c], "d_out");
    if (st == MACT_OK) st = check_access(*h, d_sel, "d_sel");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_interp_cached(*h, method, reinterpret_cast<const float4 *>(d_cache), n, d_rgb,
                                                npix, d_out, d_sel, (cudaStream_t)stream),
                       "mact_lut_interp_cached");
}

mact_status mact_lut_build_hsi(mact_handle h, int32_t n, float *d_lut4, mact_stream stream)
{
    if (!h) return inval("mact_lut_build_hsi: NULL handle");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (!d_lut4) return inval("d_lut4 is NULL");
    if ((reinterpret_cast<uintptr_t>(d_lut4) & 15) != 0) return inval("d_lut4 must be 16-byte aligned");
    mact_status st = check_access(*h, d_lut4, "d_lut4");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_build_hsi(n, reinterpret_cast<float4 *>(d_lut4), (cudaStream_t)stream),
                       "mact_lut_build_hsi");
}

mact_status mact_lut_interp_hsi(mact_handle h, const float *d_lut4, int32_t n, const uint8_t *d_rgb, int64_t npix,
                                float *const d_out[3], mact_stream stream)
{
    if (!h) return inval("mact_lut_interp_hsi: NULL handle");
    if (n < 2 || n > 64) return inval("LUT size must be 2..64");
    if (npix < 0 || npix > (int64_t(1) << 42)) return inval("pixel count out of range");
    if (npix == 0) return MACT_OK;
    if (!d_lut4 || !d_rgb || !d_out || !d_out[0] || !d_out[1] || !d_out[2]) return inval("NULL pointer");
    if ((reinterpret_cast<uintptr_t>(d_lut4) & 15) != 0) return inval("d_lut4 must be 16-byte aligned");
    if (!aligned4(d_out[0]) || !aligned4(d_out[1]) || !aligned4(d_out[2])) return inval("d_out[] must be 4-byte aligned");
    mact_status st = check_access(*h, d_lut4, "d_lut4");
    if (st == MACT_OK) st = check_access(*h, d_rgb, "d_rgb");
    for (int c = 0; c < 3 && st == MACT_OK; ++c) st = check_access(*h, d_out[c], "d_out");
    if (st != MACT_OK) return st;
    return cuda_status(launch_lut_interp_hsi(*h, reinterpret_cast<const float4 *>(d_lut4), n, d_rgb, npix, d_out,
                                             (cudaStream_t)stream),
                       "mact_lut_interp_hsi");
}

int32_t mact_host_memory_access(mact_handle h)
{
    if (!h) return inval("mact_host_memory_access: NULL handle");
    return h->any_host ? 1 : 0;
}

mact_status mact_fit_cbrt_rational(int32_t n, int32_t m, double *p, double *q, double *max_err)
{
    if (!p || !q) return inval("mact_fit_cbrt_rational: NULL p or q");
    if (n < 1 || n > 6 || m < 1 || m > 6) return inval("mact_fit_cbrt_rational: degrees must be 1..6");
    double e = 0.0;
    if (!cbrt_rational_fit(n, m, p, q, &e)) {
        set_error("Remez exchange for the cube-root rational did not converge");
        return MACT_E_UNSUPPORTED;
    }
    if (max_err) *max_err = e;
    return MACT_OK;
}

mact_status mact_fit_hsi_arctan(int32_t n, double *c, double *max_err)
{
    if (!c) return inval("mact_fit_hsi_arctan: NULL c");
    if (n < 2 || n > 5) return inval("mact_fit_hsi_arctan: degree must be 2..5");
    double e = 0.0;
    if (!hsi_unit_interval_fit(n, c, &e)) {
        set_error("Remez fit of arctan(sqrt(3)x) failed");
        return MACT_E_UNSUPPORTED;
    }
    if (max_err) *max_err = e;
    return MACT_OK;
}

const char *mact_strerror(mact_status st)
{
    switch (st) {
    case MACT_OK: return "ok";
    case MACT_E_INVAL: return "invalid argument";
    case MACT_E_NOMEM: return "out of memory or admission budget";
    case MACT_E_CUDA: return "CUDA error";
    case MACT_E_UNSUPPORTED: return "unsupported";
    case MACT_E_TIMEOUT: return "timed out";
    case MACT_E_BUSY: return "busy";
    }
    return "unknown status";
}

const char *mact_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
