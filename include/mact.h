/*
 * mact.h -- C ABI of libmact.so: MACT colour-space transforms and 3D-LUT
 * interpolation on an NVIDIA GB300 (sm_103a).
 *
 * MACT (Celebi, Kingravi & Celiker, "Fast Color Space Transformations Using
 * Minimax Approximations") replaces the elementary functions of three RGB
 * transforms by minimax polynomials or rationals:
 *   RGB -> CIELAB   cube root -> p_n(t)/q_m(t)          (Tables tab_cbrt_poly,
 *                                                        tab_cbrt_rat)
 *   RGB -> HSI      arctan(sqrt(3) x) -> P_n(|x|)       (Table tab_arctan)
 *   RGB -> SCT      arccos, arctan -> polynomials       (Tables tab_arcsin,
 *                                                        tab_arccos, tab_f, tab_g)
 * and compares them with trilinear, prism, pyramidal and tetrahedral
 * interpolation in a 3D lookup table (Section "Comparison with 3D Lookup
 * Table Interpolation Methods").
 *
 * Conventions for every entry point:
 *  - Pointers named d_* and the pointers inside mact_image are pointers the
 *    kernels dereference: device memory of the current CUDA device, or host
 *    memory mapped into its address space (cudaHostAlloc, cudaHostRegister;
 *    and, where mact_host_memory_access returns 1, any host memory).  On host
 *    memory the kernels read and write across the host link themselves, with
 *    no staging copy, so their speed is the link's (about 190 GB/s
 *    device-to-host on a Grace-hosted GB300) rather than HBM's.  Where the
 *    device cannot address pageable memory, every such pointer is checked
 *    before launch and unregistered host memory is rejected with
 *    MACT_E_INVAL.  Functions that take a pointer written by the host (an
 *    eps_avg, a ticket) say so.  The caller owns every image, LUT and output
 *    buffer; the library never frees them.
 *  - A handle owns a small device block (gamma table, coefficients) created on
 *    the device that is current when mact_create is called; use the handle on
 *    that device only.
 *  - Work is enqueued on the given stream (a cudaStream_t cast to
 *    mact_stream; NULL is the legacy default stream) and returns before it
 *    completes.  Argument errors are reported synchronously and enqueue
 *    nothing.  A CUDA launch error returns MACT_E_CUDA; the text of the last
 *    error of the calling thread is available from mact_last_error().
 *  - No C++ exception crosses this interface.
 *  - Input is interleaved 8-bit R'G'B' (3 bytes per pixel).  Output is three
 *    planes, FP32 or FP16:
 *      CIELAB: L*, a*, b* in CIE units (white = 100, 0, 0);
 *      HSI:    H in radians [0, 2 pi), S and I in [0, 1] with R = R'/255;
 *              H = 0 where max == min (hue undefined), S = 0 for black;
 *      SCT:    L in 8-bit code units [0, 441.7], angle A and angle B in
 *              radians; black gives (0, 0, 0), R = G = 0 gives B = 0;
 *      CIELUV: L*, u*, v* in CIE 1976 units (white = 100, 0, 0); black
 *              gives (0, 0, 0).
 */
#ifndef MACT_H
#define MACT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mact_ctx *mact_handle;
typedef struct mact_server *mact_server_t;
typedef struct mact_batch_plan *mact_batch_plan_t;
typedef void *mact_stream; /* cudaStream_t */

typedef enum {
    MACT_OK = 0,
    MACT_E_INVAL = -1,       /* bad argument: null pointer, size, enum, degree */
    MACT_E_NOMEM = -2,       /* device memory or admission budget exhausted */
    MACT_E_CUDA = -3,        /* a CUDA call failed; see mact_last_error() */
    MACT_E_UNSUPPORTED = -4, /* valid request this build does not implement */
    MACT_E_TIMEOUT = -5,     /* a bounded wait ran out */
    MACT_E_BUSY = -6         /* no free slot; retry later */
} mact_status;

/* MACT_CIELUV: CIE 1976 L*u*v*, the variant the paper's Conclusions name
 * (the same cube-root approximant in L*; u* = 13 L* (u' - u'n),
 * v* = 13 L* (v' - v'n), u' = 4X / (X + 15Y + 3Z), v' = 9Y / (X + 15Y + 3Z)). */
typedef enum { MACT_CIELAB = 0, MACT_HSI = 1, MACT_SCT = 2, MACT_CIELUV = 3 } mact_space;
typedef enum { MACT_F32 = 0, MACT_F16 = 1 } mact_dtype;
typedef enum { MACT_TRILINEAR = 0, MACT_PRISM = 1, MACT_PYRAMID = 2, MACT_TETRA = 3 } mact_interp;

/* Source RGB definition (Eq. equ_rgb_lin, equ_rgb_xyz and the D65 white of
 * Section "Color Space Description", CIELAB).  Inverse gamma:
 *   k = k'/slope                                  if k' < threshold
 *   k = ((k' + offset)/(1 + offset))^exponent     otherwise,   k' = code/255.
 * rgb_to_xyz is row-major (X row first).  white = (X0, Y0, Z0). */
typedef struct {
    double gamma_threshold; /* 0.081 */
    double gamma_slope;     /* 4.5 */
    double gamma_offset;    /* 0.099 */
    double gamma_exponent;  /* 1/0.45 */
    double rgb_to_xyz[9];   /* BT.709 */
    double white[3];        /* D65: 0.950456, 1.0, 1.089058 */
} mact_rgb_def;

/* Transform configuration.
 *  exact      0: MACT approximants; 1: the exact functions (cbrtf, atan2f,
 *             acosf, sqrtf) -- the "plain" form the paper times as "exact".
 *  lab_n, lab_m  cube-root approximant: lab_m > 0 selects the rational (n, m)
 *             of Table tab_cbrt_rat (2 <= n, m <= 4, the nine printed pairs);
 *             lab_m == 0 selects the polynomial of degree lab_n (2..5) of
 *             Table tab_cbrt_poly.  Default (4, 4).
 *  hsi_n      degree 2..5 of the arctan(sqrt(3) x) polynomial.  Default 5.
 *  hsi_coeffs 0: minimax fit on [0, 1], computed by the library at create
 *             time (|x| = 1 occurs in Kender's formula); 1: Table tab_arctan
 *             as printed (n = 2 with a2 = -7.497879e-01).  Default 0.
 *  sct_n, sct_m, sct_r  degrees (4 or 5) of the arcsin, arccos and f/g
 *             polynomials (Tables tab_arcsin, tab_arccos, tab_f, tab_g).
 *             Default (5, 5, 5).
 *  lab_coeffs 0: the cube-root coefficients of the tables, as printed
 *             (default).  1: the minimax rational p_n/q_m of t^(1/3) on
 *             [0.008856, 1] (Figure fig_cbrt's interval) fitted by the
 *             library's own Remez exchange at create time, for any
 *             1 <= lab_n, lab_m <= 6 -- degrees the table does not print
 *             (the paper has no counterpart beyond (4, 4)); MACT_E_UNSUPPORTED
 *             if the exchange does not converge.  Evaluated like the printed
 *             rationals (f = 1 + (p - q)/q in FP32). */
typedef struct {
    mact_rgb_def rgb;
    int32_t exact;
    int32_t lab_n, lab_m;
    int32_t hsi_n;
    int32_t hsi_coeffs;
    int32_t sct_n, sct_m, sct_r;
    int32_t lab_coeffs;
} mact_config;

/* One image.  rgb: pointer (device, or host memory the device addresses) to
 * height rows of width interleaved pixels, rows pitch_bytes apart
 * (>= 3*width; any byte alignment).  out[c]: pointers of the same kind to
 * the three output planes, rows out_pitch_elems elements apart (>= width),
 * element type given by dtype; each must be aligned to its element size
 * (4 bytes FP32, 2 bytes FP16), else MACT_E_INVAL before any launch.
 * space: mact_space; dtype: mact_dtype.  width or height 0 is an empty
 * image; at most 2^42 pixels.  Fastest when rgb is 16-byte aligned,
 * pitch_bytes == 3*width, out_pitch_elems == width and every out[c] is
 * 16-byte aligned; planes aligned only to their element size (three
 * adjacent planes of an odd pixel count) take a shared-memory transpose
 * path, and every other layout a guarded path, all with identical values. */
typedef struct {
    const uint8_t *rgb;
    int64_t width, height, pitch_bytes;
    int32_t space;
    int32_t dtype;
    void *out[3];
    int64_t out_pitch_elems;
} mact_image;

/* Fill *cfg with the paper's defaults: BT.709 + D65, CIELAB (4,4), HSI n=5 on
 * [0,1], SCT (5,5,5), approximants on. */
void mact_config_default(mact_config *cfg);

/* Validate *cfg and build a handle on the current device.  Rejects unknown
 * degrees, any RGB definition for which white maps to t > 1 + 1e-6 or a
 * non-positive white component (the cube-root approximants are fitted on
 * [0.008856, 1], Figure fig_cbrt), and gamma parameters whose linearised
 * codes are not finite, non-decreasing and within [0, 1].  These checks run
 * on the host before any CUDA call (MACT_E_INVAL).  Allocates about 4 KB of
 * device memory.  *out is written only on success. */
mact_status mact_create(const mact_config *cfg, mact_handle *out);

/* Free the handle's device block.  Work already enqueued with the handle must
 * have completed (the call synchronises the device before freeing).  Servers
 * and batch plans created from h keep using it: destroy them first (the
 * handle does not track them, so freeing it under them is undefined). */
mact_status mact_destroy(mact_handle h);

/* Convert one image to img->space (Sections "CIELAB Color Space", "HSI
 * Color Space", "Spherical Coordinate Transform").  Asynchronous on stream.
 * width or height 0 is a valid empty image (nothing is launched). */
mact_status mact_convert(mact_handle h, const mact_image *img, mact_stream stream);

/* Convert count images of any sizes, spaces and dtypes in ONE launch of a
 * persistent kernel that walks a tile work list (the batched form; Section
 * "Calculation of the Computational Gain Values" runs the transforms over an
 * image set).  Tiles are 4096 pixels (or the autotuned shape, see
 * mact_autotune_batch).  With at most 32 non-empty images the work list is
 * passed by value in the kernel's parameters: the call makes no copy, takes
 * no device memory and never waits on the host, and CTAs take tiles
 * grid-stride.  Longer lists are uploaded from pinned staging into one of 4
 * device slots owned by the handle (grown on demand), and CTAs claim tiles
 * with an atomic counter; up to 4 consecutive calls pipeline, and a slot is
 * reused only after its previous call's copy and kernel are done (the call
 * may wait on the host for that).  Result of each image equals mact_convert
 * of that image. */
mact_status mact_convert_batch(mact_handle h, const mact_image *imgs, int32_t count,
                               mact_stream stream);

/* ---- batched form for a repeated image list ------------------------------
 * A plan fixes one list of images (the pointers, sizes, spaces and dtypes of
 * imgs at creation) and the handle's current batch launch shape.  Creation
 * validates the list and uploads its device work list once (synchronously);
 * each launch is then one kernel with no host work, no copy and no
 * allocation, so it may be captured into a CUDA graph.  The images' contents
 * may change between launches; their addresses and shapes may not.  Launches
 * of one plan must not overlap on the GPU (they share the plan's counters). */
mact_status mact_batch_plan_create(mact_handle h, const mact_image *imgs, int32_t count, mact_batch_plan_t *out);

/* Launch the plan on stream (the same kernel as mact_convert_batch). */
mact_status mact_batch_plan_launch(mact_batch_plan_t plan, mact_stream stream);

/* Launch the plan through a CUDA graph: the first call captures one launch
 * on a private stream and instantiates the graph; every call replays it on
 * stream. */
mact_status mact_batch_plan_graph_launch(mact_batch_plan_t plan, mact_stream stream);

/* Free the plan (synchronises the device first). */
mact_status mact_batch_plan_destroy(mact_batch_plan_t plan);

/* One timed launch shape of the batched kernel. */
typedef struct {
    int32_t threads;        /* threads per CTA */
    int32_t px_per_thread;  /* pixels per thread per tile (tile = threads * px_per_thread) */
    int32_t ctas_per_sm;    /* resident CTAs per SM of the persistent grid */
    float ms;               /* mean time of one launch over imgs */
} mact_tune_entry;

/* Autotuner: time every supported launch shape of the batched kernel
 * (threads per CTA 128/256/512, 16 or 32 pixels per thread, full or half
 * residency) on the caller's images (reps launches each, after 2 warm-ups,
 * on a private stream; the images are converted repeatedly), keep the fastest
 * as the handle's batch shape (used by mact_convert_batch and later plans),
 * and report up to table_cap timings in table. */
mact_status mact_autotune_batch(mact_handle h, const mact_image *imgs, int32_t count, int32_t reps,
                                mact_tune_entry *table, int32_t table_cap, int32_t *n_entries);

/* Set / read the handle's batch launch shape directly (for example from a
 * cached autotuning result).  Unsupported shapes give MACT_E_UNSUPPORTED;
 * ctas_per_sm 0 means as many as fit. */
mact_status mact_set_batch_shape(mact_handle h, int32_t threads, int32_t px_per_thread, int32_t ctas_per_sm);
mact_status mact_get_batch_shape(mact_handle h, int32_t *threads, int32_t *px_per_thread, int32_t *ctas_per_sm);

/* Same result as mact_convert_batch, without any memory allocation.  The
 * paper has no counterpart: this exists for callers that cannot allocate
 * device or pinned memory at call time -- real-time or certified pipelines
 * whose memory is fixed at start-up, plug-ins and host callbacks that must
 * not enter the allocator, processes whose device memory is fully held by
 * another framework's pool.  The work list (at most 1024 images; count above
 * that returns MACT_E_INVAL) and the tile counters live in a fixed array of
 * about 90 KB compiled into the library; every GPU that loads the library
 * keeps it until the process exits.  The first call on a device that uses
 * the array looks up its device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture begins.
 * The current device must be the handle's device, else MACT_E_INVAL.
 * The launch shape is the handle's batch shape, as for mact_convert_batch.
 * Lists of more than 32 non-empty images are written into the array by small
 * upload kernels whose parameters carry the descriptors (no host buffer is
 * read after the call returns), the first of which zeroes the tile counters;
 * shorter lists go by value to the batched kernel and use no array at all.
 * Every call shares the one array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (different streams, or different
 * handles, at the same time) race and must be serialised by the caller.
 * Calls from several host threads are serialised by the library. */
mact_status mact_convert_batch_static(mact_handle h, const mact_image *imgs, int32_t count,
                                      mact_stream stream);

/* Packing step of the LUT methods: fill d_lut (n^3 x 3 FP32, layout
 * d_lut[((i*n + j)*n + k)*3 + c], R outermost) with the exact CIELAB of the
 * node codes 255*(i,j,k)/(n-1), computed in FP64 (cbrt) on the device and
 * rounded once to FP32.  2 <= n <= 64; d_lut 4-byte aligned, else
 * MACT_E_INVAL. */
mact_status mact_lut_build(mact_handle h, int32_t n, float *d_lut, mact_stream stream);

/* Extraction + interpolation (Section "Comparison with 3D Lookup Table
 * Interpolation Methods"): for each of npix interleaved pixels of d_rgb, the
 * cell along each axis is idx = v(n-1) div 255 with remainder
 * rem = v(n-1) mod 255 (v = 255 uses idx = n-2, rem = 255) and the fraction
 * is rem/255; method picks the 8-node trilinear, 6-node prism (axis R),
 * 5-node pyramid (apex at the far corner, base = face of the smallest
 * fraction) or 4-node tetrahedron (ordering of the remainders).  The three
 * interpolated values go to d_out[0..2] (FP32, npix each).  If d_sel is not
 * NULL it receives, per pixel, (lower-corner node index)*8 + simplex id.
 * d_lut layout as in mact_lut_build, 2 <= n <= 64. */
mact_status mact_lut_interp(mact_handle h, int32_t method, const float *d_lut, int32_t n,
                            const uint8_t *d_rgb, int64_t npix, float *const d_out[3],
                            int32_t *d_sel, mact_stream stream);

/* The LUT in the layout the interpolation kernels read, for repeated
 * interpolation: d_packed holds 19 n^3 floats, owned by the caller and
 * 16-byte aligned (else MACT_E_INVAL).  With m = n^3 and node
 * i = ((i_R n + i_G) n + i_B):
 *   floats [0, 4m): node i as (x, y, z, 0);
 *   floats [4m, 8m): B edges, (x_i, y_i, x_j, y_j) with j = i + 1, the next
 *     node along B (the last node of a B row repeats itself);
 *   floats [8m, 12m): R edges, the same with j = i + n^2;
 *   floats [12m, 14m): B edges, (z_i, z_j);  [14m, 16m): R edges, (z_i, z_j);
 *   floats [16m, 18m): node i as (x, y);  [18m, 19m): node i's z.
 * A LUT with n <= 17 is staged whole in every CTA's shared memory from the
 * nodes; a larger one (33^3: 575 KB of nodes) is read through L1:
 * trilinear as 4 B edges, prism as 3 R edges (fewer bytes for the same
 * loads), the pyramid as single nodes from the xy and z planes, tetrahedral
 * as 16-byte nodes.
 * mact_lut_interp repacks such a LUT into handle scratch on every call (and
 * orders calls on one handle that share that scratch); packing once with
 * mact_lut_pack and calling mact_lut_interp_packed avoids both.  The paper
 * has no counterpart: it is a memory layout of the same LUT. */
mact_status mact_lut_pack(mact_handle h, const float *d_lut, int32_t n, float *d_packed, mact_stream stream);

/* mact_lut_interp on a packed LUT (d_packed from mact_lut_pack): the same
 * cells, simplices, selection ids and values. */
mact_status mact_lut_interp_packed(mact_handle h, int32_t method, const float *d_packed, int32_t n,
                                   const uint8_t *d_rgb, int64_t npix, float *const d_out[3],
                                   int32_t *d_sel, mact_stream stream);

/* ---- differentiable RGB -> CIELAB ----------------------------------------
 * Input d_x is LINEAR RGB (the output of Eq. equ_rgb_lin, e.g. a network's
 * activations) as planar FP32 of shape (nbatch, 3, hw): plane c of image b
 * starts at d_x + (b*3 + c)*hw.  Lab uses Eq. equ_rgb_xyz and equ_xyz_lab
 * with the handle's cube-root rational (or cbrtf when created with exact = 1);
 * the backward differentiates exactly what the forward evaluates, including
 * the linear segment (slope 7.787) for t <= 0.008856.  Handles using the
 * cube-root polynomials (lab_m = 0) return MACT_E_UNSUPPORTED.  At most
 * 2^31 pixels (nbatch * hw) per call; larger calls give MACT_E_INVAL before
 * any launch.  Fastest when hw % 4 == 0 and every pointer is 16-byte
 * aligned. */

/* d_lab (nbatch, 3, hw) = CIELAB of d_x. */
mact_status mact_lab_forward(mact_handle h, const float *d_x, int64_t nbatch, int64_t hw, float *d_lab,
                             mact_stream stream);

/* d_grad_x = J(d_x)^T d_grad_lab: the vector-Jacobian product of the
 * forward at d_x (recomputed, nothing saved), shapes (nbatch, 3, hw). */
mact_status mact_lab_backward(mact_handle h, const float *d_x, const float *d_grad_lab, int64_t nbatch,
                              int64_t hw, float *d_grad_x, mact_stream stream);

/* Fused forward + loss + backward: *d_loss (one device float) = mean over
 * pixels of Delta E*ab (Eq. equ_cielab_dist) between Lab(d_x) and
 * d_target_lab (nbatch, 3, hw); if d_grad_x is not NULL it receives
 * dLoss/dx (0 where Delta E = 0).  The mean is reduced in a fixed order
 * (deterministic).  Uses a small per-handle partial-sum buffer; calls on one
 * handle are ordered by the library. */
mact_status mact_lab_delta_e_loss(mact_handle h, const float *d_x, const float *d_target_lab, int64_t nbatch,
                                  int64_t hw, float *d_loss, float *d_grad_x, mact_stream stream);

/* ---- served form -------------------------------------------------------
 * A conversion server with continuous batching (the paper has no serving
 * layer; its transforms are what each request runs).  One scheduler thread
 * per server admits queued requests in arrival order while a slot is free,
 * the input and output bytes of all admitted, unfinished requests stay
 * within mem_budget_bytes (in either mode, whether their buffers are used in
 * place or staged), and, for staged buffers, the staging arena
 * (mem_budget_bytes of device memory, allocated once by mact_serve_create)
 * has room for the request's staged input and output;
 * converts every request admitted in one tick with one launch of the batched
 * kernel (as mact_convert_batch), and copies results back, on three streams
 * (H2D, compute, D2H) so the copies of one tick overlap the kernel of
 * another.  Requests that arrive while others are on the GPU join the next
 * tick.  The result of each request equals mact_convert of that image.
 *
 * Host buffers: in direct mode (the default) the kernel reads and writes host
 * buffers it can address (pinned memory, and any host memory where
 * mact_host_memory_access returns 1) in place, across the host link, with no
 * staging and no copy; other host buffers are staged.  In staged mode every
 * host buffer is staged: input copied into the arena, output copied back. */

enum { MACT_SERVE_DIRECT = 0, MACT_SERVE_STAGED = 1 };

typedef struct {
    int64_t completed;   /* requests finished successfully */
    int64_t failed;      /* requests whose copies or launch failed */
    int64_t batches;     /* batched launches issued */
    int64_t queued;      /* waiting for admission now */
    int64_t in_flight;   /* admitted, not yet retired */
    int64_t pixels;      /* pixels of the completed requests */
    double p50_ms, p99_ms, max_ms;  /* submit-to-completion latency of completed requests */
    double gpix_per_s;   /* completed pixels / (last completion - first submit) */
    /* Stages of that latency, median and 99th percentile over the completed
     * requests: queue = submit to admission (host clock); h2d = the batch's
     * input copies; compute = from the end of those copies to the end of the
     * batch's kernel (waits for the compute stream included); d2h = from the
     * end of the kernel to the end of the request's output copy (waits behind
     * earlier output copies included).  The device stages are CUDA-event
     * times. */
    double queue_p50_ms, h2d_p50_ms, compute_p50_ms, d2h_p50_ms;
    double queue_p99_ms, h2d_p99_ms, compute_p99_ms, d2h_p99_ms;
    /* Output copies to host memory: summed copy time (from the moment the
     * D2H stream reaches a request's copies to their end) and the bandwidth
     * they ran at (bytes / that time). */
    double d2h_busy_ms, d2h_copy_gbs;
    /* Largest sum of admitted requests' input and output bytes seen (never
     * above the budget). */
    int64_t inflight_bytes_max;
} mact_serve_stats_t;

/* Create a server for handle h (on h's device), in direct mode.  max_slots
 * bounds the number of admitted, unfinished requests (1..65536);
 * mem_budget_bytes (>= 4096) bounds the input and output bytes of the
 * admitted requests, and is the size of the staging arena.
 * A tick that fails leaves its requests failed (MACT_E_CUDA from poll and
 * wait, with the reason in mact_last_error) and returns their staging
 * memory once the server's streams have drained.  For testing that path,
 * the environment variable MACT_SERVE_FAIL_EVERY=k, read here, fails every
 * k-th batch on the host after its input copies are enqueued. */
mact_status mact_serve_create(mact_handle h, size_t mem_budget_bytes, int32_t max_slots, mact_server_t *out);

/* How host buffers of requests submitted from now on are used:
 * MACT_SERVE_DIRECT or MACT_SERVE_STAGED (see above).  MACT_E_INVAL for
 * another value. */
mact_status mact_serve_set_mode(mact_server_t srv, int32_t mode);

/* Queue one image.  img->rgb and img->out[] may each be host memory (pinned
 * is fastest; staged pageable memory works but its copies block the
 * scheduler) or device memory.  The buffers must stay valid until the
 * request is done.  Returns a ticket.  MACT_E_NOMEM if the
 * request's input and output alone exceed the whole budget; MACT_E_BUSY once
 * the server is shutting down. */
mact_status mact_serve_submit(mact_server_t srv, const mact_image *img, uint64_t *ticket);

/* Non-blocking status: *done = 1 once the request has finished (its outputs
 * are written), failed, or was cancelled; *latency_ms = submit to
 * completion.  Returns MACT_E_CUDA for a failed request. */
mact_status mact_serve_poll(mact_server_t srv, uint64_t ticket, int32_t *done, double *latency_ms);

/* Block until the request is done or timeout_ms passes (MACT_E_TIMEOUT). */
mact_status mact_serve_wait(mact_server_t srv, uint64_t ticket, double timeout_ms, double *latency_ms);

/* Cancel a request that has not been admitted yet (MACT_E_BUSY once it has). */
mact_status mact_serve_cancel(mact_server_t srv, uint64_t ticket);

/* Forget a finished request's record (MACT_E_BUSY while it is pending). */
mact_status mact_serve_release(mact_server_t srv, uint64_t ticket);

/* Counters and latency percentiles over the requests completed so far. */
mact_status mact_serve_stats(mact_server_t srv, mact_serve_stats_t *out);

/* Stop accepting requests, wait up to timeout_ms for queued and in-flight
 * requests to finish, cancel any still queued after that (MACT_E_TIMEOUT),
 * wait for in-flight work, and free the server. */
mact_status mact_serve_destroy(mact_server_t srv, double timeout_ms);

/* ---- transformation error over every 24-bit colour -----------------------
 * Section "Calculation of the Color Space Transformation Errors" (Tables
 * tab_cielab, tab_hsi, tab_sct, tab_lut): the average and maximum distance,
 * over all 2^24 colours, between the transform the library computes (the
 * production FP32 kernel) and the exact transform evaluated in FP64 on the
 * device.  The distance is Delta E*ab (Eq. equ_cielab_dist) for CIELAB,
 * D_HSI (Eq. equ_hsi_dist) for HSI, and for SCT Delta E*ab after the inverse
 * SCT (Eq. equ_sct_rgb) and conversion to CIELAB.  Colours are generated
 * from their index (no input).  Blocking; allocates a few KB (and, for
 * LUTs, an n^3 float4 copy) for the duration of the call. */

/* Error of the handle's transform to space (MACT or exact per the handle). */
mact_status mact_cube_error(mact_handle h, int32_t space, double *eps_avg, double *eps_max);

/* Error of LUT interpolation (d_lut as for mact_lut_interp) against the
 * exact CIELAB. */
mact_status mact_cube_error_lut(mact_handle h, int32_t method, const float *d_lut, int32_t n, double *eps_avg,
                                double *eps_max);

/* ---- "caching" LUT layout --------------------------------------------
 * Section "Comparison with 3D Lookup Table Interpolation Methods": besides
 * the standard form, the paper implements each LUT method in a "caching"
 * form that precomputes the differences between neighbouring lattice nodes
 * and stores them with each node.  Here each cell (lower corner (i, j, k),
 * 0 <= i, j, k <= n-2) gets one 128-byte record of 8 float4: c000 and the
 * seven differences c_xyz - c000 (slot x*4 + y*2 + z; x = R, y = G, z = B;
 * the fourth lane unused), so a pixel's neighbourhood is one cache line.
 * d_cache must hold (n-1)^3 * 32 floats and be 16-byte aligned. */
mact_status mact_lut_cache_build(mact_handle h, const float *d_lut, int32_t n, float *d_cache, mact_stream stream);

/* Interpolation from the caching layout: same methods, the same cells,
 * simplices and selection ids as mact_lut_interp, the same values up to FP32
 * rounding (c000 + weighted differences). */
mact_status mact_lut_interp_cached(mact_handle h, int32_t method, const float *d_cache, int32_t n,
                                   const uint8_t *d_rgb, int64_t npix, float *const d_out[3], int32_t *d_sel,
                                   mact_stream stream);

/* ---- HSI LUT with angular hue interpolation -----------------------------
 * The closing paragraphs of Section "Comparison with 3D Lookup Table
 * Interpolation Methods": a LUT of an angular space must mix hues as angles,
 * Eq. equ_angular, theta = atan2((1-a) sin t0 + a sin t1, (1-a) cos t0 +
 * a cos t1); the paper reports trilinear HSI interpolation built on it.  The
 * paper states the pairwise formula only; here S and I take the trilinear
 * weights and H is mixed pairwise along B, then G, then R, a gray node
 * (S = 0) carrying no hue (its pair takes the other angle), and a result with
 * S = 0 takes H = 0.  A pair of antipodal hues mixed near a = 0.5 has no
 * direction and is treated as gray. */

/* Build the n^3-node HSI LUT (2 <= n <= 64) at k' = (i, j, k)/(n-1), R
 * outermost: node = float4 (cos H, sin H, S, I) of the exact HSI
 * (Eq. equ_rgb_kender), each of H, S, I rounded to FP32 first; gray nodes
 * hold (0, 0, 0, I).  d_lut4: n^3 * 4 floats, 16-byte aligned. */
mact_status mact_lut_build_hsi(mact_handle h, int32_t n, float *d_lut4, mact_stream stream);

/* Trilinear interpolation of npix interleaved uint8 pixels in an HSI LUT
 * built by mact_lut_build_hsi: d_out[0] = H (radians, [0, 2 pi)),
 * d_out[1] = S, d_out[2] = I, FP32 planes of npix elements (4-byte aligned).
 * Cells are selected by the same integer extraction as mact_lut_interp. */
mact_status mact_lut_interp_hsi(mact_handle h, const float *d_lut4, int32_t n, const uint8_t *d_rgb, int64_t npix,
                                float *const d_out[3], mact_stream stream);

/* Which host memory the kernels of handle h may be given (the paper has no
 * counterpart: it concerns where the pixels live, not how they are
 * converted).  Returns 1 when the device addresses any host memory through
 * the host page tables (cudaDevAttrPageableMemoryAccess, e.g. a Grace-hosted
 * GB300): pointers are then not checked.  Returns 0 when only device memory
 * and pinned or registered host memory may be given: every pointer argument
 * is then checked with cudaPointerGetAttributes before launch.  Setting the
 * environment variable MACT_CHECK_HOST_POINTERS to a value other than "0"
 * before mact_create forces 0.  MACT_E_INVAL for a NULL handle. */
int32_t mact_host_memory_access(mact_handle h);

/* ---- host-side minimax fits (no device work, no handle) -----------------
 * The coefficient fits mact_create performs on the host, for inspection and
 * for callers that cache them.  Both are Remez exchanges written for this
 * library; the results equioscillate at n + m + 2 (rational) or n + 2
 * (polynomial) points. */

/* Minimax rational p_n/q_m of t^(1/3) on [0.008856, 1] (Section
 * "Approximation of the Cube-Root Function"; the form of Table
 * tab_cbrt_rat, any degrees 1 <= n, m <= 6), normalised to q(0) = 1: what
 * mact_config.lab_coeffs = 1 evaluates.  p and q (7 doubles each, caller
 * owned) receive the ascending coefficients, zero-padded; *max_err (may be
 * NULL) the levelled maximum absolute error.  MACT_E_INVAL for other degrees
 * or NULL p or q; MACT_E_UNSUPPORTED if the exchange does not converge. */
mact_status mact_fit_cbrt_rational(int32_t n, int32_t m, double *p, double *q, double *max_err);

/* Minimax polynomial P_n of arctan(sqrt(3) x) on [0, 1] (Section
 * "Approximation of the Inverse Tangent Function", the degrees 2..5 of
 * Table tab_arctan): the HSI set of mact_config.hsi_coeffs = 0.  c (6
 * doubles, caller owned) receives the ascending coefficients, zero-padded;
 * *max_err (may be NULL) the levelled maximum absolute error.  MACT_E_INVAL
 * for other degrees or NULL c; MACT_E_UNSUPPORTED if the exchange fails. */
mact_status mact_fit_hsi_arctan(int32_t n, double *c, double *max_err);

/* Message for a status code (static storage). */
const char *mact_strerror(mact_status st);

/* Text of the last error raised on the calling thread ("" if none). */
const char *mact_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MACT_H */
