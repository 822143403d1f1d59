/*
 * blink.h - C ABI of the GB300 (sm_103a) dirty-imaging library: BLINK's data-parallel hot path
 * (arXiv 2505.15204): 4-bit tile voltages -> correlation -> uv gridding -> batched 2D inverse FFT ->
 * dirty images, on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers prefixed d_ are device memory owned by the caller (for example PyTorch tensors); pointers
 *   prefixed h_ and the pointers inside the descriptor structs are host memory owned by the caller and
 *   read only during the call, with two exceptions stated where they apply: page-locked calibration
 *   tables (array.gains, array.jones) and blink_pipeline_host's page-locked or device-writable buffers
 *   are used by work still queued on the stream.  The library keeps no other pointer to caller memory
 *   after returning.
 * - Calls are asynchronous and ordered on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *   default stream).  Argument errors are reported synchronously through the return value, and nothing
 *   is launched.  Device-side errors (a failed index guard, a bounded wait that ran out) are recorded
 *   in a per-context status word and reported by blink_sync().
 * - No call aborts or throws across the ABI.  blink_last_error() returns the calling thread's last
 *   error message.
 * - A context is used by one host thread at a time, and its calls share its device workspace: calls on
 *   different streams must be ordered between those streams (an event), or use separate contexts.
 * - One device per process: kernel attributes (shared-memory limits, occupancy) are set once per process
 *   for the first device that launches them, so contexts on several GPUs need one process each (the
 *   library's multi-GPU model: one process per GPU, sharding by chunk).
 * - The library allocates device memory only inside the context: per-configuration plans (cell maps,
 *   gather lists) on first use, and workspace that grows to the largest request seen.  A repeated call
 *   with the same configuration allocates nothing.
 *
 * Data layouts
 * ------------
 * voltages  uint8 [n_samples][fine_stride][n_tiles][2]: one byte per complex sample and polarisation
 *           (last axis X, Y), re = low nibble, im = high nibble, both two's-complement in [-8, 7].
 *           The channels of one call are n_fine consecutive channels of that axis; d_volt points at
 *           the first of them in sample 0.
 * baselines b = i(i+1)/2 + j for tiles i >= j (autocorrelations included); B = n_tiles(n_tiles+1)/2.
 * images    id = tau * F + f for integration tau (T = n_samples / samples_per_int) and output channel
 *           f (F = n_fine / chan_avg).
 * vis       float [T][F][B][4][2]: complex64 per polarisation product XX, XY, YX, YY, V = S / K with
 *           S the integer sum of x_i^p conj(x_j^q) and K = samples_per_int * chan_avg.
 * grid      float [n_images][N][N/2 + 1][2]: the u >= 0 half of the Hermitian uv grid, row = v
 *           (index mod N), column = u, DC at [0][0]; the u < 0 half is G(-u,-v) = conj G(u,v).
 * image     float [n_images][N][N]: row y (direction cosine m), column x (l); pixel (N/2, N/2) is the
 *           phase centre; l = (x - N/2) / (N du), m = (y - N/2) / (N du).
 */
#ifndef BLINK_H
#define BLINK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BLINK_OK = 0,
    BLINK_ERR_INVALID_ARG = 1,   /* a pointer, size or layout violates the rules of the call */
    BLINK_ERR_UNSUPPORTED = 2,   /* valid request outside what this build implements (e.g. image side) */
    BLINK_ERR_OOM = 3,           /* device allocation for a plan or workspace failed */
    BLINK_ERR_CUDA = 4,          /* a CUDA runtime call failed; the message names it */
    BLINK_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out (reported by blink_sync) */
    BLINK_ERR_DEVICE = 6         /* a device-side index or size guard failed (reported by blink_sync) */
} blink_status;

enum { BLINK_POL_I = 0, BLINK_POL_XX = 1 };            /* imaged polarisation */
enum { BLINK_CORR_FP32 = 0, BLINK_CORR_FP8 = 1 };      /* correlation arithmetic */
enum { BLINK_PREC_FP32 = 0, BLINK_PREC_BF16 = 1 };     /* grid / FFT intermediate storage */
enum { BLINK_MODE_BATCHED = 0, BLINK_MODE_PLAIN = 1 }; /* pipeline form */

typedef struct blink_context blink_context;

/* The array (Sec. 5.2.3-5.2.4: tile positions are the metadata the imager uses for (u, v, w)). */
typedef struct {
    int32_t n_tiles;            /* 1..512 */
    const double* enu_m;        /* host [n_tiles][3]: East, North, Up in metres */
    const uint8_t* flags;       /* host [n_tiles], non-zero = flagged (excluded); NULL = none flagged */
    const float* gains;         /* host [F][n_tiles][2 pol][2] (re, im) or NULL: calibration (Sec. 5.2.3), a
                                   diagonal Jones matrix per output channel and tile, applied to the products
                                   as V_ij^pq = g_i^p S_ij^pq conj(g_j^q) inside the correlation; F = the call's
                                   output channels (obs.n_fine / obs.chan_avg, for blink_pipeline_sets over
                                   the call's whole channel axis).  Copied to the device on `stream` by
                                   an asynchronous copy: pageable memory is read before the call returns,
                                   page-locked memory when the stream reaches the copy (keep it unchanged
                                   until then; under graph capture every replay reads its contents anew). */
    const float* jones;         /* host [F][n_tiles][2][2][2] (J[p][r] re, im) or NULL: full 2x2 Jones matrices
                                   (polarisation leakage included), V_ij = J_i S_ij J_j^H; takes precedence
                                   over gains; Stokes I and XX then need all four products.  Copied like
                                   gains. */
} blink_array;

/* The observation (Sec. 5.2.1-5.2.2 and the -t / -c options of the pipeline's command line). */
typedef struct {
    int32_t n_fine;             /* fine channels processed by the call */
    int32_t fine_stride;        /* fine channels per sample in the voltage buffer; 0 means n_fine */
    const double* fine_freq_hz; /* host [n_fine]: centre frequency of each processed fine channel */
    int32_t chan_avg;           /* c: consecutive fine channels averaged into one output channel (-c) */
    int32_t samples_per_int;    /* N_s: voltage samples per integration (-t / sample time) */
    int32_t n_samples;          /* samples in the buffer; a multiple of samples_per_int */
} blink_obs;

/* Imaging parameters (Sec. 5.2.4 and the -n option). */
typedef struct {
    int32_t n_pix;              /* N: image and grid side, even, in [64, 8192], with no prime factor above 5
                                   (e.g. 256, 512, 1200, 8192).  Powers of two up to 2048 run the
                                   side-specialised kernels; the other sides run mixed-radix (2, 3, 4, 5)
                                   column and row passes, two launches per wave of images. */
    double cell_lambda;         /* uv cell du in wavelengths; <= 0 selects u_max / (N/2 - 1) */
    int32_t pol;                /* BLINK_POL_I: (XX + YY) / 2; BLINK_POL_XX: XX only */
    int32_t include_autos;      /* non-zero: autocorrelations gridded at (0, 0) with weight 1 */
    int32_t precision;          /* BLINK_PREC_FP32, or BLINK_PREC_BF16 (bf16 grid/intermediate storage) */
    int32_t support;            /* gridding kernel (Sec. 5.2.4): 0 or 1 = nearest cell; W in [2, 16] = separable
                                   Kaiser-Bessel kernel of W cells, beta = pi sqrt((W/2)^2 (3/2)^2 - 0.8),
                                   on a grid of side 2 n_pix (n_pix <= 4096): every visibility is spread
                                   over the cells within W/2 of its exact (u, v) / du and kept only if that
                                   support lies inside the grid; the image is the central n_pix x n_pix of
                                   the transform divided by the kernel's Fourier transform along both axes.
                                   The default cell is then u_max / (n_pix - 1 - W/2).  Batched pipeline
                                   forms only (blink_pipeline BATCHED, blink_pipeline_sets,
                                   blink_pipeline_host); the stage calls return BLINK_ERR_UNSUPPORTED. */
    double phase_l, phase_m;    /* phase centre (Sec. 5.2.3, geometric corrections): the pointing's direction
                                   cosines (l0, m0) in the local East, North, Up frame, l0^2 + m0^2 < 1;
                                   (0, 0) = zenith.  (u, v, w) are taken in the pointing's basis (East and
                                   North carried to it by the rotation about Up x s0 that takes Up to it),
                                   every visibility is multiplied by exp(+2 pi i w) before gridding, so a
                                   source at the pointing images at pixel (N/2, N/2); the default cell uses
                                   the baselines projected on that basis.  A new pointing builds a new plan.
                                   blink_grid returns BLINK_ERR_UNSUPPORTED off zenith (its visibilities are
                                   the caller's); blink_image ignores the pointing. */
} blink_imaging;

/*
 * Stream ordering and graph capture: every entry point only enqueues work on `stream` (NULL = the legacy
 * default stream) and returns; blink_sync waits.  The first call for a new plan (array, channels and image
 * parameters) builds the plan and, in the batched form, times the persistent kernel's launch shapes on the
 * stream with a blocking event wait; make that call before any CUDA-graph capture.  Later calls with the
 * same plan and the same calibration kind (none, gains or Jones) allocate nothing and never block, so they
 * can be captured and replayed (calibration gains are copied from host memory on every call, so under
 * capture they must be page-locked).
 */

/* ---- context ---------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device` (which becomes current on the calling thread). */
blink_status blink_create(int32_t device, blink_context** out);
/* Free everything the context allocated.  Waits for its work to finish first.  NULL is a no-op. */
void blink_destroy(blink_context* ctx);
/* Message of the calling thread's last failed call ("" if none).  Valid until the next call. */
const char* blink_last_error(void);
const char* blink_status_name(blink_status status);
/* Wait for `stream`, then report (and clear) the context's device-side status word. */
blink_status blink_sync(blink_context* ctx, void* stream);
/* B = n_tiles (n_tiles + 1) / 2. */
int64_t blink_n_baselines(int32_t n_tiles);

/* ---- the hot path, one stage per call ---------------------------------------------------------- */

/*
 * Baseline geometry (Sec. 5.2.3, the geometric correction, which the paper performs inside its imager, and the
 * (u, v, w) computation of Sec. 5.2.4), in FP64 on the GPU: for every output channel f (centre = mean of
 * its chan_avg fine-channel centres) and baseline b, (u, v, w) = (r_i - r_j) * (nu_f / c) and the
 * nearest uv cell (iu, iv) = floor((u, v) / du + 1/2).  Off zenith (imaging.phase_l, phase_m) the
 * components are taken on the pointing's basis: u = (r_i - r_j).e_l nu_f / c, v = (...).e_m nu_f / c,
 * w = (...).s0 nu_f / c.  A gridding kernel (imaging.support >= 2) is rejected (BLINK_ERR_UNSUPPORTED).
 *   d_cells  int32 [F][B]: (iu & 0xFFFF) | (iv << 16) for a gridded baseline, or 0x80008000 when the
 *            baseline is flagged or falls outside |iu|, |iv| < N/2.
 *   d_uvw    double [F][B][3] or NULL.
 *   h_du     host double or NULL: receives the cell size used.
 */
blink_status blink_cells(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                         const blink_imaging* imaging, int32_t* d_cells, double* d_uvw, double* h_du,
                         void* stream);

/*
 * Correlation (Eq. 2; Sec. 5.2.2): for every integration and output channel, the lower-triangular
 * matrix of V_ij^pq = (1/K) sum x_i^p conj(x_j^q) over the N_s samples and c fine channels, as float
 * [T][F][B][4][2].  Products of 4-bit integers are summed exactly (integers below 2^24), then divided
 * by K once in IEEE FP32.  Flagged tiles' baselines are written as 0.  With array.gains the products are
 * calibrated first, V_ij^pq = g_i^p S_ij^pq conj(g_j^q) / K (FP32 arithmetic).
 *   arith  BLINK_CORR_FP32: CUDA-core FP32; BLINK_CORR_FP8: tcgen05 tensor cores, e4m3 operands,
 *          FP32 accumulation.  Without gains both give identical bits.
 */
blink_status blink_correlate(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                             int32_t arith, const uint8_t* d_volt, float* d_vis, void* stream);

/*
 * Gridding (Sec. 5.2.4): natural weighting, nearest cell, no convolution kernel.  Images
 * [first_image, first_image + n_images) of the visibility layout above are gridded; d_vis points at
 * image first_image.  Each cross baseline adds I at its cell and conj(I) at the mirror cell, each
 * autocorrelation adds I at (0, 0) (when include_autos), with I = (V_XX + V_YY) / 2 or V_XX.
 *   d_grid    float [n_images][N][N/2 + 1][2] (half plane; the Nyquist column u = N/2 is written 0).
 *   d_weight  float [n_images] or NULL: W, the sum of weights (2 per gridded cross baseline, 1 per auto).
 * The sum over a cell is taken in a fixed order, so results are bitwise reproducible.
 */
blink_status blink_grid(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                        const blink_imaging* imaging, const float* d_vis, int32_t first_image,
                        int32_t n_images, float* d_grid, float* d_weight, void* stream);

/*
 * Imaging (Eq. 4; Sec. 5.2.4): for each grid, the unnormalised inverse 2D transform
 * a[y][x] = sum G[v][u] exp(+2 pi i (u x + v y) / N) of the Hermitian grid, divided by W and shifted so
 * the phase centre is pixel (N/2, N/2).  The grid is real-valued in image space, so only Re a is formed
 * (a complex-to-real transform of the half plane).
 *   d_grid    float [n_images][N][N/2 + 1][2] as written by blink_grid.
 *   d_weight  float [n_images]: W per image (entries <= 0 are treated as 1).
 *   d_img     float [n_images][N][N].
 */
blink_status blink_image(blink_context* ctx, const blink_imaging* imaging, const float* d_grid,
                         int32_t n_images, const float* d_weight, float* d_img, void* stream);

/*
 * The whole path (Sec. 5, the imaging half of the paper's FRB search pipeline figure): correlation -> gridding ->
 * inverse FFT -> shifted, normalised dirty images for every integration and output channel of the call,
 * d_img float [T * F][N][N] in image-id order.  Only the products the imaged polarisation needs are
 * formed (XX and YY for Stokes I), calibrated with array.gains when given.
 *   arith     correlation arithmetic as in blink_correlate.
 *   mode      BLINK_MODE_BATCHED: one correlation launch and one persistent gridding + FFT launch for the
 *             whole call (the fast form; its launch shape is autotuned on a plan's first call);
 *             BLINK_MODE_PLAIN: one launch set per image with atomic gridding (the reference GPU form).
 *   d_weight  float [T * F] or NULL: W per image.
 * Images equal blink_image(blink_grid(blink_correlate(...))) up to FP32 rounding.
 */
blink_status blink_pipeline(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                            const blink_imaging* imaging, int32_t arith, int32_t mode,
                            const uint8_t* d_volt, float* d_img, float* d_weight, void* stream);

/* One set of channels imaged with its own flags and image parameters (blink_pipeline_sets). */
typedef struct {
    int32_t fine0;              /* first fine channel of the set: index into the call's channel axis */
    int32_t n_fine;             /* fine channels in the set (a multiple of obs.chan_avg) */
    const uint8_t* flags;       /* host [n_tiles] flags of this set, or NULL (array.flags is ignored) */
    blink_imaging imaging;      /* image side, cell, polarisation, autos, precision of this set */
} blink_set;

/*
 * The whole path for several sets of channels at once (the batched form of Sec. 5.2.4's parallel gridding
 * of many channels and intervals, with uneven baseline counts and image sizes): each set has its own
 * flagged tiles and image side.  obs describes the whole buffer (n_fine channels, fine_freq_hz for all of
 * them); set s covers channels [fine0, fine0 + n_fine).  Images of set s are written in the order of
 * blink_pipeline (id = tau * F_s + f) at float offset sum_{s' < s} T * F_s' * N_s'^2 of d_img.
 *   img_capacity  floats available at d_img; too small -> BLINK_ERR_INVALID_ARG before any launch.
 */
blink_status blink_pipeline_sets(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                 const blink_set* sets, int32_t n_sets, int32_t arith, const uint8_t* d_volt,
                                 float* d_img, size_t img_capacity, void* stream);

/*
 * Incoherent dedispersion of an image cube (the FRB search the images feed, Sec. 2 and 7): d_img is float
 * [n_int][n_chan][N][N] in blink_pipeline's image order (id = integration * n_chan + channel); for every
 * t < n_int - max(delays), d_out[t] = (1/n_chan) sum_f d_img[t + delays[f]][f].  All-zero delays give the
 * band-averaged image of every integration.
 *   h_delays  host int32 [n_chan], >= 0, in integrations, e.g. round(4.148808e3 s MHz^2 * DM *
 *             (nu_f^-2 - nu_top^-2) / t_int) for a dispersion measure DM in pc cm^-3 and nu in MHz.
 *   d_out     float [n_int - max(delays)][N][N].
 * N is even, in [64, 8192]; max(delays) < n_int, else BLINK_ERR_INVALID_ARG before any launch.
 */
blink_status blink_dedisperse(blink_context* ctx, const float* d_img, int32_t n_int, int32_t n_chan, int32_t n_pix,
                              const int32_t* h_delays, float* d_out, void* stream);

/*
 * Incoherent dedispersion of a stream of image cubes (Sec. 2 and 7, Table 1: the dispersive sweep of a burst
 * across the band lasts up to tens of seconds, far longer than one cube): the cubes of consecutive calls are
 * the integrations [t0, t0 + n_int) of one stream, in blink_pipeline's image order, t0 = 0 in the first call
 * and each later call's t0 the previous t0 + n_int.  With img the concatenation of all cubes and
 * D = max(delays), the output integration t is (1/n_chan) sum_f img[t + delays[f]][f], as blink_dedisperse
 * computes it on one cube; it is complete once integration t + D has been passed, and the call that passes
 * it writes it.  Each call writes the outputs t in [max(0, t0 - D), t0 + n_int - D), in order, to d_out and
 * their count to *h_n_out: n_int for every call whose t0 >= D, fewer (possibly 0) before.
 *   d_carry   device float [D][N][N], caller-owned, kept between the calls of one stream (NULL allowed when
 *             D = 0): the partial channel sums of the outputs still waiting for later cubes, D images
 *             whatever n_chan; what it holds before a call with t0 = 0 is ignored.  A stream's calls must be
 *             ordered on one stream and pass the same delays; two streams need two carry buffers.
 *   d_img     float [n_int][n_chan][N][N]; d_out float [n_int][N][N] (room for the largest count).
 *   h_delays  host int32 [n_chan], >= 0, in integrations (see blink_dedisperse).
 * Sums are FP32, in channel order within a cube and cube by cube; the result equals blink_dedisperse on the
 * concatenated cube up to that rounding.  n_int, n_chan >= 1, t0 >= 0, N even in [64, 8192], d_img, d_out
 * and d_carry 16-byte aligned, else BLINK_ERR_INVALID_ARG before any launch (*h_n_out = 0).
 */
blink_status blink_dedisperse_stream(blink_context* ctx, float* d_carry, int64_t t0, const float* d_img, int32_t n_int,
                                     int32_t n_chan, int32_t n_pix, const int32_t* h_delays, float* d_out,
                                     int32_t* h_n_out, void* stream);

/*
 * blink_pipeline on host buffers: copies h_volt to device workspace, runs the batched path and delivers
 * the images to h_img, all ordered on `stream`.
 *   images_per_pass == 0: when the device can write h_img - one page-locked allocation (cudaHostAlloc,
 *     cudaHostRegister), or pageable memory on a device that reaches it through the host's page tables
 *     (hardware-coherent links such as NVLink-C2C) - the imaging kernel writes the images straight into it,
 *     overlapping the transfer with the computation; otherwise all images are staged in device memory and
 *     copied back.
 *   images_per_pass >= 1: the images are staged and copied back in passes of at most that many (bounding
 *     the device image buffer).
 * Page-locked or directly written buffers make the call asynchronous: it returns after enqueueing
 * (blink_sync waits); a pageable buffer written directly must stay allocated until then.
 *   h_volt  host uint8 as the voltage layout (fine_stride channels per sample).
 *   h_img   host float [T * F][N][N].
 */
blink_status blink_pipeline_host(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                 const blink_imaging* imaging, int32_t arith, const uint8_t* h_volt,
                                 float* h_img, int32_t images_per_pass, void* stream);

/*
 * blink_pipeline (batched form) for a phase centre that moves during the call, as when the array tracks a
 * source (Sec. 5.2.3: the geometric corrections set the phase centre; here one per integration): integration
 * tau is imaged with its phase centre at the direction cosines (h_lm[2 tau], h_lm[2 tau + 1]) of the local East,
 * North, Up frame, each with l^2 + m^2 < 1 (imaging->phase_l and phase_m are ignored).  h_lm: host double
 * [T][2], T = obs->n_samples / obs->samples_per_int, read during the call.  Consecutive integrations with the
 * same pointing share one plan and one launch; each distinct pointing builds a plan (cells, phase table,
 * gather order) that the context caches like blink_pipeline's.  The uv cell is imaging->cell_lambda, or, when that is 0, the
 * default cell of the first integration's pointing for every integration, so that all images share one pixel
 * scale.  Images, layout and errors otherwise as blink_pipeline (BLINK_ERR_INVALID_ARG for a NULL h_lm or a
 * pointing outside the unit circle).
 */
blink_status blink_pipeline_tracking(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                     const blink_imaging* imaging, const double* h_lm, int32_t arith,
                                     const uint8_t* d_volt, float* d_img, void* stream);

/*
 * Averaged dirty images (the paper's long-exposure and band-averaged products: Sec. 6.1 averages the 1 s
 * images of every fine channel over the whole time range and band into one image, Sec. 6.2 the 20 ms
 * images of each time bin over the band): output (tau', f') is the mean of the blink_pipeline images of integrations
 * [tau' t_avg, (tau' + 1) t_avg) and output channels [f' f_avg, (f' + 1) f_avg), written to d_img as float
 * [T / t_avg][F / f_avg][N][N].  t_avg = T, f_avg = F gives one long-exposure image; t_avg = 1, f_avg = F the
 * band average of each integration.
 * The averages are formed before the transform, not after it: the mean over integrations is the image of
 * the summed correlations (one pointing per call, so the cells do not change within it; the integration
 * becomes t_avg samples_per_int long and its limits apply), and the mean over channels is one transform of
 * the sum of the channels' grids, each divided by its own W.  So an output costs one 2D transform however
 * many images it averages.  Every side the imaging descriptor allows, with or without a gridding kernel, runs
 * the mixed-radix passes here.  Equal to the mean of the individual images up to FP32 rounding.
 *   t_avg, f_avg  >= 1, dividing T and F; else BLINK_ERR_INVALID_ARG before any launch.
 */
blink_status blink_pipeline_averaged(blink_context* ctx, const blink_array* array, const blink_obs* obs,
                                     const blink_imaging* imaging, int32_t arith, int32_t t_avg, int32_t f_avg,
                                     const uint8_t* d_volt, float* d_img, void* stream);

/*
 * blink_image without any device allocation (the paper has no counterpart; this is a library service).
 * Callers that cannot allocate device memory while they image - a real-time instrument pipeline that
 * reserves all device memory when an observation starts, or an application whose device memory belongs
 * to another allocator - can use this entry point: it needs no context and calls no cudaMalloc, cudaFree
 * or allocating library routine.  Arguments, layouts and results are those of blink_image; it runs on
 * the calling thread's current CUDA device.
 *   Scratch: a fixed 16 MiB array in the library's static device memory (held by every GPU that loads
 *   the library until the process exits) holds the twiddle table and the column-pass result of as many
 *   images as fit; larger batches are processed in passes.  One image must fit: sides up to 1024 with
 *   BLINK_PREC_FP32 storage and up to 2048 with BLINK_PREC_BF16 (powers of two; for the mixed-radix
 *   sides N rows of N/2 + 1 pairs rounded up to a multiple of 4, e.g. 1200 with FP32 storage, 2400 with
 *   BF16); a larger side returns
 *   BLINK_ERR_UNSUPPORTED before anything is launched.  Every call rewrites the parts of the scratch it
 *   reads, so nothing needs clearing between calls.
 *   Set-up: the first call on a device - n_images == 0 included, which does nothing else - looks up the
 *   scratch's device address (cudaGetSymbolAddress) with that device current.  The 16 MiB are committed
 *   when the library's module for this entry point loads on the device; under CUDA's lazy module
 *   loading (the default) that is this first lookup, which can therefore fail for lack of device memory.
 *   Make that first call (a zero-image call is a warm-up) before reserving the rest of the device's
 *   memory and before any stream capture.
 *   All calls share the one scratch array: calls whose work overlaps on the GPU (different streams,
 *   or different host threads) race and corrupt each other's images.  Order them on one stream.
 */
blink_status blink_image_noalloc(const blink_imaging* imaging, const float* d_grid, int32_t n_images,
                                 const float* d_weight, float* d_img, void* stream);

/* ---- measurement -------------------------------------------------------------------------------- */

/* Pipeline stages, for per-stage GPU time. */
enum {
    BLINK_STAGE_CORRELATE = 0,   /* correlation kernels */
    BLINK_STAGE_GRID_FFT = 1,    /* gridding + the 2D inverse FFT (the batched form's persistent kernel) */
    BLINK_STAGE_ROW_FFT = 2,     /* a separate row (complex-to-real) FFT pass, where one runs */
    BLINK_STAGE_FUSED = 3,       /* correlation + gridding + 2D inverse FFT in one persistent launch */
    BLINK_N_STAGES = 4
};

/*
 * Per-stage timing of blink_pipeline (not part of the method; for measurement).  While enabled, every
 * kernel launch of the batched pipeline is bracketed by a pair of CUDA events recorded on the launch's
 * stream.  blink_read_profile waits for `stream`, then adds each stage's summed event time (ms) and
 * launch count to ms[BLINK_N_STAGES] and launches[BLINK_N_STAGES] (host arrays, overwritten), and
 * forgets the recorded events when `reset` is non-zero.
 */
blink_status blink_set_profiling(blink_context* ctx, int32_t enable);
blink_status blink_read_profile(blink_context* ctx, void* stream, double* ms, int64_t* launches, int32_t reset);

/*
 * Bounded device-side waits of the batched imaging kernel (a library service; the paper has no
 * counterpart).  The kernel's tasks wait for one another through per-image counters; each wait gives up
 * after `budget_cycles` SM clock cycles (default about one second; budget_cycles <= 0 restores it),
 * records BLINK_ERR_TIMEOUT in the context's status word and stops the launch, which then returns; the
 * next blink_sync() reports BLINK_ERR_TIMEOUT.  With `unreachable` non-zero the row tasks wait for one
 * more column task than an image has, so each of those waits runs out on purpose: this is how a test
 * exercises the failure path without a GPU fault or hang.  The images of a launch that ran out are
 * invalid.  The setting holds for later calls of the context until changed.
 */
blink_status blink_set_wait_budget(blink_context* ctx, int64_t budget_cycles, int32_t unreachable);

/*
 * The fused form of the batched imaging path (BLINK_MODE_BATCHED; a library design choice, the paper runs its
 * stages as separate kernels, Sec. 5.2): for 512^2 nearest-cell images with FP8 correlation, no calibration
 * and the zenith phase centre, one persistent launch per call correlates each image's integration on the
 * tensor cores and grids and transforms it, the correlation sums staying in an L2-resident ring.  Off by
 * default: on GB300 the separate correlation launch (its sums assembled in gather order in shared memory and
 * written out whole) is faster than correlation tasks that scatter those sums into the ring from registers.
 * Both forms give the same images, bit for bit.  Applies to later calls of the context.
 */
blink_status blink_set_fused(blink_context* ctx, int32_t enable);

/*
 * The launch shape the batched imaging kernel's autotuner kept for the context's most recent plan (a
 * diagnostic for measurements; no counterpart in the paper): out[0] column-result ring slots, out[1] the lag
 * of an image's row tasks behind its column tasks (images), out[2] resident CTAs per SM (0: as many as fit);
 * all zero before the plan's first batched call.  out: host int32[3].
 */
blink_status blink_tuned_shape(blink_context* ctx, int32_t* out);

#ifdef __cplusplus
}
#endif

#endif /* BLINK_H */
