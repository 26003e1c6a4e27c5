/*
 * wiresim: GB300 (sm_103a) kernels for the LArTPC signal-simulation hot path
 * of arXiv 2203.02479 (Dong, Knoepfel, Lin, Viren, Yu, "Evaluation of
 * Portable Programming Models to Accelerate LArTPC Detector Simulations").
 *
 * The path, per wire plane (Sec. 2.1, Sec. 2.2):
 *   diffusion   each ionization deposition ("depo") spreads into a 2D
 *               Gaussian along drift time and wire pitch (Sec. 2.2);
 *   raster      that Gaussian is binned into a patch of (wire, tick) bins
 *               (Sec. 2.2, "Raster"), optionally with binomial charge
 *               fluctuation (Sec. 3.1);
 *   scatter-add the patches are summed into a dense wire x tick grid S
 *               (Sec. 2.2, "Scatter-add"; Sec. 2.3, dense matrix);
 *   convolution the grid is convolved with the detector response R by
 *               FFT, spectrum multiply and inverse FFT (Eq. 1, Eq. 2).
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_dev are device pointers; all other pointers are host
 *     pointers.  The caller owns every buffer it passes; the library keeps
 *     only the host-side plane object and uses the caller's workspace.
 *   - Grids are float32, row-major [wire][tick] (ticks contiguous).
 *   - Work is stream-ordered on the cudaStream_t passed as `stream` (NULL
 *     is the legacy default stream).  No call synchronises the host unless
 *     its comment says so.
 *   - Every call returns a ws_status; nothing throws across the ABI.
 *     Argument errors are returned before anything is enqueued.  Errors the
 *     device detects in the data (a non-finite depo, a negative width, a
 *     patch buffer too small) never trap: the depo or patch is skipped and a
 *     bit is set in the plane's device status word (WS_DEV_*), read back by
 *     ws_plane_sync.
 *   - A plane's workspace is shared by all calls on that plane: calls on one
 *     plane must be ordered (one stream, or events between streams).
 *   - With WS_LOG set in the environment, CUDA failures and non-zero device
 *     status words read by ws_plane_sync are also printed to stderr.  The
 *     simulation entry points mark their host work with NVTX ranges.
 *
 * Units: pitch in mm, time in microseconds, charge in electrons.
 * Bin conventions (the paper is silent; the oracle follows the same):
 *   wire bin w covers pitch [w*pitch, (w+1)*pitch), tick bin k covers time
 *   [k*tick, (k+1)*tick); x and t are measured from the low edge of bin 0.
 */
#ifndef WIRESIM_H
#define WIRESIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WS_OK = 0,
    WS_ERR_INVALID_ARG = 1,       /* NULL or misaligned pointer, bad value  */
    WS_ERR_UNSUPPORTED_SIZE = 2,  /* FFT length not 2/3/5-smooth or too big */
    WS_ERR_OOM = 3,               /* host allocation of the plane failed    */
    WS_ERR_CUDA = 4,              /* a CUDA call failed: see ws_last_error  */
    WS_ERR_TIMEOUT = 5,           /* a bounded device wait gave up          */
    WS_ERR_WORKSPACE = 6,         /* workspace too small                    */
    WS_ERR_BAD_INPUT = 7          /* device status word reports bad data    */
} ws_status;

/* Bits of the plane's device status word. */
#define WS_DEV_BAD_DEPO       0x1u  /* depo with non-finite q/x/t/sigma or negative
                                       sigma or drift time: skipped            */
#define WS_DEV_PATCH_OVERFLOW 0x2u  /* ws_rasterize: patch buffer too small;
                                       patches past the capacity not written   */
#define WS_DEV_TIMEOUT        0x4u  /* a bounded spin-wait gave up             */

enum { WS_CONV_LINEAR = 0, WS_CONV_CIRCULAR = 1 };
enum { WS_PREC_FP32 = 0, WS_PREC_FP32_COMP = 1, WS_PREC_FP64 = 2 };

/* One wire plane: grid geometry and the response's shape.  Copied at
 * creation. */
typedef struct {
    int32_t nwires;           /* grid rows                                  */
    int32_t nticks;           /* grid columns                               */
    double pitch_mm;          /* wire pitch                                 */
    double tick_us;           /* sampling period                            */
    int32_t resp_nwires;      /* response rows K_w (<= 21)                  */
    int32_t resp_nticks;      /* response columns K_t                       */
    int32_t resp_wire_center; /* response row holding wire offset 0         */
    int32_t conv_mode;        /* WS_CONV_LINEAR (zero outside the grid) or
                                 WS_CONV_CIRCULAR (indices wrap, Eq. 2 on
                                 the grid itself)                           */
    int32_t fft_len_tick;     /* 0: smallest 2/3/5-smooth length >=
                                 nticks + K_t - 1 (linear) or nticks
                                 (circular); else that length               */
    double nsigma;            /* Gaussian truncation in sigmas (3.0)        */
    int32_t plane_id;         /* 0..15, part of the random-stream key       */
    int32_t fp64;             /* nonzero: also hold the FP64 tables and
                                 buffers that WS_PREC_FP64 needs (about
                                 2x the workspace)                          */
    int32_t impacts;          /* 0 or 1: one response for the whole pitch.
                                 I = 2 .. 32: the response depends on where
                                 in the pitch the charge is (I sub-pitch
                                 positions; the paper's WCT field responses
                                 are of this kind, Sec. 2.1): the response
                                 array is I x K_w x K_t (slice i for charge
                                 at [(w + i/I), (w + (i+1)/I)) pitches), the
                                 raster bins the pitch axis at pitch/I into
                                 a fine grid of nwires*I rows (fine row
                                 w*I + i), and M = sum_i R_i (*) S_i.
                                 ws_simulate (every precision),
                                 ws_simulate_batch (a batch's planes share
                                 I) and the adjoint take them               */
} ws_plane_desc;

/* Depos of one event as seen by one plane: structure of arrays of float32
 * device pointers, all of length n (Sec. 2.3: the depo arrays are laid out
 * as structures of arrays).  sigma_t_us / sigma_x_mm are either both NULL
 * (widths come from diffusion, see ws_params) or both set (given widths).
 * Every array given is 4-byte aligned (else WS_ERR_INVALID_ARG). */
typedef struct {
    const float* q;           /* charge [electrons]                         */
    const float* x_mm;        /* pitch position                             */
    const float* t_us;        /* drift time                                 */
    const float* sigma_t_us;  /* longitudinal width in time, or NULL        */
    const float* sigma_x_mm;  /* transverse width in pitch, or NULL         */
    int64_t n;
} ws_depos;

/* Physics and numerics of one simulation call. */
typedef struct {
    double DL_mm2_us;         /* longitudinal diffusion constant            */
    double DT_mm2_us;         /* transverse diffusion constant              */
    double v_mm_us;           /* drift speed                                */
    int32_t fluctuate;        /* 0: expected value p*q*w per bin;
                                 1: Binomial(floor(q*w + 1/2), p) per bin,
                                    independent bins; bin (w, k) takes word
                                    k % 4 of the Philox block with counter
                                    (0, w*ceil(nticks/4) + k/4, depo,
                                    event << 4 | plane), one block per
                                    four ticks of a wire;
                                 2: charge-conserving: K ~ Binomial(
                                    floor(q + 1/2), p) survivors per depo,
                                    spread over its bins multinomially by
                                    conditional binomials over the in-grid
                                    wires, then ticks (Philox counters
                                    (5,0,depo,.), (4,wire,depo,.),
                                    (3,bin,depo,.)); electrons of off-grid
                                    bins are lost, an interior depo keeps
                                    exactly K.  Other values are invalid.   */
    double p_survive;         /* electron survival probability p            */
    uint64_t seed;            /* Philox key                                 */
    uint32_t event_id;        /* < 2^28, part of the Philox counter         */
    int32_t fluct_exact_max;  /* bins with N <= this sample Binomial(N, p)
                                 by inversion of its CDF (single precision,
                                 the word's top 24 bits); larger N use the
                                 normal approximation (Box-Muller on the
                                 word's two 16-bit halves); 0 .. 64         */
    int32_t precision;        /* WS_PREC_FP32: float throughout;
                                 WS_PREC_FP32_COMP: float with compensated
                                 (TwoSum) scatter-add and FP64 edge weights
                                 for axes narrower than 1/8 bin;
                                 WS_PREC_FP64: double throughout (needs a
                                 plane created with fp64 != 0).  Only
                                 ws_simulate honours it; the batch, patch
                                 and adjoint entry points run FP32.         */
    uint32_t depo_offset;     /* index of depos[0] in the event's whole depo
                                 list: the random counters carry each
                                 depo's index in that list (depo_offset +
                                 i), so an event's depos split over calls
                                 or GPUs draw exactly as in one call.
                                 depo_offset + n <= 2^32                    */
} ws_params;

/* Patches as produced by ws_rasterize: caller-allocated device arrays.
 * Patch i covers wires [w0[i], w0[i]+nw[i]) and ticks [t0[i], t0[i]+nt[i])
 * of the grid (already clipped to it); its values are val[off[i] ...
 * off[i] + nw[i]*nt[i]) row-major [wire][tick].  off has n + 1 entries,
 * off[n] being the total number of bins.  Every array is aligned to its
 * element size (else WS_ERR_INVALID_ARG). */
typedef struct {
    float* val;
    int32_t* w0;
    int32_t* t0;
    int32_t* nw;
    int32_t* nt;
    int64_t* off;
    int64_t capacity_bins;    /* length of val                              */
    int64_t n;                /* number of patches (== depos)               */
} ws_patches;

/* Plane facts chosen at creation, for callers and tests. */
typedef struct {
    int32_t fft_len_tick;     /* L_t                                        */
    int32_t nfreq;            /* L_t/2 + 1 half-spectrum bins               */
    int32_t nfreq_stride;     /* row stride of the spectra, complex elems   */
    int32_t npasses;          /* FFT radix passes                           */
    int32_t radices[16];
    size_t workspace_bytes;
    int32_t wire_conv_variant;  /* autotuned wire-convolution kernel: wire
                                   block 16 (0, 1, 4, 5, 8, 9) or 8 (2, 3,
                                   6, 7), Karatsuba three-product taps
                                   (odd), tiles by TMA (4..7) or TMA chunks
                                   into a ring kept along a run of wire
                                   blocks (8, 9); 4..9 linear mode only.
                                   Impact planes (linear mode): blocks of
                                   16 / 32 wires by 128 (0 / 1) or 64
                                   (2 / 3) frequencies                      */
    int32_t row_fft_fixed_shape; /* 1: this L_t's FP32 tick-axis transforms
                                   run kernels compiled for its radix plan
                                   (each row pair fetched into shared memory
                                   by bulk copies, first and middle passes
                                   in place, the last pass writing global
                                   memory); 0: the generic kernels          */
    int32_t batch_units_per_wave;  /* wave size ws_batch_autotune recorded
                                      on this plane (0: none)               */
    int32_t batch_wire_conv_variant; /* wire-convolution kernel of batches
                                      whose first plane this is (-1: the
                                      plane's own)                          */
} ws_plane_info;

typedef struct ws_plane ws_plane;

/* Bytes of device workspace a plane with this description needs (response
 * spectrum, twiddles, two spectra of nwires x (L_t/2+1) complex64, status
 * word, scan scratch, noise spectra, a 64-bit row mark and a row class per
 * wire for ws_simulate's active rows; with impacts I > 1 also the fine grid
 * of nwires*I x nticks floats and I times the compensated path's low-part
 * grid, the first spectrum, the response spectrum, the adjoint's taps and
 * the response gradient's spectra, and with fp64 I times the double grid,
 * first spectrum and response spectrum).  Host-only; fails with
 * WS_ERR_UNSUPPORTED_SIZE if the FFT length is not 2/3/5-smooth or exceeds
 * 14336, or for a grid (fine grid on an impact plane) of 2^31 cells or
 * more, and with WS_ERR_INVALID_ARG for impacts outside 0 .. 32. */
ws_status ws_plane_workspace_bytes(const ws_plane_desc* desc, size_t* bytes);

/* Create a plane over a caller-owned device workspace (>= the size above,
 * 256-byte aligned) and compute the response spectrum once (the transform
 * of R in Eq. 2) on `stream`.  It also autotunes the wire-convolution
 * kernel by timing its variants on the plane's buffers, which SYNCHRONISES
 * `stream` once (impact planes time their four TMA kernels in linear mode
 * and skip the timing otherwise).  response_dev: K_w x K_t float32, row-major, row r holding wire
 * offset r - resp_wire_center, column j tick offset j (causal); on an
 * impact plane I such slices, slice i first-index-major.  The response is
 * read during this call's stream work only.
 * The plane object itself is host memory, freed by ws_plane_destroy. */
ws_status ws_plane_create(const ws_plane_desc* desc, const float* response_dev,
                          void* workspace_dev, size_t workspace_bytes, void* stream,
                          ws_plane** out);

/* Free the host plane object; the workspace stays the caller's. */
ws_status ws_plane_destroy(ws_plane* plane);

/* The plane's plan (ws_plane_info: transform length and radices, spectrum
 * stride, workspace size, chosen wire-convolution kernel) into *info.
 * Host-only; WS_ERR_INVALID_ARG for a NULL plane or info. */
ws_status ws_plane_get_info(const ws_plane* plane, ws_plane_info* info);

/* Exact number of in-grid patch bins ws_rasterize will write for these
 * depos.  SYNCHRONISES `stream` (reads one counter back). */
ws_status ws_patch_capacity(ws_plane* plane, const ws_depos* depos, const ws_params* params,
                            void* stream, int64_t* bins_out);

/* Diffusion + raster (+ fluctuation) of every depo into its own patch
 * (Sec. 2.2 "Raster", Sec. 3.1).  A lane per depo for its geometry and
 * edge tables, its patch's bins spread over the warp (a warp per depo for
 * patches above 16 ticks x 8 wires, 32 fine wires on impact planes, whose
 * patches lie on the fine grid of nwires*I rows; a lane per depo for the
 * whole patch with fluctuate = 2).  Each bin holds
 * q * p * w_t * w_x (expected value), a binomial survivor count or its
 * share of the depo's multinomially spread survivors (see fluctuate), with
 * w the Gaussian mass of the bin clipped to mu +- nsigma*sigma over the
 * window's total mass.  Writes out->off (exclusive scan of patch sizes),
 * w0/t0/nw/nt and val.  If the total exceeds capacity_bins the device
 * status word gets WS_DEV_PATCH_OVERFLOW and the patches that do not fit are
 * not written (their nw/nt are set to 0). */
ws_status ws_rasterize(ws_plane* plane, const ws_depos* depos, const ws_params* params,
                       ws_patches* out, void* stream);

/* Scatter-add of patches into a grid (Sec. 2.2 "Scatter-add"):
 * grid_dev[w][t] += val of every patch bin at (w, t).  The grid is
 * accumulated into, not cleared.  grid_dev is nwires x nticks, or on a
 * plane with impacts I > 1 the fine grid of nwires*I x nticks. */
ws_status ws_scatter(ws_plane* plane, const ws_patches* patches, float* grid_dev,
                     void* stream);

/* Eq. 2: out = IFFT(R_hat * FFT(grid)), i.e. Eq. 1's sum of
 * R[d + c][j] * S[w - d][t - j] with S = 0 outside the grid (linear) or
 * indices wrapping (circular).  grid_dev and out_dev are nwires x nticks;
 * they may be the same buffer.  Uses the plane's workspace.  On a plane
 * with impacts I > 1, grid_dev is the fine grid (nwires*I x nticks, row
 * w*I + i), out_dev is nwires x nticks and they must not overlap. */
ws_status ws_convolve(ws_plane* plane, const float* grid_dev, float* out_dev, void* stream);

/* The whole hot path for one plane and one event: clear out_dev, raster +
 * fluctuate + scatter-add every depo straight into it (no patch buffer),
 * then convolve in place, adding the plane's noise term if one is set
 * (ws_plane_set_noise).  out_dev: nwires x nticks float32, every row
 * written.  On noise-free linear planes with fixed-shape transforms (L_t
 * 6250, 6000, 6400, 3200 or 1200) only the wire rows a depo can reach are
 * cleared and transformed, and waveform rows out of the response's reach
 * of all of them are written as zeros: the same result as transforming
 * every row (an untouched row is zero through Eq. 2's linear stages).  On
 * an impact plane (I > 1) the raster fills the plane's fine grid and whole
 * wires are marked (their I fine rows cleared and transformed together).
 * A per-plane epoch in the workspace, advanced on the device, keeps calls
 * and CUDA graph replays apart; calls on one plane must not overlap. */
ws_status ws_simulate(ws_plane* plane, const ws_depos* depos, const ws_params* params,
                      float* out_dev, void* stream);

/* The convolution of ws_convolve for callers that cannot allocate device
 * memory (no cudaMalloc, no workspace to hand over): only the response,
 * the input grid and the output grid are passed.  The paper has no
 * counterpart; this is a deployment convenience.
 *   - Scratch is one 16 MiB file-scope __device__ array inside the library,
 *     held by every GPU that loads it until the process exits.  Planes whose
 *     scratch (twiddles + response spectrum + two nwires x (L_t/2+1)
 *     complex64 spectra, each rounded to 256 bytes) exceeds 16 MiB are
 *     rejected with WS_ERR_WORKSPACE before anything is enqueued (e.g. up to
 *     ~330 wires at 6000 ticks).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - Every call shares the array and recomputes the response spectrum; it
 *     keeps the last call's contents.  Calls that overlap on the GPU race on
 *     it: order them on one stream.
 *   - Allocates nothing (no cudaMalloc/cudaFree, no allocating library
 *     call).  desc, grid_dev and out_dev as for ws_plane_create and
 *     ws_convolve (grid and out may be the same buffer); planes with
 *     impacts > 1 are rejected with WS_ERR_UNSUPPORTED_SIZE. */
ws_status ws_convolve_noalloc(const ws_plane_desc* desc, const float* response_dev,
                              const float* grid_dev, float* out_dev, void* stream);

/* Device workspace of ws_simulate_batch: three wave slots, each a
 * large-patch hand-over list and, per unit of a wave, two spectra (max
 * nwires x (L_t/2+1) complex64; the first I times that on impact planes),
 * a row mark and row class per wire, and on impact planes a fine grid of
 * I x max nwires x nticks floats.  units_per_wave: 1 .. 32, or 0 for the
 * largest wave (32 units), which holds every wave size. */
ws_status ws_batch_workspace_bytes(ws_plane* const* planes, int nplanes, int units_per_wave,
                                   size_t* bytes);

/* Many events on a detector of nplanes planes in one call: the units
 * (event e, plane p), in event-major order u = e * nplanes + p, run in waves
 * of units_per_wave; each stage of a wave (grid clear, raster + fluctuation +
 * scatter-add, tick transform, wire convolution, inverse transform) is ONE
 * launch over all the wave's units, so events with very different depo
 * counts share the GPU (the paper runs independent processes per GPU for
 * throughput, Sec. 3.3).  depos[u] are unit u's depos; out_dev[u] its
 * nwires(p) x nticks output (cleared, then simulated); event e uses
 * event_id = params->event_id + e.  All planes must share the transform
 * length, tick count, response shape and impact positions I (else
 * WS_ERR_UNSUPPORTED_SIZE).  With I > 1 each unit rasters into a fine grid
 * in its wave slot, marks whole wires, and the impact wire convolution runs
 * once over the wave's units (units of up to 32 / I per launch).
 * Each plane's noise term (ws_plane_set_noise) is added as in ws_simulate.
 * Results equal ws_simulate unit by unit (up to summation order); units of
 * noise-free planes skip untouched wire rows as ws_simulate does, with the
 * marks in the workspace slots cleared at the start of every call.  With more
 * than one wave, the waves go round `stream` and up to two more streams
 * owned by the library (per host thread and device): wave k runs on stream
 * k % S, S = min(waves, 3), each with its own workspace slot.  The extra
 * streams fork from `stream` at the start of the call and join it at the
 * end through events, so one wave's raster overlaps the other waves'
 * transforms and the call stays ordered on `stream`.  Makes no host
 * synchronisation, so it can be captured into a CUDA graph. */
ws_status ws_simulate_batch(ws_plane* const* planes, int nplanes, const ws_depos* depos, int nevents,
                            const ws_params* params, float* const* out_dev, void* workspace_dev,
                            size_t workspace_bytes, int units_per_wave, void* stream);
/* units_per_wave == 0 in ws_simulate_batch: the wave size ws_batch_autotune
 * recorded on planes[0] if the workspace holds it, else the largest wave
 * (at most 32 units, at most nevents * nplanes) the workspace holds. */

/* Autotuner of ws_simulate_batch's wave size (the throughput motivation is
 * the paper's Sec. 3.3): runs the batch on the caller's own inputs for each
 * candidate wave size (1 .. 4 units, whole events of nplanes x 1, 2, 4, ...
 * units, and the largest wave; only sizes whose workspace fits
 * workspace_bytes), once to warm up and then three interleaved timed rounds
 * (CUDA events on `stream`), keeps the fastest by its best round, writes it
 * to *units_per_wave_out and records it on every plane of the call for
 * later calls with units_per_wave == 0.  Arguments as for
 * ws_simulate_batch; out_dev ends up holding the batch's result.
 * Then, at that wave size, it times the wire-convolution kernels the
 * planes allow (one kernel serves every unit of a launch) and records the
 * fastest on planes[0] for batches, unless a kernel was already chosen for
 * batches on planes[0] (by an earlier run or ws_plane_set_wire_conv_variant);
 * the planes keep their own kernels for single-plane calls.
 * SYNCHRONISES `stream` (so it cannot be captured into a graph: call it
 * before capturing).  WS_ERR_WORKSPACE if no candidate fits. */
ws_status ws_batch_autotune(ws_plane* const* planes, int nplanes, const ws_depos* depos, int nevents,
                            const ws_params* params, float* const* out_dev, void* workspace_dev,
                            size_t workspace_bytes, void* stream, int* units_per_wave_out);

/* Noise term N(t, x) of Eq. 1 (Sec. 2.1 names it; the paper's port leaves
 * it out, and its model is this library's reading): from now on
 * ws_simulate and ws_simulate_batch add to each wire w of this plane the
 * stationary Gaussian noise with half spectrum, on the plane's tick
 * transform length L (ws_plane_info.fft_len_tick),
 *   Nhat_w[k] = amp[k] xi_w[k] + coh_amp[k] xi'_{floor(w / coh_group)}[k],
 *   k = 0 .. L/2,   n_w[t] = (1/L) sum_{k<L} Nhat_w[k] e^{2 pi i k t / L}
 * over the Hermitian extension, for t < nticks.  xi and xi' are complex
 * normals (z1 + i z2)/sqrt 2 (z1 alone at k = 0 and k = L/2) from
 * Box-Muller, u = (top 23 bits of a Philox word + 1/2) / 2^23, keyed by
 * the call's seed with counter (1, k, floor(w/2), event << 4 | plane) for
 * the incoherent part (words 2(w%2), 2(w%2)+1) and (2, k, floor(g/2), ...)
 * for group g's coherent part; the fluctuation's counters start with 0, so
 * the streams never overlap.  amp_dev, coh_amp_dev: L/2 + 1 float32 device
 * amplitudes, copied (stream-ordered) into the plane's workspace;
 * coh_amp_dev may be NULL (no coherent part; coh_group is then ignored,
 * else it must be >= 1).  Both NULL switch the noise off.  The noise is
 * added to the half spectra (in place, one more launch) between the wire
 * convolution and the inverse transform, where the 1/L is already folded
 * in.  ws_convolve (the pure convolution) and the adjoint are unaffected
 * (the noise does not depend on the inputs). */
ws_status ws_plane_set_noise(ws_plane* plane, const float* amp_dev, const float* coh_amp_dev,
                             int32_t coh_group, void* stream);

/* Replace the plane's response (K_w x K_t float32 device array, same shape
 * as at creation) and recompute its spectrum on `stream`. */
ws_status ws_plane_set_response(ws_plane* plane, const float* response_dev, void* stream);

/* Adjoint of ws_simulate in expected-value mode (fluctuate == 0): given
 * grad_out_dev = dL/dM (nwires x nticks float32), computes
 *   gq, gx, gt [n floats]: dL/dq, dL/dx, dL/dt per depo (t through the
 *       Gaussian mean and, when widths come from diffusion, through
 *       sigma_L = sqrt(2 D_L t)/v and sigma_T = sqrt(2 D_T t));
 *   gDL, gDT [1 double each]: dL/dD_L, dL/dD_T (zero with given widths);
 *   gR [K_w x K_t floats]: dL/dR (I x K_w x K_t on an impact plane: one
 *       slice per sub-pitch position).
 * dL/dS is Eq. 2's adjoint (correlation with the response, by FFT); each
 * patch is recomputed, not stored.  On an impact plane dL/dS is formed on
 * the fine grid (position i's rows by the correlation with slice i) and
 * the depo gradients are those of the raster at pitch / I.  Derivatives of the clamped-edge bin
 * weights hold everywhere except where a window bound crosses a bin edge.
 * Any output pointer may be NULL to skip it (gR == NULL skips the
 * response-gradient work).  All outputs are device pointers aligned to
 * their element size (else WS_ERR_INVALID_ARG); uses the plane's
 * workspace. */
ws_status ws_simulate_backward(ws_plane* plane, const ws_depos* depos, const ws_params* params,
                               const float* grad_out_dev, float* gq, float* gx, float* gt,
                               double* gDL, double* gDT, float* gR, void* stream);

/* Copy the plane's device status word to *bits.  SYNCHRONISES `stream`. */
ws_status ws_plane_sync(ws_plane* plane, void* stream, uint32_t* bits);

/* Clear the plane's device status word (stream-ordered). */
ws_status ws_plane_clear_status(ws_plane* plane, void* stream);

/* Override the autotuned wire-convolution kernel (0..9, see
 * ws_plane_info.wire_conv_variant; 4..9 need linear mode; impact planes
 * 0..3, 1..3 in linear mode) for this plane's calls and for batches whose
 * first plane it is; all variants compute the same sum. */
ws_status ws_plane_set_wire_conv_variant(ws_plane* plane, int variant);

/* Launch tracing (timing of each kernel with CUDA events).  With
 * max_records > 0, every later launch on this plane is bracketed by a pair
 * of CUDA events, up to max_records launches (later ones are not recorded);
 * max_records == 0 turns tracing off.  Creates host-side CUDA events only. */
ws_status ws_plane_trace(ws_plane* plane, int max_records);

typedef struct {
    const char* name;         /* kernel name (static string)                */
    int64_t launches;
    double total_ms;          /* summed event-to-event device time          */
} ws_trace_stat;

/* Per-kernel totals of the records since tracing began or the last read;
 * clears the records.  SYNCHRONISES on the last recorded event.  Writes at
 * most max_stats entries and their count to *nstats. */
ws_status ws_plane_trace_read(ws_plane* plane, ws_trace_stat* stats, int max_stats, int* nstats);

/* Failure-detection check of the bounded waits (no counterpart in the
 * paper).  Launches one CTA on `stream` that waits on an mbarrier expecting
 * an arrival nobody makes, the wait the TMA kernels use for their copies
 * (they give up after 2^18 attempts, about a second): after `iters`
 * attempts (1 .. 2^20) it gives up, ORs WS_DEV_TIMEOUT into
 * *status_dev (device uint32_t, caller-owned) and returns; if cycles_dev is
 * not NULL the SM cycles spent waiting go to *cycles_dev (device uint64_t).
 * The context stays usable.  Stream-ordered, no host synchronisation. */
ws_status ws_selftest_bounded_wait(uint32_t* status_dev, int iters, unsigned long long* cycles_dev, void* stream);

/* Static text naming a status code ("unknown status" for other values). */
const char* ws_status_string(ws_status status);

/* Text of the last CUDA error seen by a ws_* call on this thread ("" if
 * none). */
const char* ws_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WIRESIM_H */
