// Internal declarations shared by the wiresim translation units (never
// installed; the public boundary is include/wiresim.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wiresim.h"

namespace ws {

constexpr int kMaxPasses = 16;
constexpr int kMaxFftLen = 14336;   // two complex64 buffers of this length fit in shared memory
constexpr int kMaxRespWires = 21;   // wire taps of the register-blocked wire convolution
constexpr int kMaxImpacts = 32;     // sub-pitch response positions of a plane
constexpr int64_t kScanScratch = 65536;

// Mixed-radix Stockham plan for one complex transform length.
struct FftPlan {
    int L;
    int npass;
    int radix[kMaxPasses];
    int ns[kMaxPasses];     // product of the radices before pass p
    int twoff[kMaxPasses];  // offset of pass p's Ns base twiddles
};

// Launch geometry and constants of a raster pass.
constexpr int kExactCap = 64;   // largest fluct_exact_max ((1 - s)^N stays a normal float)

struct RasterArgs {
    const float* q;
    const float* x;
    const float* t;
    const float* sig_t;   // may be null (widths from diffusion)
    const float* sig_x;
    int64_t n;
    int nwires, nticks;
    float pitch, tick;
    float nsig;
    float two_DL, two_DT, inv_v;
    int fluct;
    float p;              // survival probability (expected-value scale)
    uint32_t T;           // floor(p * 2^32), 0 for p <= 0
    int keep_all;         // p >= 1: every electron survives
    uint32_t key0, key1;  // Philox key from the seed
    uint32_t evpl;        // (event_id << 4) | plane_id
    uint32_t depo0;       // index of depo 0 in the event's whole list (the counters' depo word)
    int exact_max;        // N <= exact_max: CDF inversion; above: normal approximation
    int wide;             // grid binned at pitch / I (impact planes): wider lane-per-depo patches
    // CDF inversion on s = min(p, 1-p) (float): r = s / (1 - s), base = 1 - s
    float inv_r, inv_base;
    int inv_flip;         // p > 1/2: the search counts losses, k = N - k'
    uint32_t* status;
    // precision path (WS_PREC_*) and its extra state
    int prec;
    float* lo;            // compensated path: low parts of the grid
    double* grid64;       // FP64 path: the grid in double
    double two_DL64, two_DT64, v64, pitch64, tick64, nsig64, p64;
};

// ---- unit tables for launches that cover several (event, plane) units
constexpr int kMaxUnits = 32;

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 multiplies
// whose high halves are mixed with the other counter words and the key; the
// key advances by two Weyl constants per round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ---- shared-memory mbarriers and bulk (TMA) copies
constexpr int kWaitIters = 1 << 18;   // try_wait attempts before giving up (~1 s: an attempt suspends ~4 us)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// Bounded wait: false if the phase did not complete within `iters` attempts.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int iters = kWaitIters) {
    for (int it = 0; it < iters; ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// One thread: expect `bytes` on bar, then copy [src, src + each) into dst
// with the bulk copy engine (addresses and sizes multiples of 16 bytes).
__device__ __forceinline__ void bulk_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Noise term N(t, x) of Eq. 1 for one unit, added to the half spectra Y
// between the wire convolution and the inverse transform (amp null: none).  Wire w, bin k:
// Nhat = A[k] xi_w[k] + Ac[k] xi'_{w / group}[k], xi = (z1 + i z2)/sqrt 2
// (z1 alone at k = 0 and k = L/2), z1, z2 by Box-Muller from words
// 2 (w % 2), 2 (w % 2) + 1 of the Philox block with counter
// (1, k, w / 2, evpl) (coherent: (2, k, g / 2, evpl), words by g % 2).
struct NoiseUnit {
    const float* amp;     // incoherent amplitude spectrum A[k], L/2 + 1 entries
    const float* coh;     // coherent amplitude spectrum, or null
    int group;            // wires per coherent group (>= 1 with coh)
    uint32_t evpl;        // event << 4 | plane
    double scale;         // 1 / L: the inverse transform is unnormalised
};

// ---- active rows
// A simulation marks, before its raster, every wire row of a unit's grid that
// the raster may touch (a superset: each depo's clipped wire range widened by
// one wire); rows[w] == the call's epoch marks row w.  Two epoch words: the
// marking kernel reads `base` and marks with base + 1, which it stores to
// `epoch`; the clearing kernel that follows it clears the marked rows (the
// raster adds into no other row) and copies `epoch` to `base` for the next
// call.  Marks of earlier calls so go stale without being cleared, also
// across CUDA graph replays, and every later stage reads `epoch` once at its
// start.  An unmarked row of S is zero, so the stages after the raster skip
// it exactly:
// The clearing kernel also classifies every row once per call (RowClass
// bits), so the row transforms decide per row pair from two words:
//   forward      transforms row pairs with a marked row (an unmarked row of
//                such a pair reads as zero); writes zero spectra for rows
//                within K_w - 1 wires of a marked row (the wire convolution
//                may read them); leaves other rows alone;
//   wire conv    skips tiles none of whose output rows is live; output row
//                w is live if a row of its window [w + c - K_w + 1, w + c]
//                is marked (only live rows' spectra are ever read);
//   inverse      writes zero waveforms for rows that are not live (reading
//                no spectrum for them) and transforms the others.
// The result is the same as transforming every row: unmarked rows are exact
// zeros through each stage.
// Marks and epochs are 64-bit: an epoch never comes round again.
using mark_t = unsigned long long;
struct RowMarks {
    mark_t* rows[kMaxUnits];      // per unit, nwires entries; null: every row active
    uint32_t* cls[kMaxUnits];     // per unit, nwires row classes (written by the clearing kernel)
    mark_t* epoch;                // the call's epoch (written by the marking kernel)
    mark_t* base;                 // the previous call's epoch (copied from `epoch` by the clearing kernel)
    int kw = 0, center = 0;       // response wires and centre row (the classes' windows)
    // per unit, grid rows per marked row: impact planes mark whole wires, and
    // wire w's grid rows are w * I .. w * I + I - 1 (0 or 1: one row per wire)
    int impacts[kMaxUnits] = {};
};

__device__ __forceinline__ mark_t read_epoch(const mark_t* e) { return *(const volatile mark_t*)e; }

// Row classes (one word per wire row, written for every row by the clearing
// kernel): the row is marked; a marked row lies in [w - K_w + 1, w + K - 1]
// with K = kMaxRespWires (its spectrum may be read: the register-blocked
// kernels read every live output's K-row window, whose taps past K_w are
// zero, and zero times a stale non-finite value is not zero); a marked row
// lies in its wire-convolution window [w + c - K_w + 1, w + c] (its output
// is live).
enum : uint32_t { ROW_MARKED = 1u, ROW_NEEDED = 2u, ROW_LIVE = 4u };

// Whether any row of [lo, hi] (clipped to [0, n)) is marked; every thread of
// the CTA calls it (one barrier).
__device__ __forceinline__ bool cta_any_marked(const mark_t* rows, mark_t cur, int lo, int hi, int n) {
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
    bool any = false;
    for (int w = lo + (int)threadIdx.x; w <= hi; w += (int)blockDim.x) any = any || rows[w] == cur;
    return __syncthreads_or(any) != 0;
}

// Host-side batch descriptions.
struct RowBatch {          // row transforms: unit i has nrows[i] rows in[i] -> out[i]
    int n;
    const void* in[kMaxUnits];
    const void* in2[kMaxUnits];   // optional float low parts added to in (compensated grids)
    void* out[kMaxUnits];
    int nrows[kMaxUnits];
    uint32_t* status = nullptr;   // device status word: lets the fixed-shape kernels fetch rows by
                                  // bulk copies (a copy that never lands is reported there)
    // active rows (fixed-shape FP32 kernels only): per unit the row classes
    // of the call (null: every row marked, needed and live); row r takes the
    // class of entry r / rdiv (the fine rows of an impact plane share their
    // wire's class; 0 or 1: one entry per row)
    const uint32_t* rows[kMaxUnits] = {};
    int rdiv[kMaxUnits] = {};
};
struct NoiseBatch {        // noise added to the spectra Y[i] (nwires[i] rows) of each unit
    int n = 0;
    void* Y[kMaxUnits];
    int nwires[kMaxUnits];
    NoiseUnit noise[kMaxUnits] = {};
    uint32_t key0 = 0, key1 = 0;       // Philox key (the call's seed)
};
struct ConvBatch {         // wire convolutions: unit i maps X[i] -> Y[i] with taps Rt[i]
    int n;
    const void* X[kMaxUnits];
    void* Y[kMaxUnits];
    const void* Rt[kMaxUnits];
    int nwires[kMaxUnits];
    // active rows (FP32 kernels; null: compute every tile): a tile is skipped
    // when none of its output rows is live
    const mark_t* rows[kMaxUnits] = {};
    const mark_t* epoch = nullptr;
};
// Device-side tables (kernel parameters, read in place as __grid_constant__).
struct RowUnits {
    int n;
    int prefix[kMaxUnits + 1];   // cumulative row pairs
    const void* in[kMaxUnits];
    const void* in2[kMaxUnits];
    void* out[kMaxUnits];
    int nrows[kMaxUnits];
    uint32_t* status;
    const uint32_t* rows[kMaxUnits];   // row classes, or null
    int rdiv[kMaxUnits];               // rows per class entry (>= 1)
};
struct NoiseUnits {
    int n;
    int prefix[kMaxUnits + 1];   // cumulative blocks of kNoiseRows wires
    void* Y[kMaxUnits];
    int nwires[kMaxUnits];
    NoiseUnit noise[kMaxUnits];
    uint32_t key0, key1;
};
struct ConvUnits {
    int n;
    int prefix[kMaxUnits + 1];   // cumulative wire blocks
    const void* X[kMaxUnits];
    void* Y[kMaxUnits];
    const void* Rt[kMaxUnits];
    int nwires[kMaxUnits];
    const mark_t* rows[kMaxUnits];
    const mark_t* epoch;
};

// ---- FFT / convolution launchers (fft.cu)
// Pass twiddle table: Ns base twiddles per pass (see FftPlan::twoff).
cudaError_t launch_twiddles(float2* tw, const FftPlan& plan, cudaStream_t s);
// Real rows -> half spectra: out[r][k] = scale * sum_n in[r][n] e^{-2 pi i k n / L}
// for k < nfreq; rows shorter than L are zero padded.
cudaError_t launch_fwd_rows(const FftPlan& plan, const float2* tw, const float* in, int nrows,
                            int ncols, int64_t in_stride, float2* out, int64_t out_stride,
                            int nfreq, float scale, cudaStream_t s, uint32_t* status = nullptr);
// Half spectra -> real rows: out[r][n] = sum_k Y[r][k] e^{+2 pi i k n / L} over the
// Hermitian-extended spectrum, for n < ncols.
cudaError_t launch_inv_rows(const FftPlan& plan, const float2* tw, const float2* in, int nrows,
                            int64_t in_stride, int nfreq, float* out, int ncols,
                            int64_t out_stride, cudaStream_t s, uint32_t* status = nullptr);
// Noise term of Eq. 1 added in place to each unit's spectra (float2 or
// double2 rows of `stride`, nfreq bins of a length-L transform); units with
// a null amplitude are skipped.
cudaError_t launch_add_noise(const NoiseBatch& nb, int nfreq, int L, int64_t stride, cudaStream_t s);
cudaError_t launch_add_noise64(const NoiseBatch& nb, int nfreq, int L, int64_t stride, cudaStream_t s);
// Y[w][k] = sum_r Rt[r][k] * X[w + center - r][k]  (zero or wrapped outside).
// Batched forms: one launch over every unit (all units share plan, strides,
// response shape and wire-convolution variant).
// True when the plan's radix sequence has fixed-shape FP32 row kernels.
bool row_fft_fixed_shape(const FftPlan& plan);
cudaError_t launch_fwd_rows_batch(const FftPlan& plan, const float2* tw, const RowBatch& rb, int ncols,
                                  int64_t in_stride, int64_t out_stride, int nfreq, float scale, cudaStream_t s);
cudaError_t launch_inv_rows_batch(const FftPlan& plan, const float2* tw, const RowBatch& rb, int64_t in_stride,
                                  int nfreq, int ncols, int64_t out_stride, cudaStream_t s);
cudaError_t launch_wire_conv_batch(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, int circular,
                                   cudaStream_t s, int variant, uint32_t* status = nullptr);
// FP64 path (precision WS_PREC_FP64): double twiddles, spectra and sums;
// the forward transform reads float or double rows, the inverse writes float.
cudaError_t launch_twiddles64(double2* tw, const FftPlan& plan, cudaStream_t s);
cudaError_t launch_fwd_rows64(const FftPlan& plan, const double2* tw, const void* in, bool in_double, int nrows,
                              int ncols, int64_t in_stride, double2* out, int64_t out_stride, int nfreq, float scale,
                              cudaStream_t s);
cudaError_t launch_inv_rows64(const FftPlan& plan, const double2* tw, const double2* in, int nrows, int64_t in_stride,
                              int nfreq, float* out, int ncols, int64_t out_stride, cudaStream_t s);
cudaError_t launch_wire_conv64(const double2* X, double2* Y, const double2* Rt, int nwires, int nfreq, int64_t stride,
                               int kw, int center, int circular, cudaStream_t s);
// FP64 wire convolution over sub-pitch impact positions (X: nwires*impacts
// fine rows; Y[w][k] = sum_i sum_r Rt[i*kw + r][k] X[(w + center - r)*impacts + i][k]).
cudaError_t launch_wire_conv_impacts64(const double2* X, double2* Y, const double2* Rt, int nwires, int impacts,
                                       int nfreq, int64_t stride, int kw, int center, int circular, cudaStream_t s);
// Compensated input: rows are hi + lo (two float grids).
cudaError_t launch_fwd_rows_comp(const FftPlan& plan, const float2* tw, const float* hi, const float* lo, int nrows,
                                 int ncols, int64_t in_stride, float2* out, int64_t out_stride, int nfreq,
                                 cudaStream_t s);
// variant: 0 = 16 wires per thread, 1 = 16 Karatsuba, 2 = 8, 3 = 8 Karatsuba,
// with plain loads; 4..7 the same four fed by TMA tile copies; 8, 9 = 16
// wires (plain, Karatsuba) fed by TMA chunk copies into a ring that a CTA
// keeps along a run of wire blocks (4..9: linear mode only; they report a
// copy that never lands in *status).
constexpr int kWireConvVariants = 10;
cudaError_t launch_wire_conv(const float2* X, float2* Y, const float2* Rt, int nwires,
                             int nfreq, int64_t stride, int kw, int center, int circular,
                             cudaStream_t s, int variant = 0, uint32_t* status = nullptr);
// Wire convolution with sub-pitch impact positions: Y[w][k] = sum_i sum_r
// Rt[i*kw + r][k] * X[(w + center - r)*impacts + i][k] (X has nwires*impacts
// rows, zero or wrapped outside the wires).
cudaError_t launch_wire_conv_impacts(const float2* X, float2* Y, const float2* Rt, int nwires, int impacts,
                                     int nfreq, int64_t stride, int kw, int center, int circular, cudaStream_t s);
// TMA-fed wire convolution (wconv_tma.cu), variant 0..5 = 4..9 above.
bool tma_available();
cudaError_t launch_bounded_wait_selftest(uint32_t* status, int iters, unsigned long long* cycles, cudaStream_t s);
cudaError_t launch_wire_conv_tma(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, int variant,
                                 uint32_t* status, cudaStream_t s);
// The impact wire convolution fed by TMA (linear mode; a copy that never
// lands sets WS_DEV_TIMEOUT in *status) over the units of cb (X: I x
// nwires fine rows each; units share I, the frequency layout and the
// response width), as few launches as its tensor maps allow; variant 0 / 1:
// blocks of 16 / 32 output wires by 128 frequencies, 2 / 3: the same by 64.  CTAs claim blocks from sched[0] (two
// zeroed words, left zeroed by each launch; launches sharing them must not
// overlap).  With active-row marks (cb.rows, one per wire, and cb.epoch)
// blocks whose outputs are all dead are skipped and their Y rows not
// written.
constexpr int kImpactConvVariants = 4;
cudaError_t launch_wire_conv_impacts_tma(const ConvBatch& cb, int impacts, int nfreq, int64_t stride, int kw,
                                         int center, unsigned* sched, uint32_t* status, cudaStream_t s,
                                         int variant = 0);

// Hand-over list of depos whose patches are too large for the lane-per-depo
// raster kernel (workspace-resident; count and done must start at zero and
// are reset by the second kernel).
struct LargeList {
    long long* list;      // entries (unit << 40) | depo index
    unsigned* count;
    unsigned* done;
    unsigned cap;
};
constexpr unsigned kLargeListCap = 65536;

// Adjoint helpers (fft.cu): flipped conjugate taps; response-gradient
// spectra accumulated (A must start at zero).
cudaError_t launch_adj_coeffs(const float2* Rt, float2* A, int kw, int64_t stride, int nfreq, cudaStream_t s);
cudaError_t launch_resp_grad(const float2* XG, const float2* XS, float2* A, int nwires, int nfreq, int64_t stride,
                             int kw, int center, int circular, float scale, cudaStream_t s);

// ---- raster / scatter launchers (raster.cu)
cudaError_t launch_raster_scatter(const RasterArgs& a, float* grid, const LargeList& L, cudaStream_t s);
// Batched raster: unit i rasterises a[i] into grid[i]; one launch pair for all.
struct RasterBatch {
    int n;
    int prec;             // one precision for the whole batch
    RasterArgs a[kMaxUnits];
    float* grid[kMaxUnits];
};
struct RasterUnits {
    int n;
    long long gprefix[kMaxUnits + 1];   // cumulative 16-depo groups
    long long dprefix[kMaxUnits + 1];   // cumulative depos
    RasterArgs a[kMaxUnits];
    float* grid[kMaxUnits];
    mark_t* rows[kMaxUnits];            // active-row marks (mark / clear kernels), or null
    uint32_t* cls[kMaxUnits];           // row classes (clear kernel), with marks
    int imp[kMaxUnits];                 // grid rows per marked row (impact positions; 1: plain)
};
struct ZeroSizes {
    long long count[kMaxUnits];
};
cudaError_t launch_raster_scatter_batch(const RasterBatch& rb, const LargeList& L, cudaStream_t s);
cudaError_t launch_zero_grids(const RasterBatch& rb, const int64_t* counts, cudaStream_t s);
// Active rows: mark every unit's rows its depos may touch (units with null
// marks are skipped), then clear the marked rows of every unit's grid (and
// of its compensated low-part grid, if any; a unit with null marks is
// cleared whole).
cudaError_t launch_mark_rows(const RasterBatch& rb, const RowMarks& m, cudaStream_t s);
cudaError_t launch_zero_marked_rows(const RasterBatch& rb, const RowMarks& m, cudaStream_t s);
cudaError_t launch_patch_sizes(const RasterArgs& a, int64_t* sizes, unsigned long long* total,
                               cudaStream_t s);
// Adjoint of the expected-value raster: per-depo dL/dq, dL/dx, dL/dt from
// dS = dL/dS; dL/dD_L and dL/dD_T accumulated into gDL / gDT (FP64).
cudaError_t launch_depo_grads(const RasterArgs& a, const float* dS, float* gq, float* gx, float* gt, double* gDL,
                              double* gDT, double DL, double DT, const LargeList& L, cudaStream_t s);
cudaError_t launch_scan_inplace(int64_t* v, int64_t n, int64_t* scratch, cudaStream_t s);
cudaError_t launch_raster_patches(const RasterArgs& a, const ws_patches& p, const LargeList& L, cudaStream_t s);
cudaError_t launch_scatter_patches(const ws_patches& p, float* grid, int nwires, int nticks,
                                   cudaStream_t s);

int num_sms();

// Planner and error recording shared with the allocation-free entry point.
ws_status conv_plan(const ws_plane_desc* desc, FftPlan* plan, int* nfreq, int* fstride);
ws_status record_cuda_error(cudaError_t e, const char* where);

}  // namespace ws

struct ws_trace;

// The plane: host object pointing into the caller's workspace.
struct ws_plane {
    ws_trace* trace;    // launch trace, or null
    int wconv_variant;  // wire-convolution kernel chosen by the autotuner
    int batch_upw;      // batch wave size chosen by ws_batch_autotune (0: not tuned)
    int batch_wconv;    // batch wire-convolution kernel chosen by it (-1: not tuned)
    ws_plane_desc desc;
    ws::FftPlan plan;
    int nfreq;          // L/2 + 1
    int fstride;        // row stride of spectra (complex elements)
    size_t ws_bytes;
    uint32_t* status;   // device status word
    unsigned long long* counter;
    float2* tw;         // L twiddles e^{-2 pi i q / L}
    float2* Rt;         // K_w x fstride response spectrum (scaled by 1/L)
    float2* X;          // nwires x fstride
    float2* Y;          // nwires x fstride
    int64_t* scan;      // scan scratch
    ws::LargeList large;  // hand-over list of large patches
    float2* Radj;       // K_w x fstride flipped conjugate taps (adjoint)
    float2* Racc;       // K_w x fstride response-gradient spectra
    int impacts;        // sub-pitch response positions (1: none)
    float* fine;        // nwires*impacts x nticks fine grid (impacts > 1)
    float* noise_amp;   // fstride noise amplitudes (incoherent), then fstride coherent
    int noise_mode;     // 0 none, 1 incoherent, 2 incoherent + coherent
    int noise_group;    // wires per coherent group
    float* grid2;       // nwires x nticks float scratch grid (adjoint, compensated low parts)
    bool fp64;          // FP64 buffers present
    double2* tw64;      // FP64 pass twiddles
    double2* Rt64;      // FP64 response spectrum
    double2* X64;       // FP64 spectra
    double2* Y64;
    double* g64;        // FP64 grid
    ws::mark_t* rows;        // nwires active-row marks (ws_simulate)
    ws::mark_t* rows_epoch;  // their epoch words (ws::RowMarks epoch and base, status region)
    ws::mark_t* rows_base;
    unsigned* sched;         // impact wire convolution's claim counter and finished CTAs (status region)
    uint32_t* row_cls;       // nwires row classes (ws_simulate)
};
