// C ABI of the wiresim library (include/wiresim.h): argument checking, the
// FFT planner, the workspace layout and the launch sequences of each entry
// point.  No entry point allocates device memory; all device storage is the
// caller's (the plane's workspace, depo arrays, grids, patch buffers).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ws_internal.cuh"

// Per-plane launch trace: a ring of (kernel, start event, end event) records
// filled while tracing is on and aggregated by ws_plane_trace_read.
struct ws_trace {
    std::vector<cudaEvent_t> start, stop;
    std::vector<int> kind;
    int used = 0;
    int64_t dropped = 0;
};

namespace {

thread_local char g_last_error[256] = "";

const char* const kKernelNames[] = {"memset_grid", "raster_scatter", "fwd_rows", "wire_conv", "inv_rows",
                                    "patch_sizes", "scan", "raster_patches", "scatter_patches", "depo_grads",
                                    "resp_grad", "add_noise", "mark_rows"};
enum { K_MEMSET, K_RASTER_SCATTER, K_FWD, K_WCONV, K_INV, K_SIZES, K_SCAN, K_RPATCH, K_SCATTER, K_DGRAD,
       K_RGRAD, K_NOISE, K_MARK, K_COUNT };

// Record a start event for a traced launch; returns the record slot or -1.
int trace_begin(ws_plane* pl, int kind, cudaStream_t s) {
    ws_trace* t = pl->trace;
    if (!t) return -1;
    if (t->used >= (int)t->start.size()) { ++t->dropped; return -1; }
    const int i = t->used++;
    t->kind[i] = kind;
    cudaEventRecord(t->start[i], s);
    return i;
}

void trace_end(ws_plane* pl, int slot, cudaStream_t s) {
    if (slot >= 0) cudaEventRecord(pl->trace->stop[slot], s);
}


// Host logging of failures: set WS_LOG (to anything) in the environment.
bool log_enabled() {
    static const bool on = getenv("WS_LOG") != nullptr;
    return on;
}

ws_status cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", where, cudaGetErrorString(e));
    if (log_enabled()) fprintf(stderr, "wiresim: %s\n", g_last_error);
    return WS_ERR_CUDA;
}

// An NVTX range over an entry point's host work (its launches), for
// profilers; costs nothing when no tool listens.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

#define WS_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// A launch bracketed by trace events when the plane is tracing.
#define WS_LAUNCH(pl, kind, s, call)                    \
    do {                                                \
        const int slot_ = trace_begin((pl), (kind), (s)); \
        cudaError_t e_ = (call);                        \
        trace_end((pl), slot_, (s));                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool smooth235(int n) {
    if (n <= 0) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

int next_smooth(int n) {
    while (!smooth235(n)) ++n;
    return n;
}

// Radix passes for L: greedily the largest supported radix that divides
// what is left (25, 16, 20, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2), so a 6250-point
// transform is 25 x 25 x 10 and a 6000-point one 25 x 16 x 15.
bool make_plan(int L, ws::FftPlan* p) {
    if (!smooth235(L) || L < 2 || L > ws::kMaxFftLen) return false;
    static const int kRadices[] = {25, 16, 20, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
    p->L = L;
    p->npass = 0;
    int n = L, ns = 1, off = 0;
    while (n > 1) {
        int r = 0;
        for (int c : kRadices)
            if (n % c == 0) { r = c; break; }
        if (r == 0 || p->npass >= ws::kMaxPasses) return false;
        p->radix[p->npass] = r;
        p->ns[p->npass] = ns;
        p->twoff[p->npass] = off;
        off += ns;
        ns *= r;
        n /= r;
        ++p->npass;
    }
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    ws::FftPlan plan;
    int nfreq, fstride;
    size_t off_status, off_tw, off_rt, off_x, off_y, off_scan, off_large, off_radj, off_racc, off_grid2, off_noise,
        off_rows, off_cls;
    size_t off_fine;
    int impacts;
    size_t off_tw64, off_rt64, off_x64, off_y64, off_g64, total;
};

ws_status plan_layout(const ws_plane_desc* d, Layout* lay) {
    if (!d) return WS_ERR_INVALID_ARG;
    if (d->nwires <= 0 || d->nticks <= 0 || d->resp_nwires <= 0 || d->resp_nticks <= 0 ||
        d->resp_wire_center < 0 || d->resp_wire_center >= d->resp_nwires || !(d->pitch_mm > 0) ||
        !(d->tick_us > 0) || !(d->nsigma > 0) || d->plane_id < 0 || d->plane_id > 15 ||
        (d->conv_mode != WS_CONV_LINEAR && d->conv_mode != WS_CONV_CIRCULAR) || d->fft_len_tick < 0)
        return WS_ERR_INVALID_ARG;
    if (d->resp_nwires > ws::kMaxRespWires) return WS_ERR_UNSUPPORTED_SIZE;
    if (d->impacts < 0 || d->impacts > ws::kMaxImpacts) return WS_ERR_INVALID_ARG;
    const int I = d->impacts > 1 ? d->impacts : 1;
    if ((int64_t)I * d->nwires * d->nticks > (int64_t)INT32_MAX) return WS_ERR_UNSUPPORTED_SIZE;   // 32-bit bin index
    lay->impacts = I;
    int L;
    if (d->fft_len_tick > 0) {
        L = d->fft_len_tick;
        if (d->conv_mode == WS_CONV_LINEAR && L < d->nticks + d->resp_nticks - 1) return WS_ERR_INVALID_ARG;
        if (d->conv_mode == WS_CONV_CIRCULAR && L != d->nticks) return WS_ERR_INVALID_ARG;
    } else {
        if (d->conv_mode == WS_CONV_LINEAR) {
            L = next_smooth(d->nticks + d->resp_nticks - 1);
            if (L < 2) L = 2;
        } else {
            L = d->nticks;
        }
    }
    if (d->resp_nticks > L) return WS_ERR_UNSUPPORTED_SIZE;
    if (!make_plan(L, &lay->plan)) return WS_ERR_UNSUPPORTED_SIZE;
    lay->nfreq = L / 2 + 1;
    lay->fstride = (lay->nfreq + 31) & ~31;
    size_t o = 0;
    lay->off_status = o; o = align256(o + 256);
    lay->off_tw = o; o = align256(o + sizeof(float2) * (size_t)L);
    lay->off_rt = o; o = align256(o + sizeof(float2) * (size_t)I * d->resp_nwires * lay->fstride);
    lay->off_x = o; o = align256(o + sizeof(float2) * (size_t)I * d->nwires * lay->fstride);
    lay->off_y = o; o = align256(o + sizeof(float2) * (size_t)d->nwires * lay->fstride);
    lay->off_scan = o; o = align256(o + sizeof(int64_t) * (size_t)ws::kScanScratch);
    lay->off_large = o; o = align256(o + sizeof(long long) * (size_t)ws::kLargeListCap);
    lay->off_radj = o; o = align256(o + sizeof(float2) * (size_t)I * d->resp_nwires * lay->fstride);
    lay->off_racc = o; o = align256(o + sizeof(float2) * (size_t)I * d->resp_nwires * lay->fstride);
    lay->off_grid2 = o; o = align256(o + sizeof(float) * (size_t)I * d->nwires * d->nticks);
    lay->off_noise = o; o = align256(o + 2 * sizeof(float) * (size_t)lay->fstride);
    lay->off_rows = o; o = align256(o + sizeof(ws::mark_t) * (size_t)d->nwires);
    lay->off_cls = o; o = align256(o + sizeof(uint32_t) * (size_t)d->nwires);
    lay->off_fine = 0;
    if (I > 1) { lay->off_fine = o; o = align256(o + sizeof(float) * (size_t)I * d->nwires * d->nticks); }
    lay->off_tw64 = lay->off_rt64 = lay->off_x64 = lay->off_y64 = lay->off_g64 = 0;
    if (d->fp64) {
        lay->off_tw64 = o; o = align256(o + sizeof(double2) * (size_t)L);
        lay->off_rt64 = o; o = align256(o + sizeof(double2) * (size_t)I * d->resp_nwires * lay->fstride);
        lay->off_x64 = o; o = align256(o + sizeof(double2) * (size_t)I * d->nwires * lay->fstride);
        lay->off_y64 = o; o = align256(o + sizeof(double2) * (size_t)d->nwires * lay->fstride);
        lay->off_g64 = o; o = align256(o + sizeof(double) * (size_t)I * d->nwires * d->nticks);
    }
    lay->total = o;
    return WS_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// Patch arrays are read and written as their element types (a null pointer
// counts as aligned; the callers check which may be null).
bool patches_aligned(const ws_patches* p) {
    return aligned(p->val, 4) && aligned(p->w0, 4) && aligned(p->t0, 4) && aligned(p->nw, 4) && aligned(p->nt, 4) &&
           aligned(p->off, 8);
}

ws_status check_depos(const ws_depos* d) {
    if (!d || d->n < 0) return WS_ERR_INVALID_ARG;
    if (d->n == 0) return WS_OK;
    if (!d->q || !d->x_mm || !d->t_us) return WS_ERR_INVALID_ARG;
    if ((d->sigma_t_us == nullptr) != (d->sigma_x_mm == nullptr)) return WS_ERR_INVALID_ARG;
    if (!aligned(d->q, 4) || !aligned(d->x_mm, 4) || !aligned(d->t_us, 4)) return WS_ERR_INVALID_ARG;
    if (d->sigma_t_us && (!aligned(d->sigma_t_us, 4) || !aligned(d->sigma_x_mm, 4))) return WS_ERR_INVALID_ARG;
    if (d->n > ((int64_t)1 << 32)) return WS_ERR_UNSUPPORTED_SIZE;  // depo index is a 32-bit counter word
    return WS_OK;
}

// The depos' indices in the event's list (depo_offset + i) fit the
// counters' 32-bit depo word.
ws_status check_depo_span(const ws_depos* d, const ws_params* p) {
    return (uint64_t)p->depo_offset + (uint64_t)d->n > ((uint64_t)1 << 32) ? WS_ERR_INVALID_ARG : WS_OK;
}

ws_status check_params(const ws_params* p) {
    if (!p) return WS_ERR_INVALID_ARG;
    if (!(p->v_mm_us > 0) || !(p->DL_mm2_us >= 0) || !(p->DT_mm2_us >= 0)) return WS_ERR_INVALID_ARG;
    if (!(p->p_survive >= 0) || !(p->p_survive <= 1)) return WS_ERR_INVALID_ARG;
    if (p->event_id >= (1u << 28)) return WS_ERR_INVALID_ARG;
    if (p->fluct_exact_max < 0 || p->fluct_exact_max > ws::kExactCap) return WS_ERR_INVALID_ARG;
    if (p->fluctuate < 0 || p->fluctuate > 2) return WS_ERR_INVALID_ARG;
    if (p->precision != WS_PREC_FP32 && p->precision != WS_PREC_FP32_COMP && p->precision != WS_PREC_FP64)
        return WS_ERR_INVALID_ARG;
    return WS_OK;
}

ws::RasterArgs raster_args(const ws_plane* pl, const ws_depos* d, const ws_params* p) {
    ws::RasterArgs a;
    a.q = d->q; a.x = d->x_mm; a.t = d->t_us;
    a.sig_t = d->sigma_t_us; a.sig_x = d->sigma_x_mm;
    a.n = d->n;
    // impact planes bin the pitch axis at pitch / I (fine row w * I + i)
    a.nwires = pl->desc.nwires * pl->impacts; a.nticks = pl->desc.nticks;
    a.pitch = (float)(pl->desc.pitch_mm / pl->impacts); a.tick = (float)pl->desc.tick_us;
    a.nsig = (float)pl->desc.nsigma;
    a.two_DL = (float)(2.0 * p->DL_mm2_us);
    a.two_DT = (float)(2.0 * p->DT_mm2_us);
    a.inv_v = (float)(1.0 / p->v_mm_us);
    a.fluct = p->fluctuate;
    a.p = (float)p->p_survive;
    if (!(p->p_survive > 0)) a.T = 0u;
    else if (p->p_survive >= 1.0) a.T = 0xFFFFFFFFu;
    else a.T = (uint32_t)floor(p->p_survive * 4294967296.0);
    a.key0 = (uint32_t)(p->seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(p->seed >> 32);
    a.evpl = (p->event_id << 4) | ((uint32_t)pl->desc.plane_id & 15u);
    a.depo0 = p->depo_offset;
    a.keep_all = p->p_survive >= 1.0 ? 1 : 0;
    a.exact_max = p->fluct_exact_max;
    a.wide = pl->impacts > 1 ? 1 : 0;
    {
        const float pf = a.p;
        a.inv_flip = pf > 0.5f ? 1 : 0;
        const float sv = a.inv_flip ? 1.0f - pf : pf;
        a.inv_base = 1.0f - sv;
        a.inv_r = sv / a.inv_base;
    }
    a.status = pl->status;
    a.prec = p->precision;
    a.lo = nullptr;
    a.grid64 = nullptr;
    a.two_DL64 = 2.0 * p->DL_mm2_us;
    a.two_DT64 = 2.0 * p->DT_mm2_us;
    a.v64 = p->v_mm_us;
    a.pitch64 = pl->desc.pitch_mm / pl->impacts;
    a.tick64 = pl->desc.tick_us;
    a.nsig64 = pl->desc.nsigma;
    a.p64 = p->p_survive;
    return a;
}

// The plane's noise term for one simulation call (false: no noise set).
bool noise_unit(const ws_plane* pl, uint32_t event_id, ws::NoiseUnit* nz) {
    if (pl->noise_mode == 0) return false;
    nz->amp = pl->noise_amp;
    nz->coh = pl->noise_mode == 2 ? pl->noise_amp + pl->fstride : nullptr;
    nz->group = pl->noise_group;
    nz->evpl = (event_id << 4) | ((uint32_t)pl->desc.plane_id & 15u);
    nz->scale = 1.0 / (double)pl->plan.L;
    return true;
}

// One plane's noise over its spectra Y (float2, or double2 for the FP64
// path) if the plane has noise set.
ws_status add_plane_noise(ws_plane* pl, const ws_params* p, void* Y, bool fp64, cudaStream_t s) {
    ws::NoiseBatch nb;
    if (!noise_unit(pl, p->event_id, &nb.noise[0])) return WS_OK;
    nb.n = 1;
    nb.Y[0] = Y;
    nb.nwires[0] = pl->desc.nwires;
    nb.key0 = (uint32_t)(p->seed & 0xFFFFFFFFu);
    nb.key1 = (uint32_t)(p->seed >> 32);
    if (fp64) {
        WS_LAUNCH(pl, K_NOISE, s, ws::launch_add_noise64(nb, pl->nfreq, pl->plan.L, pl->fstride, s));
    } else {
        WS_LAUNCH(pl, K_NOISE, s, ws::launch_add_noise(nb, pl->nfreq, pl->plan.L, pl->fstride, s));
    }
    return WS_OK;
}

// Whether a plane's simulations skip inactive rows: FP32 fixed-shape row
// transforms, linear convolution (windows do not wrap) and no noise term
// (noise makes every row of the output live).  An impact plane marks whole
// wires (its I fine rows together); its wire convolution is the TMA one.
bool marks_apply(const ws_plane* pl) {
    return pl->desc.conv_mode == WS_CONV_LINEAR && pl->noise_mode == 0 && ws::row_fft_fixed_shape(pl->plan) &&
           (pl->impacts == 1 || ws::tma_available());
}

// The impact wire convolution of the units of cb (fine spectra X -> Y; the
// planes share I, the convolution mode and the response width, pl is one
// of them), with the call's marks or without (rows null); the launches are
// traced on plane `tr`.
ws_status impacts_wconv(ws_plane* pl, ws_plane* tr, const ws::ConvBatch& cb, unsigned* sched, cudaStream_t s,
                        int variant) {
    const ws_plane_desc& d = pl->desc;
    if (d.conv_mode == WS_CONV_LINEAR && ws::tma_available()) {
        WS_LAUNCH(tr, K_WCONV, s, ws::launch_wire_conv_impacts_tma(cb, pl->impacts, pl->nfreq, pl->fstride,
                                                                   d.resp_nwires, d.resp_wire_center, sched,
                                                                   pl->status, s, variant));
        return WS_OK;
    }
    for (int j = 0; j < cb.n; ++j) {
        if (cb.rows[j]) return WS_ERR_UNSUPPORTED_SIZE;
        WS_LAUNCH(tr, K_WCONV, s, ws::launch_wire_conv_impacts((const float2*)cb.X[j], (float2*)cb.Y[j],
                                                               (const float2*)cb.Rt[j], cb.nwires[j], pl->impacts,
                                                               pl->nfreq, pl->fstride, d.resp_nwires,
                                                               d.resp_wire_center, d.conv_mode == WS_CONV_CIRCULAR,
                                                               s));
    }
    return WS_OK;
}

// One plane's spectra as a one-unit convolution batch (marks optional).
ws::ConvBatch plane_conv(const ws_plane* pl, const ws::mark_t* rows, const ws::mark_t* epoch) {
    ws::ConvBatch cb;
    cb.n = 1;
    cb.X[0] = pl->X;
    cb.Y[0] = pl->Y;
    cb.Rt[0] = pl->Rt;
    cb.nwires[0] = pl->desc.nwires;
    cb.rows[0] = rows;
    cb.epoch = epoch;
    return cb;
}

// ws_simulate_backward on an impact plane (M = sum_i R_i (*) S_i over the
// fine rows S_i[w] = S_fine[w * I + i]): G's tick transform once (into Y);
// dL/dR_i from the recomputed fine grid, its I positions transformed in
// one launch (into X, I x nwires rows), correlated with G's spectrum slice
// by slice and inverse-transformed in one launch; dL/dS_fine from the I
// correlations of G's spectrum with the slices' adjoint taps (one launch
// over I units into X) and one inverse transform storing every I-th fine
// row per position; then the depo gradients of the raster on the fine
// grid.  The plane's fine grid holds S, then dL/dS.
ws_status backward_impacts(ws_plane* pl, const ws_depos* depos, const ws_params* params, const float* G,
                           float* gq, float* gx, float* gt, double* gDL, double* gDT, float* gR, cudaStream_t s) {
    const ws_plane_desc& d = pl->desc;
    const int I = pl->impacts, circ = d.conv_mode == WS_CONV_CIRCULAR;
    const int64_t fine_stride = (int64_t)I * d.nticks;
    const size_t slice = (size_t)d.resp_nwires * pl->fstride;   // one slice's response spectrum rows
    const size_t rows = (size_t)d.nwires * pl->fstride;          // one position's spectra
    ws::RasterArgs a = raster_args(pl, depos, params);
    WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows(pl->plan, pl->tw, G, d.nwires, d.nticks, d.nticks, pl->Y,
                                                pl->fstride, pl->nfreq, 1.0f, s));
    ws::RowBatch fb, ib;
    fb.n = ib.n = I;
    fb.status = ib.status = nullptr;
    if (gR) {
        const size_t fine_bytes = sizeof(float) * (size_t)I * d.nwires * d.nticks;
        WS_LAUNCH(pl, K_MEMSET, s, cudaMemsetAsync(pl->fine, 0, fine_bytes, s));
        WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, pl->fine, pl->large, s));
        for (int i = 0; i < I; ++i) {
            fb.in[i] = pl->fine + (size_t)i * d.nticks;
            fb.in2[i] = nullptr;
            fb.out[i] = pl->X + (size_t)i * rows;
            fb.nrows[i] = d.nwires;
            ib.in[i] = pl->Racc + (size_t)i * slice;
            ib.in2[i] = nullptr;
            ib.out[i] = gR + (size_t)i * d.resp_nwires * d.resp_nticks;
            ib.nrows[i] = d.resp_nwires;
        }
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows_batch(pl->plan, pl->tw, fb, d.nticks, fine_stride, pl->fstride,
                                                          pl->nfreq, 1.0f, s));
        WS_CUDA(cudaMemsetAsync(pl->Racc, 0, sizeof(float2) * slice * I, s));
        for (int i = 0; i < I; ++i)
            WS_LAUNCH(pl, K_RGRAD, s, ws::launch_resp_grad(pl->Y, pl->X + (size_t)i * rows, pl->Racc + (size_t)i * slice,
                                                           d.nwires, pl->nfreq, pl->fstride, d.resp_nwires,
                                                           d.resp_wire_center, circ, 1.0f / (float)pl->plan.L, s));
        WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows_batch(pl->plan, pl->tw, ib, pl->fstride, pl->nfreq, d.resp_nticks,
                                                          d.resp_nticks, s));
    }
    ws::ConvBatch cb;
    cb.n = I;
    for (int i = 0; i < I; ++i) {
        cb.X[i] = pl->Y;
        cb.Y[i] = pl->X + (size_t)i * rows;
        cb.Rt[i] = pl->Radj + (size_t)i * slice;
        cb.nwires[i] = d.nwires;
        ib.in[i] = pl->X + (size_t)i * rows;
        ib.in2[i] = nullptr;
        ib.out[i] = pl->fine + (size_t)i * d.nticks;
        ib.nrows[i] = d.nwires;
    }
    const int variant = (circ || !ws::tma_available()) ? 0 : 9;
    WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv_batch(cb, pl->nfreq, pl->fstride, d.resp_nwires,
                                                         d.resp_nwires - 1 - d.resp_wire_center, circ, s, variant,
                                                         pl->status));
    WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows_batch(pl->plan, pl->tw, ib, pl->fstride, pl->nfreq, d.nticks,
                                                      fine_stride, s));
    if (gDL) WS_CUDA(cudaMemsetAsync(gDL, 0, sizeof(double), s));
    if (gDT) WS_CUDA(cudaMemsetAsync(gDT, 0, sizeof(double), s));
    WS_LAUNCH(pl, K_DGRAD, s, ws::launch_depo_grads(a, pl->fine, gq, gx, gt, gDL, gDT, params->DL_mm2_us,
                                                    params->DT_mm2_us, pl->large, s));
    return WS_OK;
}

// ws_simulate's FP32 / compensated path with active rows: mark, clear the
// marked rows, raster, then the three transform stages over marked / live
// rows only (the same result as clearing and transforming every row).  The
// grid is `out` itself, or the fine grid of an impact plane.
ws_status simulate_marked(ws_plane* pl, ws::RasterArgs a, float* out, cudaStream_t s) {
    const ws_plane_desc& d = pl->desc;
    const int I = pl->impacts;
    float* grid = I > 1 ? pl->fine : out;
    ws::RasterBatch rb;
    rb.n = 1;
    rb.prec = a.prec;
    rb.a[0] = a;
    rb.grid[0] = grid;
    ws::RowMarks m;
    m.rows[0] = pl->rows;
    m.cls[0] = pl->row_cls;
    m.epoch = pl->rows_epoch;
    m.base = pl->rows_base;
    m.kw = d.resp_nwires;
    m.center = d.resp_wire_center;
    m.impacts[0] = I;
    WS_LAUNCH(pl, K_MARK, s, ws::launch_mark_rows(rb, m, s));
    WS_LAUNCH(pl, K_MEMSET, s, ws::launch_zero_marked_rows(rb, m, s));
    WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, grid, pl->large, s));
    ws::RowBatch fb, ib;
    fb.n = ib.n = 1;
    fb.in[0] = grid;
    fb.in2[0] = a.lo;
    fb.out[0] = pl->X;
    fb.nrows[0] = d.nwires * I;
    fb.rdiv[0] = I;
    ib.in[0] = pl->Y;
    ib.in2[0] = nullptr;
    ib.out[0] = out;
    ib.nrows[0] = d.nwires;
    fb.status = ib.status = pl->status;
    fb.rows[0] = ib.rows[0] = pl->row_cls;
    WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows_batch(pl->plan, pl->tw, fb, d.nticks, d.nticks, pl->fstride,
                                                      pl->nfreq, 1.0f, s));
    const ws::ConvBatch cb = plane_conv(pl, pl->rows, pl->rows_epoch);
    if (I > 1) {
        const ws_status st = impacts_wconv(pl, pl, cb, pl->sched, s, pl->wconv_variant);
        if (st != WS_OK) return st;
    } else {
        WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv_batch(cb, pl->nfreq, pl->fstride, d.resp_nwires,
                                                             d.resp_wire_center, 0, s, pl->wconv_variant, pl->status));
    }
    WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows_batch(pl->plan, pl->tw, ib, pl->fstride, pl->nfreq, d.nticks,
                                                      d.nticks, s));
    return WS_OK;
}

// Eq. 2 on a grid (the fine grid of an impact plane), adding the plane's
// noise term with noise_params; lo: the compensated grid's low parts (added
// by the forward transform), or null.
ws_status convolve_impl(ws_plane* pl, const float* grid, float* out, cudaStream_t s,
                        const ws_params* noise_params = nullptr, const float* lo = nullptr) {
    const ws_plane_desc& d = pl->desc;
    if (lo) {
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows_comp(pl->plan, pl->tw, grid, lo, d.nwires * pl->impacts, d.nticks,
                                                         d.nticks, pl->X, pl->fstride, pl->nfreq, s));
    } else {
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows(pl->plan, pl->tw, grid, d.nwires * pl->impacts, d.nticks,
                                                    d.nticks, pl->X, pl->fstride, pl->nfreq, 1.0f, s, pl->status));
    }
    if (pl->impacts > 1) {
        const ws_status st =
            impacts_wconv(pl, pl, plane_conv(pl, nullptr, nullptr), pl->sched, s, pl->wconv_variant);
        if (st != WS_OK) return st;
    } else {
        WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv(pl->X, pl->Y, pl->Rt, d.nwires, pl->nfreq, pl->fstride,
                                                       d.resp_nwires, d.resp_wire_center,
                                                       d.conv_mode == WS_CONV_CIRCULAR, s, pl->wconv_variant,
                                                       pl->status));
    }
    if (noise_params) {
        const ws_status st = add_plane_noise(pl, noise_params, pl->Y, false, s);
        if (st != WS_OK) return st;
    }
    WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows(pl->plan, pl->tw, pl->Y, d.nwires, pl->fstride, pl->nfreq, out,
                                                d.nticks, d.nticks, s, pl->status));
    return WS_OK;
}

}  // namespace

namespace ws {
// Transform plan of a plane description (same planner as ws_plane_create).
ws_status conv_plan(const ws_plane_desc* desc, FftPlan* plan, int* nfreq, int* fstride) {
    Layout lay;
    ws_status st = plan_layout(desc, &lay);
    if (st != WS_OK) return st;
    *plan = lay.plan;
    *nfreq = lay.nfreq;
    *fstride = lay.fstride;
    return WS_OK;
}

ws_status record_cuda_error(cudaError_t e, const char* where) { return cuda_fail(e, where); }
}  // namespace ws

extern "C" {

const char* ws_status_string(ws_status s) {
    switch (s) {
        case WS_OK: return "ok";
        case WS_ERR_INVALID_ARG: return "invalid argument";
        case WS_ERR_UNSUPPORTED_SIZE: return "unsupported size";
        case WS_ERR_OOM: return "out of host memory";
        case WS_ERR_CUDA: return "CUDA error";
        case WS_ERR_TIMEOUT: return "device wait timed out";
        case WS_ERR_WORKSPACE: return "workspace too small or misaligned";
        case WS_ERR_BAD_INPUT: return "bad input data";
    }
    return "unknown status";
}

const char* ws_last_error(void) { return g_last_error; }

ws_status ws_plane_workspace_bytes(const ws_plane_desc* desc, size_t* bytes) {
    if (!bytes) return WS_ERR_INVALID_ARG;
    Layout lay;
    ws_status st = plan_layout(desc, &lay);
    if (st != WS_OK) return st;
    *bytes = lay.total;
    return WS_OK;
}

ws_status ws_plane_create(const ws_plane_desc* desc, const float* response_dev, void* workspace_dev,
                          size_t workspace_bytes, void* stream, ws_plane** out) {
    if (!out || !response_dev) return WS_ERR_INVALID_ARG;
    *out = nullptr;
    Layout lay;
    ws_status st = plan_layout(desc, &lay);
    if (st != WS_OK) return st;
    if (!workspace_dev || !aligned(workspace_dev, 256) || workspace_bytes < lay.total) return WS_ERR_WORKSPACE;
    if (!aligned(response_dev, 4)) return WS_ERR_INVALID_ARG;
    ws_plane* pl = new (std::nothrow) ws_plane;
    if (!pl) return WS_ERR_OOM;
    pl->trace = nullptr;
    char* base = (char*)workspace_dev;
    pl->desc = *desc;
    pl->plan = lay.plan;
    pl->nfreq = lay.nfreq;
    pl->fstride = lay.fstride;
    pl->ws_bytes = lay.total;
    pl->status = (uint32_t*)(base + lay.off_status);
    pl->counter = (unsigned long long*)(base + lay.off_status + 8);
    pl->tw = (float2*)(base + lay.off_tw);
    pl->Rt = (float2*)(base + lay.off_rt);
    pl->X = (float2*)(base + lay.off_x);
    pl->Y = (float2*)(base + lay.off_y);
    pl->scan = (int64_t*)(base + lay.off_scan);
    pl->large.list = (long long*)(base + lay.off_large);
    pl->large.count = (unsigned*)(base + lay.off_status + 16);
    pl->large.done = (unsigned*)(base + lay.off_status + 20);
    pl->large.cap = ws::kLargeListCap;
    pl->Radj = (float2*)(base + lay.off_radj);
    pl->Racc = (float2*)(base + lay.off_racc);
    pl->grid2 = (float*)(base + lay.off_grid2);
    pl->noise_amp = (float*)(base + lay.off_noise);
    pl->impacts = lay.impacts;
    pl->fine = lay.impacts > 1 ? (float*)(base + lay.off_fine) : nullptr;
    pl->noise_mode = 0;
    pl->noise_group = 1;
    pl->fp64 = desc->fp64 != 0;
    pl->tw64 = pl->fp64 ? (double2*)(base + lay.off_tw64) : nullptr;
    pl->Rt64 = pl->fp64 ? (double2*)(base + lay.off_rt64) : nullptr;
    pl->X64 = pl->fp64 ? (double2*)(base + lay.off_x64) : nullptr;
    pl->Y64 = pl->fp64 ? (double2*)(base + lay.off_y64) : nullptr;
    pl->g64 = pl->fp64 ? (double*)(base + lay.off_g64) : nullptr;
    pl->rows = (ws::mark_t*)(base + lay.off_rows);
    pl->rows_epoch = (ws::mark_t*)(base + lay.off_status + 24);   // zeroed with the status region below
    pl->rows_base = (ws::mark_t*)(base + lay.off_status + 32);
    pl->sched = (unsigned*)(base + lay.off_status + 40);
    pl->row_cls = (uint32_t*)(base + lay.off_cls);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(base + lay.off_status, 0, 256, s);
    // marks start below every epoch (the first call marks with 1)
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->rows, 0, sizeof(ws::mark_t) * (size_t)desc->nwires, s);
    if (e == cudaSuccess) e = ws::launch_twiddles(pl->tw, lay.plan, s);
    // Response spectrum: per response row, the tick transform scaled by 1/L so
    // that the inverse transform needs no scaling.
    if (e == cudaSuccess)
        e = ws::launch_fwd_rows(lay.plan, pl->tw, response_dev, lay.impacts * desc->resp_nwires, desc->resp_nticks,
                                desc->resp_nticks, pl->Rt, lay.fstride, lay.nfreq, 1.0f / (float)lay.plan.L, s);
    for (int i = 0; i < lay.impacts && e == cudaSuccess; ++i)   // one adjoint tap set per response slice
        e = ws::launch_adj_coeffs(pl->Rt + (size_t)i * desc->resp_nwires * lay.fstride,
                                  pl->Radj + (size_t)i * desc->resp_nwires * lay.fstride, desc->resp_nwires,
                                  lay.fstride, lay.nfreq, s);
    if (e == cudaSuccess && pl->fp64) e = ws::launch_twiddles64(pl->tw64, lay.plan, s);
    if (e == cudaSuccess && pl->fp64)
        e = ws::launch_fwd_rows64(lay.plan, pl->tw64, response_dev, false, lay.impacts * desc->resp_nwires,
                                  desc->resp_nticks,
                                  desc->resp_nticks, pl->Rt64, lay.fstride, lay.nfreq, 1.0f / (float)lay.plan.L, s);
    // Autotune the wire convolution on this plane's own buffers: every
    // variant once to warm up, then three rounds over all variants of three
    // timed launches each (rounds interleave the variants, so a drifting
    // clock biases none); a variant's time is its best round, and the
    // fastest variant is kept.
    pl->wconv_variant = 0;
    pl->batch_upw = 0;
    pl->batch_wconv = -1;
    if (e == cudaSuccess)
        e = cudaMemsetAsync(pl->X, 0, sizeof(float2) * (size_t)lay.impacts * desc->nwires * lay.fstride, s);
    const int circ = desc->conv_mode == WS_CONV_CIRCULAR;
    // impact planes: the TMA kernel's two wire-block sizes (linear mode), else
    // their one generic kernel
    const int nvar = lay.impacts > 1 ? ((circ || !ws::tma_available()) ? 1 : ws::kImpactConvVariants)
                                     : ((circ || !ws::tma_available()) ? 4 : ws::kWireConvVariants);
    if (e == cudaSuccess && nvar > 1) {
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        e = cudaEventCreate(&t0);
        if (e == cudaSuccess) e = cudaEventCreate(&t1);
        float best_of[ws::kWireConvVariants];
        for (int v = 0; v < nvar; ++v) best_of[v] = 1e30f;
        auto conv = [&](int v) {
            if (lay.impacts > 1)
                return ws::launch_wire_conv_impacts_tma(plane_conv(pl, nullptr, nullptr), lay.impacts, lay.nfreq,
                                                        lay.fstride, desc->resp_nwires, desc->resp_wire_center,
                                                        pl->sched, pl->status, s, v);
            return ws::launch_wire_conv(pl->X, pl->Y, pl->Rt, desc->nwires, lay.nfreq, lay.fstride,
                                        desc->resp_nwires, desc->resp_wire_center, circ, s, v, pl->status);
        };
        for (int v = 0; v < nvar && e == cudaSuccess; ++v) e = conv(v);
        for (int round = 0; round < 3 && e == cudaSuccess; ++round) {
            for (int v = 0; v < nvar && e == cudaSuccess; ++v) {
                e = cudaEventRecord(t0, s);
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = conv(v);
                if (e == cudaSuccess) e = cudaEventRecord(t1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e == cudaSuccess && ms < best_of[v]) best_of[v] = ms;
            }
        }
        for (int v = 1; v < nvar; ++v)
            if (best_of[v] < best_of[pl->wconv_variant]) pl->wconv_variant = v;
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
    }
    if (e != cudaSuccess) {
        delete pl;
        return cuda_fail(e, "ws_plane_create");
    }
    *out = pl;
    return WS_OK;
}

static void trace_free(ws_plane* pl) {
    if (!pl->trace) return;
    for (size_t i = 0; i < pl->trace->start.size(); ++i) {
        cudaEventDestroy(pl->trace->start[i]);
        cudaEventDestroy(pl->trace->stop[i]);
    }
    delete pl->trace;
    pl->trace = nullptr;
}

ws_status ws_plane_destroy(ws_plane* plane) {
    if (plane) trace_free(plane);
    delete plane;
    return WS_OK;
}

ws_status ws_plane_set_wire_conv_variant(ws_plane* pl, int variant) {
    if (!pl || variant < 0 || variant >= ws::kWireConvVariants) return WS_ERR_INVALID_ARG;
    if (pl->impacts > 1) {   // the TMA impact kernel's wire blocks of 16 / 32 (linear mode)
        if (variant >= ws::kImpactConvVariants) return WS_ERR_UNSUPPORTED_SIZE;
        if (variant > 0 && (pl->desc.conv_mode == WS_CONV_CIRCULAR || !ws::tma_available()))
            return WS_ERR_UNSUPPORTED_SIZE;
    }
    if (variant >= 4 && (pl->desc.conv_mode == WS_CONV_CIRCULAR || !ws::tma_available())) return WS_ERR_UNSUPPORTED_SIZE;
    pl->wconv_variant = variant;
    pl->batch_wconv = variant;   // an explicit choice holds for batches too
    return WS_OK;
}

ws_status ws_plane_trace(ws_plane* pl, int max_records) {
    if (!pl || max_records < 0) return WS_ERR_INVALID_ARG;
    trace_free(pl);
    if (max_records == 0) return WS_OK;
    ws_trace* t = new (std::nothrow) ws_trace;
    if (!t) return WS_ERR_OOM;
    t->start.resize(max_records);
    t->stop.resize(max_records);
    t->kind.resize(max_records);
    for (int i = 0; i < max_records; ++i) {
        cudaError_t e = cudaEventCreate(&t->start[i]);
        if (e == cudaSuccess) e = cudaEventCreate(&t->stop[i]);
        if (e != cudaSuccess) {
            t->start.resize(i);
            t->stop.resize(i);
            pl->trace = t;
            trace_free(pl);
            return cuda_fail(e, "ws_plane_trace");
        }
    }
    pl->trace = t;
    return WS_OK;
}

ws_status ws_plane_trace_read(ws_plane* pl, ws_trace_stat* stats, int max_stats, int* nstats) {
    if (!pl || !nstats || (max_stats > 0 && !stats)) return WS_ERR_INVALID_ARG;
    *nstats = 0;
    ws_trace* t = pl->trace;
    if (!t) return WS_OK;
    double ms[K_COUNT] = {0};
    int64_t cnt[K_COUNT] = {0};
    for (int i = 0; i < t->used; ++i) {
        WS_CUDA(cudaEventSynchronize(t->stop[i]));
        float m = 0.f;
        WS_CUDA(cudaEventElapsedTime(&m, t->start[i], t->stop[i]));
        ms[t->kind[i]] += m;
        cnt[t->kind[i]] += 1;
    }
    int n = 0;
    for (int k = 0; k < K_COUNT; ++k) {
        if (!cnt[k]) continue;
        if (n < max_stats) {
            stats[n].name = kKernelNames[k];
            stats[n].launches = cnt[k];
            stats[n].total_ms = ms[k];
        }
        ++n;
    }
    *nstats = n < max_stats ? n : max_stats;
    t->used = 0;
    t->dropped = 0;
    return WS_OK;
}

ws_status ws_plane_get_info(const ws_plane* pl, ws_plane_info* info) {
    if (!pl || !info) return WS_ERR_INVALID_ARG;
    memset(info, 0, sizeof *info);
    info->fft_len_tick = pl->plan.L;
    info->nfreq = pl->nfreq;
    info->nfreq_stride = pl->fstride;
    info->npasses = pl->plan.npass;
    for (int i = 0; i < pl->plan.npass; ++i) info->radices[i] = pl->plan.radix[i];
    info->workspace_bytes = pl->ws_bytes;
    info->wire_conv_variant = pl->wconv_variant;
    info->row_fft_fixed_shape = ws::row_fft_fixed_shape(pl->plan) ? 1 : 0;
    info->batch_units_per_wave = pl->batch_upw;
    info->batch_wire_conv_variant = pl->batch_wconv;
    return WS_OK;
}

ws_status ws_patch_capacity(ws_plane* pl, const ws_depos* depos, const ws_params* params, void* stream,
                            int64_t* bins_out) {
    if (!pl || !bins_out) return WS_ERR_INVALID_ARG;
    ws_status st = check_depos(depos);
    if (st == WS_OK) st = check_params(params);
    if (st == WS_OK) st = check_depo_span(depos, params);
    if (st != WS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ws::RasterArgs a = raster_args(pl, depos, params);
    WS_CUDA(cudaMemsetAsync(pl->counter, 0, sizeof(unsigned long long), s));
    if (depos->n > 0) WS_CUDA(ws::launch_patch_sizes(a, nullptr, pl->counter, s));
    unsigned long long total = 0;
    WS_CUDA(cudaMemcpyAsync(&total, pl->counter, sizeof total, cudaMemcpyDeviceToHost, s));
    WS_CUDA(cudaStreamSynchronize(s));
    *bins_out = (int64_t)total;
    return WS_OK;
}

ws_status ws_rasterize(ws_plane* pl, const ws_depos* depos, const ws_params* params, ws_patches* out,
                       void* stream) {
    if (!pl || !out) return WS_ERR_INVALID_ARG;
    ws_status st = check_depos(depos);
    if (st == WS_OK) st = check_params(params);
    if (st == WS_OK) st = check_depo_span(depos, params);
    if (st != WS_OK) return st;
    if (out->n != depos->n || out->capacity_bins < 0 || !out->off) return WS_ERR_INVALID_ARG;
    if (depos->n > 0 && (!out->w0 || !out->t0 || !out->nw || !out->nt)) return WS_ERR_INVALID_ARG;
    if (out->capacity_bins > 0 && !out->val) return WS_ERR_INVALID_ARG;
    if (!patches_aligned(out)) return WS_ERR_INVALID_ARG;
    if ((depos->n + 1 + 4095) / 4096 > ws::kScanScratch) return WS_ERR_UNSUPPORTED_SIZE;
    cudaStream_t s = (cudaStream_t)stream;
    ws::RasterArgs a = raster_args(pl, depos, params);
    WS_LAUNCH(pl, K_SIZES, s, ws::launch_patch_sizes(a, out->off, nullptr, s));
    WS_LAUNCH(pl, K_SCAN, s, ws::launch_scan_inplace(out->off, depos->n + 1, pl->scan, s));
    WS_LAUNCH(pl, K_RPATCH, s, ws::launch_raster_patches(a, *out, pl->large, s));
    return WS_OK;
}

ws_status ws_scatter(ws_plane* pl, const ws_patches* patches, float* grid_dev, void* stream) {
    if (!pl || !patches || !grid_dev || patches->n < 0) return WS_ERR_INVALID_ARG;
    if (patches->n > 0 && (!patches->off || !patches->w0 || !patches->t0 || !patches->nw || !patches->nt))
        return WS_ERR_INVALID_ARG;
    if (!aligned(grid_dev, 4) || !patches_aligned(patches)) return WS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    WS_LAUNCH(pl, K_SCATTER, s, ws::launch_scatter_patches(*patches, grid_dev, pl->desc.nwires * pl->impacts,
                                                          pl->desc.nticks, s));
    return WS_OK;
}

ws_status ws_convolve(ws_plane* pl, const float* grid_dev, float* out_dev, void* stream) {
    NvtxRange range("ws_convolve");
    if (!pl || !grid_dev || !out_dev) return WS_ERR_INVALID_ARG;
    if (!aligned(grid_dev, 4) || !aligned(out_dev, 4)) return WS_ERR_INVALID_ARG;
    if (pl->impacts > 1) {   // fine input and coarse output must not overlap
        const char* g0 = (const char*)grid_dev;
        const char* g1 = g0 + sizeof(float) * (size_t)pl->impacts * pl->desc.nwires * pl->desc.nticks;
        const char* o0 = (const char*)out_dev;
        const char* o1 = o0 + sizeof(float) * (size_t)pl->desc.nwires * pl->desc.nticks;
        if (o0 < g1 && g0 < o1) return WS_ERR_INVALID_ARG;
    }
    return convolve_impl(pl, grid_dev, out_dev, (cudaStream_t)stream);
}

ws_status ws_simulate(ws_plane* pl, const ws_depos* depos, const ws_params* params, float* out_dev,
                      void* stream) {
    NvtxRange range("ws_simulate");
    if (!pl || !out_dev || !aligned(out_dev, 4)) return WS_ERR_INVALID_ARG;
    ws_status st = check_depos(depos);
    if (st == WS_OK) st = check_params(params);
    if (st == WS_OK) st = check_depo_span(depos, params);
    if (st != WS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const ws_plane_desc& d = pl->desc;
    const size_t grid_bytes = sizeof(float) * (size_t)d.nwires * d.nticks;
    ws::RasterArgs a = raster_args(pl, depos, params);
    if (pl->impacts > 1 && params->precision == WS_PREC_FP64) {
        // FP64 on the fine grid: double grid, transforms and impact sum
        if (!pl->fp64) return WS_ERR_WORKSPACE;
        const int I = pl->impacts;
        WS_LAUNCH(pl, K_MEMSET, s, cudaMemsetAsync(pl->g64, 0, 2 * grid_bytes * I, s));
        a.grid64 = pl->g64;
        WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, out_dev, pl->large, s));
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows64(pl->plan, pl->tw64, pl->g64, true, d.nwires * I, d.nticks,
                                                      d.nticks, pl->X64, pl->fstride, pl->nfreq, 1.0f, s));
        WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv_impacts64(pl->X64, pl->Y64, pl->Rt64, d.nwires, I, pl->nfreq,
                                                                 pl->fstride, d.resp_nwires, d.resp_wire_center,
                                                                 d.conv_mode == WS_CONV_CIRCULAR, s));
        st = add_plane_noise(pl, params, pl->Y64, true, s);
        if (st != WS_OK) return st;
        WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows64(pl->plan, pl->tw64, pl->Y64, d.nwires, pl->fstride, pl->nfreq,
                                                      out_dev, d.nticks, d.nticks, s));
        return WS_OK;
    }
    if (pl->impacts > 1) {
        // compensated: the fine grid's low parts in grid2 (fine-sized on impact planes)
        if (params->precision == WS_PREC_FP32_COMP) a.lo = pl->grid2;
        if (marks_apply(pl)) return simulate_marked(pl, a, out_dev, s);
        WS_LAUNCH(pl, K_MEMSET, s, cudaMemsetAsync(pl->fine, 0, grid_bytes * pl->impacts, s));
        if (a.lo) WS_CUDA(cudaMemsetAsync(pl->grid2, 0, grid_bytes * pl->impacts, s));
        WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, pl->fine, pl->large, s));
        return convolve_impl(pl, pl->fine, out_dev, s, params, a.lo);
    }
    if (params->precision == WS_PREC_FP64) {
        if (!pl->fp64) return WS_ERR_WORKSPACE;
        // FP64 throughout: double grid, double transforms, float output.
        WS_LAUNCH(pl, K_MEMSET, s, cudaMemsetAsync(pl->g64, 0, 2 * grid_bytes, s));
        a.grid64 = pl->g64;
        WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, out_dev, pl->large, s));
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows64(pl->plan, pl->tw64, pl->g64, true, d.nwires, d.nticks, d.nticks,
                                                      pl->X64, pl->fstride, pl->nfreq, 1.0f, s));
        WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv64(pl->X64, pl->Y64, pl->Rt64, d.nwires, pl->nfreq, pl->fstride,
                                                         d.resp_nwires, d.resp_wire_center,
                                                         d.conv_mode == WS_CONV_CIRCULAR, s));
        st = add_plane_noise(pl, params, pl->Y64, true, s);
        if (st != WS_OK) return st;
        WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows64(pl->plan, pl->tw64, pl->Y64, d.nwires, pl->fstride, pl->nfreq,
                                                      out_dev, d.nticks, d.nticks, s));
        return WS_OK;
    }
    if (marks_apply(pl)) {
        if (params->precision == WS_PREC_FP32_COMP) a.lo = pl->grid2;
        return simulate_marked(pl, a, out_dev, s);
    }
    WS_LAUNCH(pl, K_MEMSET, s, cudaMemsetAsync(out_dev, 0, grid_bytes, s));
    if (params->precision == WS_PREC_FP32_COMP) {
        // Compensated scatter: the grid's low parts go to grid2 and are added
        // back by the forward transform.
        WS_CUDA(cudaMemsetAsync(pl->grid2, 0, grid_bytes, s));
        a.lo = pl->grid2;
        WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, out_dev, pl->large, s));
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows_comp(pl->plan, pl->tw, out_dev, pl->grid2, d.nwires, d.nticks,
                                                         d.nticks, pl->X, pl->fstride, pl->nfreq, s));
        WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv(pl->X, pl->Y, pl->Rt, d.nwires, pl->nfreq, pl->fstride,
                                                       d.resp_nwires, d.resp_wire_center,
                                                       d.conv_mode == WS_CONV_CIRCULAR, s, pl->wconv_variant, pl->status));
        st = add_plane_noise(pl, params, pl->Y, false, s);
        if (st != WS_OK) return st;
        WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows(pl->plan, pl->tw, pl->Y, d.nwires, pl->fstride, pl->nfreq, out_dev,
                                                    d.nticks, d.nticks, s, pl->status));
        return WS_OK;
    }
    WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, out_dev, pl->large, s));
    return convolve_impl(pl, out_dev, out_dev, s, params);
}

ws_status ws_plane_set_noise(ws_plane* pl, const float* amp_dev, const float* coh_amp_dev, int32_t coh_group,
                             void* stream) {
    if (!pl) return WS_ERR_INVALID_ARG;
    if (!amp_dev && !coh_amp_dev) {
        pl->noise_mode = 0;
        return WS_OK;
    }
    if (!amp_dev || !aligned(amp_dev, 4) || (coh_amp_dev && (!aligned(coh_amp_dev, 4) || coh_group < 1)))
        return WS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * (size_t)pl->nfreq;
    WS_CUDA(cudaMemcpyAsync(pl->noise_amp, amp_dev, bytes, cudaMemcpyDeviceToDevice, s));
    if (coh_amp_dev)
        WS_CUDA(cudaMemcpyAsync(pl->noise_amp + pl->fstride, coh_amp_dev, bytes, cudaMemcpyDeviceToDevice, s));
    pl->noise_mode = coh_amp_dev ? 2 : 1;
    pl->noise_group = coh_amp_dev ? coh_group : 1;
    return WS_OK;
}

ws_status ws_plane_set_response(ws_plane* pl, const float* response_dev, void* stream) {
    if (!pl || !response_dev || !aligned(response_dev, 4)) return WS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const ws_plane_desc& d = pl->desc;
    WS_CUDA(ws::launch_fwd_rows(pl->plan, pl->tw, response_dev, pl->impacts * d.resp_nwires, d.resp_nticks,
                                d.resp_nticks, pl->Rt, pl->fstride, pl->nfreq, 1.0f / (float)pl->plan.L, s));
    for (int i = 0; i < pl->impacts; ++i)
        WS_CUDA(ws::launch_adj_coeffs(pl->Rt + (size_t)i * d.resp_nwires * pl->fstride,
                                      pl->Radj + (size_t)i * d.resp_nwires * pl->fstride, d.resp_nwires,
                                      pl->fstride, pl->nfreq, s));
    if (pl->fp64)
        WS_CUDA(ws::launch_fwd_rows64(pl->plan, pl->tw64, response_dev, false, pl->impacts * d.resp_nwires,
                                      d.resp_nticks,
                                      d.resp_nticks, pl->Rt64, pl->fstride, pl->nfreq, 1.0f / (float)pl->plan.L, s));
    return WS_OK;
}

ws_status ws_simulate_backward(ws_plane* pl, const ws_depos* depos, const ws_params* params,
                               const float* grad_out_dev, float* gq, float* gx, float* gt, double* gDL,
                               double* gDT, float* gR, void* stream) {
    NvtxRange range("ws_simulate_backward");
    if (!pl || !grad_out_dev || !aligned(grad_out_dev, 4)) return WS_ERR_INVALID_ARG;
    ws_status st = check_depos(depos);
    if (st == WS_OK) st = check_params(params);
    if (st == WS_OK) st = check_depo_span(depos, params);
    if (st != WS_OK) return st;
    if (params->fluctuate) return WS_ERR_INVALID_ARG;  // the adjoint is of the expected-value path
    if (!aligned(gq, 4) || !aligned(gx, 4) || !aligned(gt, 4) || !aligned(gR, 4) || !aligned(gDL, 8) ||
        !aligned(gDT, 8))
        return WS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const ws_plane_desc& d = pl->desc;
    const int circ = d.conv_mode == WS_CONV_CIRCULAR;
    if (pl->impacts > 1) return backward_impacts(pl, depos, params, grad_out_dev, gq, gx, gt, gDL, gDT, gR, s);
    // dL/dS = adjoint convolution of G: tick transform, wire correlation with
    // conj(R_hat), inverse transform.
    WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows(pl->plan, pl->tw, grad_out_dev, d.nwires, d.nticks, d.nticks, pl->X,
                                                pl->fstride, pl->nfreq, 1.0f, s));
    WS_LAUNCH(pl, K_WCONV, s, ws::launch_wire_conv(pl->X, pl->Y, pl->Radj, d.nwires, pl->nfreq, pl->fstride,
                                                   d.resp_nwires, d.resp_nwires - 1 - d.resp_wire_center, circ, s,
                                                   pl->wconv_variant, pl->status));
    WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows(pl->plan, pl->tw, pl->Y, d.nwires, pl->fstride, pl->nfreq,
                                                pl->grid2, d.nticks, d.nticks, s));
    ws::RasterArgs a = raster_args(pl, depos, params);
    if (gDL) WS_CUDA(cudaMemsetAsync(gDL, 0, sizeof(double), s));
    if (gDT) WS_CUDA(cudaMemsetAsync(gDT, 0, sizeof(double), s));
    WS_LAUNCH(pl, K_DGRAD, s, ws::launch_depo_grads(a, pl->grid2, gq, gx, gt, gDL, gDT, params->DL_mm2_us,
                                                    params->DT_mm2_us, pl->large, s));
    if (gR) {
        // dL/dR: recompute S, transform it, correlate with the transform of G
        // (still in X) over wires, inverse transform, keep the response window.
        const size_t grid_bytes = sizeof(float) * (size_t)d.nwires * d.nticks;
        WS_LAUNCH(pl, K_MEMSET, s, cudaMemsetAsync(pl->grid2, 0, grid_bytes, s));
        WS_LAUNCH(pl, K_RASTER_SCATTER, s, ws::launch_raster_scatter(a, pl->grid2, pl->large, s));
        WS_LAUNCH(pl, K_FWD, s, ws::launch_fwd_rows(pl->plan, pl->tw, pl->grid2, d.nwires, d.nticks, d.nticks,
                                                    pl->Y, pl->fstride, pl->nfreq, 1.0f, s));
        WS_CUDA(cudaMemsetAsync(pl->Racc, 0, sizeof(float2) * (size_t)d.resp_nwires * pl->fstride, s));
        WS_LAUNCH(pl, K_RGRAD, s, ws::launch_resp_grad(pl->X, pl->Y, pl->Racc, d.nwires, pl->nfreq, pl->fstride,
                                                       d.resp_nwires, d.resp_wire_center, circ,
                                                       1.0f / (float)pl->plan.L, s));
        WS_LAUNCH(pl, K_INV, s, ws::launch_inv_rows(pl->plan, pl->tw, pl->Racc, d.resp_nwires, pl->fstride,
                                                    pl->nfreq, gR, d.resp_nticks, d.resp_nticks, s));
    }
    return WS_OK;
}

}  // extern "C"

namespace {

// Wave slots, each with its own counters, large-patch list and spectra, so
// that consecutive waves run on kBatchSlots streams (wave k in slot k % S).
constexpr int kBatchSlots = 3;

// A unit's spectra: X (I x nwires rows for impact planes) then Y (nwires
// rows); impact planes also keep a unit's fine grid (I x nwires rows of
// ticks) in the slot.
struct BatchLayout {
    size_t off_counters, off_list, off_spec, xspec_bytes, spec_bytes, off_rows, rows_bytes, off_cls, cls_bytes,
        off_fine, fine_bytes, slot_bytes, total;
};
// Within a slot's 256-byte counter block (cleared at the start of every call):
// the large-patch list's count and done words, the active-row epochs (base
// at byte 8, epoch at byte 16) and the impact wire convolution's claim words
// (byte 24; its launches on a slot run one after another).  The slot's marks are cleared at the
// start of every call too, so the waves of a call that share a slot mark
// with epochs 1, 2, ... above every mark there.
constexpr size_t kBatchClearBytes = 64;
constexpr size_t kBatchRowsBase = 8;
constexpr size_t kBatchRowsEpoch = 16;
constexpr size_t kBatchSched = 24;   // the impact wire convolution's two claim words

ws_status batch_layout(ws_plane* const* planes, int nplanes, int units_per_wave, BatchLayout* lay) {
    if (units_per_wave == 0) units_per_wave = ws::kMaxUnits;
    if (!planes || nplanes <= 0 || units_per_wave < 0 || units_per_wave > ws::kMaxUnits) return WS_ERR_INVALID_ARG;
    int maxw = 0;
    const ws_plane* p0 = planes[0];
    if (!p0) return WS_ERR_INVALID_ARG;
    for (int i = 0; i < nplanes; ++i) {
        const ws_plane* p = planes[i];
        if (!p) return WS_ERR_INVALID_ARG;
        // one launch per stage needs one transform plan, one response shape
        // and one pitch binning (impact positions)
        if (p->impacts != p0->impacts || p->plan.L != p0->plan.L || p->plan.npass != p0->plan.npass || p->fstride != p0->fstride ||
            p->desc.nticks != p0->desc.nticks || p->desc.resp_nwires != p0->desc.resp_nwires ||
            p->desc.resp_wire_center != p0->desc.resp_wire_center || p->desc.conv_mode != p0->desc.conv_mode)
            return WS_ERR_UNSUPPORTED_SIZE;
        for (int j = 0; j < p->plan.npass; ++j)
            if (p->plan.radix[j] != p0->plan.radix[j]) return WS_ERR_UNSUPPORTED_SIZE;
        if (p->desc.nwires > maxw) maxw = p->desc.nwires;
    }
    size_t o = 0;
    lay->off_counters = o; o = align256(o + 256);
    lay->off_list = o; o = align256(o + sizeof(long long) * (size_t)ws::kLargeListCap);
    const int I = p0->impacts;
    lay->xspec_bytes = align256(sizeof(float2) * (size_t)I * maxw * p0->fstride);
    lay->spec_bytes = align256(sizeof(float2) * (size_t)maxw * p0->fstride);
    lay->off_spec = o; o += (size_t)units_per_wave * (lay->xspec_bytes + lay->spec_bytes);
    lay->rows_bytes = align256(sizeof(ws::mark_t) * (size_t)maxw);
    lay->off_rows = o; o += (size_t)units_per_wave * lay->rows_bytes;
    lay->cls_bytes = align256(sizeof(uint32_t) * (size_t)maxw);
    lay->off_cls = o; o += (size_t)units_per_wave * lay->cls_bytes;
    lay->fine_bytes = I > 1 ? align256(sizeof(float) * (size_t)I * maxw * p0->desc.nticks) : 0;
    lay->off_fine = o; o += (size_t)units_per_wave * lay->fine_bytes;
    lay->slot_bytes = o;
    lay->total = kBatchSlots * o;
    return WS_OK;
}

// The library's k-th extra stream (k < kBatchSlots - 1) for this thread and
// device (created once, kept for the life of the process).
cudaError_t aux_stream(int k, cudaStream_t* out) {
    thread_local cudaStream_t streams[64][kBatchSlots - 1] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || k < 0 || k >= kBatchSlots - 1) return cudaErrorInvalidDevice;
    if (!streams[dev][k]) {
        e = cudaStreamCreateWithFlags(&streams[dev][k], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *out = streams[dev][k];
    return cudaSuccess;
}

ws_status batch_waves(ws_plane* const* planes, int nplanes, const ws_depos* depos, const ws_params* params,
                      float* const* out_dev, char* ws_base, const BatchLayout& lay, int units_per_wave, int nunits,
                      const cudaStream_t* ss, int nstreams);

// Whether a wave of `upw` units fits `bytes` of batch workspace.
bool wave_fits(ws_plane* const* planes, int nplanes, int upw, size_t bytes) {
    BatchLayout lay;
    return batch_layout(planes, nplanes, upw, &lay) == WS_OK && lay.total <= bytes;
}

// Wave size of a call with units_per_wave == 0: the autotuner's choice
// recorded on the first plane if it fits the workspace, else the largest
// wave (at most kMaxUnits, at most the call's units) that fits; 1 if none
// does (the call then fails its workspace check).
int auto_wave_size(ws_plane* const* planes, int nplanes, int nunits, size_t bytes) {
    const int tuned = planes[0]->batch_upw;
    if (tuned > 0 && wave_fits(planes, nplanes, tuned, bytes)) return tuned;
    int upw = nunits < ws::kMaxUnits ? nunits : ws::kMaxUnits;
    while (upw > 1 && !wave_fits(planes, nplanes, upw, bytes)) --upw;
    return upw;
}

}  // namespace

extern "C" {

ws_status ws_batch_workspace_bytes(ws_plane* const* planes, int nplanes, int units_per_wave, size_t* bytes) {
    if (!bytes) return WS_ERR_INVALID_ARG;
    BatchLayout lay;
    ws_status st = batch_layout(planes, nplanes, units_per_wave, &lay);
    if (st != WS_OK) return st;
    *bytes = lay.total;
    return WS_OK;
}

ws_status ws_simulate_batch(ws_plane* const* planes, int nplanes, const ws_depos* depos, int nevents,
                            const ws_params* params, float* const* out_dev, void* workspace_dev,
                            size_t workspace_bytes, int units_per_wave, void* stream) {
    NvtxRange range("ws_simulate_batch");
    if (units_per_wave == 0 && planes && nplanes > 0 && planes[0])
        units_per_wave = nevents > 0 ? auto_wave_size(planes, nplanes, nevents * nplanes, workspace_bytes) : 1;
    BatchLayout lay;
    ws_status st = batch_layout(planes, nplanes, units_per_wave, &lay);
    if (st != WS_OK) return st;
    if (!depos || !out_dev || nevents < 0) return WS_ERR_INVALID_ARG;
    st = check_params(params);
    if (st != WS_OK) return st;
    if (params->precision != WS_PREC_FP32) return WS_ERR_UNSUPPORTED_SIZE;
    if (!workspace_dev || !aligned(workspace_dev, 256) || workspace_bytes < lay.total) return WS_ERR_WORKSPACE;
    if (params->event_id + (uint64_t)nevents > (1u << 28)) return WS_ERR_INVALID_ARG;
    const int nunits = nevents * nplanes;
    for (int u = 0; u < nunits; ++u) {
        st = check_depos(&depos[u]);
        if (st == WS_OK) st = check_depo_span(&depos[u], params);
        if (st != WS_OK) return st;
        if (!out_dev[u] || !aligned(out_dev[u], 4)) return WS_ERR_INVALID_ARG;
    }
    if (nunits == 0) return WS_OK;
    // Waves go round the caller's stream and the library's extra streams
    // (wave k in slot k % S, S = min(waves, kBatchSlots)): one wave's raster
    // runs beside the others' transforms.  Fork and join go through events,
    // so the call stays stream-ordered for the caller and can be captured
    // into a graph.
    const int nwaves = (nunits + units_per_wave - 1) / units_per_wave;
    const int nstreams = nwaves < kBatchSlots ? nwaves : kBatchSlots;
    cudaStream_t ss[kBatchSlots];
    for (int k = 0; k < kBatchSlots; ++k) ss[k] = (cudaStream_t)stream;
    cudaEvent_t fork = nullptr, join[kBatchSlots] = {};
    auto release = [&]() {
        if (fork) cudaEventDestroy(fork);
        for (int k = 0; k < kBatchSlots; ++k)
            if (join[k]) cudaEventDestroy(join[k]);
    };
    if (nstreams > 1) {
        cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, ss[0]);
        for (int k = 1; k < nstreams && e == cudaSuccess; ++k) {
            e = aux_stream(k - 1, &ss[k]);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ss[k], fork, 0);
        }
        if (e != cudaSuccess) {
            release();
            return cuda_fail(e, "batch fork");
        }
    }
    ws_status wst = batch_waves(planes, nplanes, depos, params, out_dev, (char*)workspace_dev, lay, units_per_wave,
                                nunits, ss, nstreams);
    cudaError_t e = cudaSuccess;
    for (int k = 1; k < nstreams; ++k) {
        if (e == cudaSuccess) e = cudaEventRecord(join[k], ss[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ss[0], join[k], 0);
    }
    release();
    if (e != cudaSuccess && wst == WS_OK) return cuda_fail(e, "batch join");
    return wst;
}

ws_status ws_batch_autotune(ws_plane* const* planes, int nplanes, const ws_depos* depos, int nevents,
                            const ws_params* params, float* const* out_dev, void* workspace_dev,
                            size_t workspace_bytes, void* stream, int* units_per_wave_out) {
    NvtxRange range("ws_batch_autotune");
    if (!units_per_wave_out || !planes || nplanes <= 0 || nevents <= 0) return WS_ERR_INVALID_ARG;
    for (int i = 0; i < nplanes; ++i)
        if (!planes[i]) return WS_ERR_INVALID_ARG;
    const int nunits = nevents * nplanes;
    const int most = nunits < ws::kMaxUnits ? nunits : ws::kMaxUnits;
    // Candidates: every size up to 4 units; whole events (nplanes x 1, 2, 4,
    // ...); the largest wave; all of them limited to what the workspace holds.
    int cand[2 * ws::kMaxUnits];
    int nc = 0;
    auto add = [&](int u) {
        if (u < 1 || u > most || !wave_fits(planes, nplanes, u, workspace_bytes)) return;
        for (int i = 0; i < nc; ++i)
            if (cand[i] == u) return;
        cand[nc++] = u;
    };
    for (int u = 1; u <= 4; ++u) add(u);
    for (int k = 1; k * nplanes <= most; k *= 2) add(k * nplanes);
    add(most - most % nplanes);
    add(most);
    if (nc == 0) return WS_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return cuda_fail(e, "ws_batch_autotune");
    }
    // Every candidate once to warm up, then three rounds over all candidates
    // (interleaved, so a drifting clock biases none); a candidate's time is
    // its best round, the fastest candidate is kept.
    float best_of[2 * ws::kMaxUnits];
    ws_status st = WS_OK;
    for (int i = 0; i < nc && st == WS_OK; ++i) {
        best_of[i] = 1e30f;
        st = ws_simulate_batch(planes, nplanes, depos, nevents, params, out_dev, workspace_dev, workspace_bytes,
                               cand[i], stream);
    }
    for (int round = 0; round < 3 && st == WS_OK; ++round) {
        for (int i = 0; i < nc && st == WS_OK; ++i) {
            e = cudaEventRecord(t0, s);
            if (e == cudaSuccess)
                st = ws_simulate_batch(planes, nplanes, depos, nevents, params, out_dev, workspace_dev,
                                       workspace_bytes, cand[i], stream);
            if (e == cudaSuccess && st == WS_OK) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess && st == WS_OK) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess && st == WS_OK) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess && st == WS_OK) st = cuda_fail(e, "ws_batch_autotune");
            if (st == WS_OK && ms < best_of[i]) best_of[i] = ms;
        }
    }
    int best = 0;
    if (st == WS_OK) {
        for (int i = 1; i < nc; ++i)
            if (best_of[i] < best_of[best]) best = i;
        for (int i = 0; i < nplanes; ++i) planes[i]->batch_upw = cand[best];
    }
    // Then the wire-convolution kernel at that wave size (one kernel serves
    // every unit of a launch): each variant the planes allow, timed the same
    // way; the planes keep their own choice for single-plane calls.
    const int circ = planes[0]->desc.conv_mode == WS_CONV_CIRCULAR;
    // a kernel already chosen for batches on these planes (by an earlier
    // run of the autotuner or ws_plane_set_wire_conv_variant) is kept
    const int nvar = planes[0]->batch_wconv >= 0             ? 0
                     : planes[0]->impacts > 1                  ? ((circ || !ws::tma_available()) ? 0 : ws::kImpactConvVariants)
                     : (circ || !ws::tma_available())          ? 4
                                                               : ws::kWireConvVariants;
    float var_ms[ws::kWireConvVariants];
    for (int v = 0; v < nvar; ++v) var_ms[v] = 1e30f;
    const int keep = planes[0]->batch_wconv;
    for (int round = 0; round < 3 && st == WS_OK; ++round) {
        for (int v = 0; v < nvar && st == WS_OK; ++v) {
            planes[0]->batch_wconv = v;
            if (round == 0)
                st = ws_simulate_batch(planes, nplanes, depos, nevents, params, out_dev, workspace_dev,
                                       workspace_bytes, cand[best], stream);
            if (st == WS_OK) e = cudaEventRecord(t0, s);
            if (st == WS_OK && e == cudaSuccess)
                st = ws_simulate_batch(planes, nplanes, depos, nevents, params, out_dev, workspace_dev,
                                       workspace_bytes, cand[best], stream);
            if (e == cudaSuccess && st == WS_OK) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess && st == WS_OK) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess && st == WS_OK) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess && st == WS_OK) st = cuda_fail(e, "ws_batch_autotune");
            if (st == WS_OK && ms < var_ms[v]) var_ms[v] = ms;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != WS_OK) {
        planes[0]->batch_wconv = keep;
        return st;
    }
    if (nvar > 0) {
        int bv = 0;
        for (int v = 1; v < nvar; ++v)
            if (var_ms[v] < var_ms[bv]) bv = v;
        planes[0]->batch_wconv = bv;
    }
    *units_per_wave_out = cand[best];
    return WS_OK;
}

}  // extern "C"

namespace {

ws_status batch_waves(ws_plane* const* planes, int nplanes, const ws_depos* depos, const ws_params* params,
                      float* const* out_dev, char* ws_base, const BatchLayout& lay, int units_per_wave, int nunits,
                      const cudaStream_t* ss, int nstreams) {
    ws_plane* p0 = planes[0];
    const ws_plane_desc& d0 = p0->desc;
    const int circ = d0.conv_mode == WS_CONV_CIRCULAR;
    // the wire-convolution kernel the batch autotuner picked for these
    // planes, else the first plane's own
    const int wconv = p0->batch_wconv >= 0 ? p0->batch_wconv : p0->wconv_variant;
    // active rows for every unit whose plane allows them (see marks_apply;
    // the transform plan, convolution mode and impact positions are shared
    // by the batch)
    const int I = p0->impacts;
    const bool marked = d0.conv_mode == WS_CONV_LINEAR && ws::row_fft_fixed_shape(p0->plan) &&
                        (I == 1 || ws::tma_available());
    for (int slot = 0; slot < nstreams; ++slot) {
        char* sb = ws_base + slot * lay.slot_bytes;
        WS_CUDA(cudaMemsetAsync(sb + lay.off_counters, 0, kBatchClearBytes, ss[slot]));
        if (marked) WS_CUDA(cudaMemsetAsync(sb + lay.off_rows, 0, (size_t)units_per_wave * lay.rows_bytes, ss[slot]));
    }
    for (int u0 = 0, wave = 0; u0 < nunits; u0 += units_per_wave, ++wave) {
        const int nu = nunits - u0 < units_per_wave ? nunits - u0 : units_per_wave;
        const int slot = wave % nstreams;
        cudaStream_t s = ss[slot];
        char* base = ws_base + slot * lay.slot_bytes;
        ws::LargeList L;
        L.list = (long long*)(base + lay.off_list);
        L.count = (unsigned*)(base + lay.off_counters);
        L.done = (unsigned*)(base + lay.off_counters + 4);
        L.cap = ws::kLargeListCap;
        ws::RasterBatch rb;
        ws::RowBatch fb, ib;
        ws::ConvBatch cb;
        int64_t counts[ws::kMaxUnits];
        ws::NoiseBatch nb;
        bool noisy = false;
        rb.n = fb.n = ib.n = cb.n = nb.n = nu;
        fb.status = ib.status = p0->status;
        rb.prec = WS_PREC_FP32;
        nb.key0 = (uint32_t)(params->seed & 0xFFFFFFFFu);
        nb.key1 = (uint32_t)(params->seed >> 32);
        ws::RowMarks m;
        m.epoch = (ws::mark_t*)(base + lay.off_counters + kBatchRowsEpoch);
        m.base = (ws::mark_t*)(base + lay.off_counters + kBatchRowsBase);
        for (int j = 0; j < nu; ++j) {
            const int u = u0 + j, e = u / nplanes, pi = u % nplanes;
            ws_plane* pl = planes[pi];
            ws_params pe = *params;
            pe.event_id = params->event_id + (uint32_t)e;
            float2* X = (float2*)(base + lay.off_spec + (size_t)j * (lay.xspec_bytes + lay.spec_bytes));
            float2* Y = (float2*)((char*)X + lay.xspec_bytes);
            // the grid: the output itself, or the unit's fine grid
            float* G = I > 1 ? (float*)(base + lay.off_fine + (size_t)j * lay.fine_bytes) : out_dev[u];
            m.rows[j] = (marked && marks_apply(pl)) ? (ws::mark_t*)(base + lay.off_rows + (size_t)j * lay.rows_bytes)
                                                    : nullptr;
            m.cls[j] = m.rows[j] ? (uint32_t*)(base + lay.off_cls + (size_t)j * lay.cls_bytes) : nullptr;
            m.impacts[j] = I;
            fb.rows[j] = ib.rows[j] = m.cls[j];
            fb.rdiv[j] = I;
            cb.rows[j] = m.rows[j];
            rb.a[j] = raster_args(pl, &depos[u], &pe);
            rb.grid[j] = G;
            counts[j] = (int64_t)I * pl->desc.nwires * pl->desc.nticks;
            fb.in[j] = G;
            fb.in2[j] = nullptr;
            fb.out[j] = X;
            fb.nrows[j] = I * pl->desc.nwires;
            cb.X[j] = X;
            cb.Y[j] = Y;
            cb.Rt[j] = pl->Rt;
            cb.nwires[j] = pl->desc.nwires;
            ib.in[j] = Y;
            ib.in2[j] = nullptr;
            ib.out[j] = out_dev[u];
            ib.nrows[j] = pl->desc.nwires;
            nb.Y[j] = Y;
            nb.nwires[j] = pl->desc.nwires;
            if (noise_unit(pl, pe.event_id, &nb.noise[j])) noisy = true;
            else nb.noise[j] = ws::NoiseUnit{};
        }
        if (marked) {
            cb.epoch = m.epoch;
            m.kw = d0.resp_nwires;
            m.center = d0.resp_wire_center;
            WS_LAUNCH(p0, K_MARK, s, ws::launch_mark_rows(rb, m, s));
            WS_LAUNCH(p0, K_MEMSET, s, ws::launch_zero_marked_rows(rb, m, s));
        } else {
            WS_LAUNCH(p0, K_MEMSET, s, ws::launch_zero_grids(rb, counts, s));
        }
        WS_LAUNCH(p0, K_RASTER_SCATTER, s, ws::launch_raster_scatter_batch(rb, L, s));
        WS_LAUNCH(p0, K_FWD, s, ws::launch_fwd_rows_batch(p0->plan, p0->tw, fb, d0.nticks, d0.nticks, p0->fstride,
                                                          p0->nfreq, 1.0f, s));
        if (I > 1) {   // the wave's units in as few launches as their tensor maps allow
            cb.epoch = marked ? m.epoch : nullptr;
            const ws_status st = impacts_wconv(p0, p0, cb, (unsigned*)(base + lay.off_counters + kBatchSched), s,
                                               wconv < ws::kImpactConvVariants ? wconv : 0);
            if (st != WS_OK) return st;
        } else {
            WS_LAUNCH(p0, K_WCONV, s, ws::launch_wire_conv_batch(cb, p0->nfreq, p0->fstride, d0.resp_nwires,
                                                                 d0.resp_wire_center, circ, s, wconv, p0->status));
        }
        if (noisy) WS_LAUNCH(p0, K_NOISE, s, ws::launch_add_noise(nb, p0->nfreq, p0->plan.L, p0->fstride, s));
        WS_LAUNCH(p0, K_INV, s, ws::launch_inv_rows_batch(p0->plan, p0->tw, ib, p0->fstride, p0->nfreq, d0.nticks,
                                                          d0.nticks, s));
    }
    return WS_OK;
}

}  // namespace

extern "C" {

ws_status ws_selftest_bounded_wait(uint32_t* status_dev, int iters, unsigned long long* cycles_dev, void* stream) {
    if (!status_dev || iters < 1 || iters > (1 << 20) || !aligned(status_dev, 4)) return WS_ERR_INVALID_ARG;
    WS_CUDA(ws::launch_bounded_wait_selftest(status_dev, iters, cycles_dev, (cudaStream_t)stream));
    return WS_OK;
}

ws_status ws_plane_sync(ws_plane* pl, void* stream, uint32_t* bits) {
    if (!pl || !bits) return WS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t v = 0;
    WS_CUDA(cudaMemcpyAsync(&v, pl->status, sizeof v, cudaMemcpyDeviceToHost, s));
    WS_CUDA(cudaStreamSynchronize(s));
    *bits = v;
    if (v && log_enabled())
        fprintf(stderr, "wiresim: device status 0x%x%s%s%s\n", v, (v & WS_DEV_BAD_DEPO) ? " bad-depo" : "",
                (v & WS_DEV_PATCH_OVERFLOW) ? " patch-overflow" : "", (v & WS_DEV_TIMEOUT) ? " timeout" : "");
    return WS_OK;
}

ws_status ws_plane_clear_status(ws_plane* pl, void* stream) {
    if (!pl) return WS_ERR_INVALID_ARG;
    WS_CUDA(cudaMemsetAsync(pl->status, 0, sizeof(uint32_t), (cudaStream_t)stream));
    return WS_OK;
}

}  // extern "C"
