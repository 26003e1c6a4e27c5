// Diffusion, raster, binomial fluctuation and scatter-add (Sec. 2.2, Sec. 3.1).
//
// Parallel over depos (Sec. 2.3: parallelism at the level of individual
// ionization electron groups).  The erfc of the standardized bin edges of a
// patch go into per-warp shared-memory tables, neighbouring edges are
// differenced into 1D bin weights for each axis, and the outer product is
// emitted bin by bin, either straight into the grid with atomics (fused
// raster + scatter) or into a patch buffer.
//
// Bin weight of bin [e0, e1] clipped to mu +- n sigma: with u = (e - mu) /
// (sqrt 2 sigma) clamped to +-n/sqrt 2 and c = erfc(|u|), the mass is
//   (c0 - c1)/2 if u0 >= 0,  (c1 - c0)/2 if u1 <= 0,  1 - (c0 + c1)/2 else,
// which equals (erf(u1) - erf(u0))/2 without cancelling in the tails; it is
// divided by the window mass erf(n / sqrt 2).
//
// Precision P (template parameter, from ws_params.precision):
//   0  FP32: weights, values and grid in float;
//   1  FP32 with compensated scatter: each atomicAdd's returned old value
//      gives the exact rounding error of the addition (TwoSum), added to a
//      second float grid that the forward transform adds back; axes
//      narrower than an eighth of a bin take their edge differences in FP64;
//   2  FP64: widths, bin ranges, weights, values, binomial tail and the grid
//      in double.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.cuh"

namespace ws {
namespace {

constexpr int kChunk = 64;        // bins per axis held in the per-warp tables
constexpr int kWarpsPerBlock = 8;

template <int P> struct PrecT { using W = float; };
template <> struct PrecT<2> { using W = double; };

__device__ __forceinline__ float erfc_t(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_t(double x) { return erfc(x); }

// Exact branch: sequential-search inversion of the Binomial(N, s) CDF,
// s = min(p, 1 - p), in single precision with every operation rounded in a
// fixed order (f_0 = (1 - s)^N by binary powering over the bits of N, low
// bit first; f_{k+1} = ((f_k r) (N - k)) / (k + 1) with r = s / (1 - s) and
// the correctly rounded reciprocal of k + 1; F_k = F_{k-1} + f_k), u the top
// 24 bits of the word over 2^24; k = the first k with u < F_k (N if none),
// mirrored to N - k for p > 1/2.  Any IEEE-754 machine doing these steps
// takes the same decisions.  recip[i] holds 1/i.
__device__ __forceinline__ int invert_binomial_s(int N, uint32_t x0, float inv_base, float inv_r, int flip,
                                                 const float* recip) {
    float f = 1.0f, base = inv_base;
    for (int n = N; n > 0; n >>= 1) {
        if (n & 1) f = __fmul_rn(f, base);
        base = __fmul_rn(base, base);
    }
    const float u = __fmul_rn(__uint2float_rn(x0 >> 8), 5.9604644775390625e-8f);
    float F = f;
    int k = 0;
    while (!(u < F) && k < N) {
        f = __fmul_rn(f, inv_r);
        f = __fmul_rn(f, __int2float_rn(N - k));
        f = __fmul_rn(f, recip[k + 1]);
        F = __fadd_rn(F, f);
        ++k;
    }
    return flip ? N - k : k;
}

__device__ __forceinline__ int invert_binomial(int N, uint32_t x0, const RasterArgs& a, const float* recip) {
    return invert_binomial_s(N, x0, a.inv_base, a.inv_r, a.inv_flip, recip);
}

// Normal approximation of Binomial(N, p) from Box-Muller uniforms u1, u2,
// with the integer part of N p taken exactly from the 64-bit product N T.
// In single precision the approximation itself is far coarser than the
// rounding, so the fast logarithm, cosine and reciprocal square root are
// used; the FP64 path uses the double-precision functions.
template <int P>
__device__ __forceinline__ int normal_from_uniforms(double du1, double du2, float fu1, float fu2, int N,
                                                    const RasterArgs& a) {
    const uint64_t nt = (uint64_t)(uint32_t)N * (uint64_t)a.T;
    const int ipart = (int)(uint32_t)(nt >> 32);
    if constexpr (P == 2) {
        const double two_m32 = 2.3283064365386962890625e-10;
        const double z = sqrt(-2.0 * log(du1)) * cospi(2.0 * du2);
        const double frac = (double)(uint32_t)nt * two_m32;
        const double pe = (double)a.T * two_m32;
        const double sd = sqrt(((double)ipart + frac) * (1.0 - pe));
        const int k = ipart + (int)floor(frac + z * sd + 0.5);
        return k < 0 ? 0 : (k > N ? N : k);
    } else {
        const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
        // z sd = sqrt(-2 ln u1 * N p (1 - p)) cos(2 pi u2), one square root
        // (reciprocal-square-root form); cos(2 pi u2) = -cos(2 pi (u2 - 1/2)),
        // argument within [-pi, pi]
        const float frac = (float)(uint32_t)nt * two_m32;
        const float pe = (float)a.T * two_m32;
        const float t = fmaxf(-2.f * __logf(fu1), 0.f) * (((float)ipart + frac) * (1.f - pe));
        const float rs = t > 0.f ? t * rsqrtf(t) : 0.f;
        const float dz = -rs * __cosf(6.28318530717958648f * (fu2 - 0.5f));
        const int k = ipart + (int)floorf(frac + dz + 0.5f);
        return k < 0 ? 0 : (k > N ? N : k);
    }
}

// The per-bin normal branch: Box-Muller on the two 16-bit halves of the
// bin's word, u1 = (x >> 16 + 1/2) / 2^16, u2 = (x & 0xFFFF + 1/2) / 2^16
// (both exact in float).
template <int P>
__device__ __forceinline__ int normal_word(uint32_t x, int N, const RasterArgs& a) {
    const float f1 = ((float)(x >> 16) + 0.5f) * (1.0f / 65536.0f);
    const float f2 = ((float)(x & 0xFFFFu) + 0.5f) * (1.0f / 65536.0f);
    return normal_from_uniforms<P>((double)f1, (double)f2, f1, f2, N, a);
}

// The depo-level normal branch of the charge-conserving fluctuation's
// survivor count: Box-Muller on words 0 and 1 of its block,
// u = (x + 1/2) / 2^32.
template <int P>
__device__ __forceinline__ int normal_pair(uint4 x, int N, const RasterArgs& a) {
    const float two_m32 = 2.3283064365386963e-10f;
    const double d32 = 2.3283064365386962890625e-10;
    return normal_from_uniforms<P>(((double)x.x + 0.5) * d32, ((double)x.y + 0.5) * d32,
                                   fmaf((float)x.x, two_m32, 0.5f * two_m32),
                                   fmaf((float)x.y, two_m32, 0.5f * two_m32), N, a);
}

// The same search on a table: row N (N = 1 .. kExactCap, at offset
// N (N - 1) / 2) holds F_0 .. F_{N-1} built by invert_binomial's operations
// for one (r, 1 - s).  F is nondecreasing, so the first k with u < F_k is
// the number of entries F_j <= u: a branch-free binary search of fixed
// length (steps 64, 32, ..., 1 cover rows of up to kExactCap = 64 entries)
// keeps the lanes of a warp together whatever their N.
__device__ void fill_cdf(float* cdf, const float* recip, const RasterArgs& a, int rows) {
    for (int N = threadIdx.x + 1; N <= rows; N += blockDim.x) {
        float f = 1.0f, base = a.inv_base;
        for (int n = N; n > 0; n >>= 1) {
            if (n & 1) f = __fmul_rn(f, base);
            base = __fmul_rn(base, base);
        }
        float* row = cdf + N * (N - 1) / 2;
        float F = f;
        row[0] = F;
        for (int k = 0; k + 1 < N; ++k) {
            f = __fmul_rn(f, a.inv_r);
            f = __fmul_rn(f, __int2float_rn(N - k));
            f = __fmul_rn(f, recip[k + 1]);
            F = __fadd_rn(F, f);
            row[k + 1] = F;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int invert_binomial_table(int N, uint32_t x0, const RasterArgs& a, const float* cdf) {
    const float u = __fmul_rn(__uint2float_rn(x0 >> 8), 5.9604644775390625e-8f);
    const float* row = cdf + N * (N - 1) / 2;
    int k = 0;
#pragma unroll
    for (int step = 64; step >= 1; step >>= 1) {
        const int j = k + step;
        if (j <= N && !(u < row[j - 1])) k = j;
    }
    return a.inv_flip ? N - k : k;
}

// Random stream of the per-bin fluctuation: one Philox block per quad (the
// four consecutive ticks 4g .. 4g+3 of one wire w of one depo), counter
// (0, w * ceil(nticks / 4) + g, depo, event << 4 | plane); bin (w, k) takes
// word k % 4.
__device__ __forceinline__ uint32_t quad_index(int w, int k, int nticks) {
    return (uint32_t)w * (uint32_t)((nticks + 3) >> 2) + (uint32_t)(k >> 2);
}

__device__ __forceinline__ uint32_t word_of(const uint4& x, int j) {
    return j == 0 ? x.x : (j == 1 ? x.y : (j == 2 ? x.z : x.w));
}

// Survivor count of a bin holding N electrons from its word x: CDF
// inversion for N <= exact_max, else the normal approximation.  cdf: the
// table for this unit's (r, 1 - s), or null for the direct search.
template <int P>
__device__ __forceinline__ int draw_word(int N, uint32_t x, const RasterArgs& a, const float* recip,
                                         const float* cdf) {
    if (N <= a.exact_max) return cdf ? invert_binomial_table(N, x, a, cdf) : invert_binomial(N, x, a, recip);
    return normal_word<P>(x, N, a);
}

// Survivor count of bin (w, k) holding N electrons (its quad's block
// computed for this bin alone).
template <int P>
__device__ __forceinline__ int binomial_bin(int N, const RasterArgs& a, int w, int k, uint32_t depo,
                                            const float* recip, const float* cdf) {
    if (N <= 0 || a.T == 0u) return 0;
    if (a.keep_all) return N;
    const uint4 x = philox4x32_10(make_uint4(0u, quad_index(w, k, a.nticks), depo, a.evpl), a.key0, a.key1);
    return draw_word<P>(N, word_of(x, k & 3), a, recip, cdf);
}

// Reciprocals 1/i, i = 0 .. kExactCap, correctly rounded, into shared memory
// (entry 0 unused).
__device__ __forceinline__ void fill_recip(float* recip) {
    for (int i = threadIdx.x; i <= kExactCap; i += blockDim.x) recip[i] = i > 0 ? __frcp_rn((float)i) : 0.f;
    __syncthreads();
}

// Electrons in a bin of expected charge v (saturating at 1e9).
__device__ __forceinline__ int electrons(float v) { return (int)floorf(fminf(v, 1.0e9f) + 0.5f); }
__device__ __forceinline__ int electrons(double v) { return (int)floor(fmin(v, 1.0e9) + 0.5); }

// Scatter-add of one bin value into the grid at the unit's precision.
__device__ __forceinline__ float two_sum_err(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int P>
__device__ __forceinline__ void emit(const RasterArgs& a, float* grid, int64_t idx, typename PrecT<P>::W v) {
    if (v == 0) return;
    if constexpr (P == 0) {
        atomicAdd(grid + idx, v);
    } else if constexpr (P == 1) {
        const float old = atomicAdd(grid + idx, v);
        const float err = two_sum_err(old, v);
        if (err != 0.f) atomicAdd(a.lo + idx, err);
    } else {
        atomicAdd(a.grid64 + idx, v);
    }
}

// Per-depo geometry: widths and the patch's bin range clipped to the grid.
template <typename W>
struct ExtentT {
    W mu_t, mu_x, st, sx;
    int k0, k1, w0, w1;   // inclusive, clipped
    bool point_t, point_x;
};
using Extent = ExtentT<float>;

template <typename W>
__device__ __forceinline__ bool axis_range(W mu, W sigma, W delta, W nsig, int nbins, int* lo, int* hi, bool* point) {
    W lo_e, hi_e;
    *point = !(sigma > (W)1e-6 * delta);
    if (*point) {
        lo_e = hi_e = mu;
    } else {
        lo_e = mu - nsig * sigma;
        hi_e = mu + nsig * sigma;
    }
    // Bins beyond the grid are clipped; clamp before converting to int.
    const W fa = fmin(fmax(floor(lo_e / delta), (W)-1), (W)nbins);
    const W fb = fmin(fmax(floor(hi_e / delta), (W)-1), (W)nbins);
    int l = (int)fa, h = (int)fb;
    if (l < 0) l = 0;
    if (h > nbins - 1) h = nbins - 1;
    *lo = l;
    *hi = h;
    return l <= h;
}

// A depo's inputs as loaded from the arrays (widths only if given).
struct DepoIn {
    float q, x, t, sig_t, sig_x;
};

__device__ __forceinline__ DepoIn load_depo(const RasterArgs& a, int64_t i) {
    DepoIn d;
    d.q = __ldg(a.q + i);
    d.x = __ldg(a.x + i);
    d.t = __ldg(a.t + i);
    d.sig_t = a.sig_t ? __ldg(a.sig_t + i) : 0.f;
    d.sig_x = a.sig_t ? __ldg(a.sig_x + i) : 0.f;
    return d;
}

// Returns false if the depo has no in-grid bins or is invalid (then *bad).
template <typename W>
__device__ __forceinline__ bool depo_extent(const RasterArgs& a, const DepoIn& in, ExtentT<W>* e, W* q, bool* bad) {
    *bad = false;
    const float qf = in.q, xf = in.x, tf = in.t;
    bool ok = isfinite(qf) && isfinite(xf) && isfinite(tf);
    const W ti = (W)tf;
    W st, sx;
    if (a.sig_t) {
        st = (W)in.sig_t;
        sx = (W)in.sig_x;
    } else {
        ok = ok && tf >= 0.f;
        const W tt = ti > (W)0 ? ti : (W)0;
        if constexpr (sizeof(W) == 8) {
            st = sqrt(a.two_DL64 * tt) / a.v64;
            sx = sqrt(a.two_DT64 * tt);
        } else {
            st = sqrtf(a.two_DL * tt) * a.inv_v;
            sx = sqrtf(a.two_DT * tt);
        }
    }
    ok = ok && isfinite(st) && isfinite(sx) && st >= (W)0 && sx >= (W)0;
    if (!ok) {
        *bad = true;
        return false;
    }
    *q = (W)qf;
    e->mu_t = ti; e->mu_x = (W)xf; e->st = st; e->sx = sx;
    const W tick = sizeof(W) == 8 ? (W)a.tick64 : (W)a.tick;
    const W pitch = sizeof(W) == 8 ? (W)a.pitch64 : (W)a.pitch;
    const W nsig = sizeof(W) == 8 ? (W)a.nsig64 : (W)a.nsig;
    if (!axis_range<W>(ti, st, tick, nsig, a.nticks, &e->k0, &e->k1, &e->point_t)) return false;
    if (!axis_range<W>((W)xf, sx, pitch, nsig, a.nwires, &e->w0, &e->w1, &e->point_x)) return false;
    return true;
}

template <typename W>
__device__ __forceinline__ bool depo_extent(const RasterArgs& a, int64_t i, ExtentT<W>* e, W* q, bool* bad) {
    return depo_extent<W>(a, load_depo(a, i), e, q, bad);
}

// Weight of a bin from its two clamped standardized edges u and erfc(|u|).
template <typename W>
__device__ __forceinline__ W bin_mass(W u0, W u1, W c0, W c1) {
    if (u0 >= (W)0) return (W)0.5 * (c0 - c1);
    if (u1 <= (W)0) return (W)0.5 * (c1 - c0);
    return (W)1 - (W)0.5 * (c0 + c1);
}

// Weights of bins [first, first + nb) of one axis into w[0..nb) (warp-wide).
template <typename W>
__device__ __forceinline__ void axis_weights(W mu, W sigma, W delta, W nsig, bool point, int first, int nb,
                                             W inv_norm, W* u_s, W* c_s, W* w, int lane) {
    if (point) {
        // A point charge lands in one bin: the range has exactly that bin.
        for (int b = lane; b < nb; b += 32) w[b] = (W)1;
        __syncwarp();
        return;
    }
    const W inv_s2 = (W)1 / ((W)1.41421356237309504880 * sigma);
    const W umax = nsig * (W)0.70710678118654752440;
    for (int j = lane; j <= nb; j += 32) {
        const W e = (W)(first + j) * delta;
        W u = (e - mu) * inv_s2;
        u = fmin(fmax(u, -umax), umax);
        u_s[j] = u;
        c_s[j] = erfc_t(fabs(u));
    }
    __syncwarp();
    for (int b = lane; b < nb; b += 32) w[b] = bin_mass(u_s[b], u_s[b + 1], c_s[b], c_s[b + 1]) * inv_norm;
    __syncwarp();
}

// Same, computed by one lane for its own depo (WC: arithmetic, WO: output).
template <typename WC, typename WO>
__device__ __forceinline__ void lane_axis_weights(WC mu, WC sigma, WC delta, WC nsig, bool point, int first, int nb,
                                                  WC inv_norm, WO* w) {
    if (point) {
        w[0] = (WO)1;
        return;
    }
    const WC inv_s2 = (WC)1 / ((WC)1.41421356237309504880 * sigma);
    const WC umax = nsig * (WC)0.70710678118654752440;
    WC u_prev = 0, c_prev = 0;
    for (int j = 0; j <= nb; ++j) {
        const WC e = (WC)(first + j) * delta;
        const WC u = fmin(fmax((e - mu) * inv_s2, -umax), umax);
        const WC c = erfc_t(fabs(u));
        if (j > 0) w[j - 1] = (WO)(bin_mass(u_prev, u, c_prev, c) * inv_norm);
        u_prev = u;
        c_prev = c;
    }
}

enum { EMIT_GRID = 0, EMIT_PATCH = 1 };

// Unit owning global item b: the last u with prefix[u] <= b.
__device__ __forceinline__ int find_unit64(const long long* prefix, int n, long long b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kSmallT = 16;  // largest patch (ticks x wires) the lane-per-depo kernel takes
constexpr int kSmallW = 8;
constexpr int kWideW = 32;   // the same for planes binned at pitch / I (impact positions)

template <int SW, typename W>
__device__ __forceinline__ bool is_large(const ExtentT<W>& e) {
    return (e.k1 - e.k0 + 1) > kSmallT || (e.w1 - e.w0 + 1) > SW;
}

template <typename W>
__device__ __forceinline__ W window_norm(const RasterArgs& a) {
    if constexpr (sizeof(W) == 8) return 1.0 / erf(a.nsig64 * 0.70710678118654752440);
    else return 1.f / erff(a.nsig * 0.707106781186547524f);
}

// Warp per depo for the large patches the lane-per-depo kernel handed over:
// the list's (unit, depo) entries if they fit in it, else every depo of
// every unit whose patch is large.  The last block to finish resets the
// list counter for the next launch.
template <int MODE, int P, int SW>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
raster_kernel(const __grid_constant__ RasterUnits U, ws_patches pt, const long long* __restrict__ list,
              unsigned* list_count, unsigned list_cap, unsigned* done, int cdf_rows) {
    using W = typename PrecT<P>::W;
    __shared__ W s_u[kWarpsPerBlock][kChunk + 1];
    __shared__ W s_c[kWarpsPerBlock][kChunk + 1];
    __shared__ W s_wt[kWarpsPerBlock][kChunk];
    __shared__ W s_wx[kWarpsPerBlock][kChunk];
    __shared__ float s_recip[kExactCap + 1];
    const unsigned nlist = *(volatile unsigned*)list_count;
    const bool use_list = nlist <= list_cap;
    // an empty list needs no work and no reset (the counters are zero)
    if (use_list && nlist == 0u) return;
    fill_recip(s_recip);
    // exact-branch CDF rows for unit 0's survival probability, as in the
    // lane-per-depo kernel (dynamic shared memory)
    extern __shared__ float s_cdf_large[];
    const RasterArgs& a0 = U.a[0];
    if (cdf_rows > 0) fill_cdf(s_cdf_large, s_recip, a0, cdf_rows);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;

    const int64_t nitems = use_list ? (int64_t)nlist : U.dprefix[U.n];
    for (int64_t it = (int64_t)blockIdx.x * kWarpsPerBlock + wib; it < nitems; it += nwarps) {
        int u;
        int64_t i;
        if (use_list) {
            const long long entry = list[it];
            u = (int)(entry >> 40);
            i = entry & ((1ll << 40) - 1);
        } else {
            u = find_unit64(U.dprefix, U.n, it);
            i = it - U.dprefix[u];
        }
        const RasterArgs& a = U.a[u];
        float* __restrict__ grid = U.grid[u];
        const float* cdf = (cdf_rows > 0 && a.exact_max <= cdf_rows && a.inv_r == a0.inv_r &&
                            a.inv_base == a0.inv_base) ? s_cdf_large : nullptr;
        ExtentT<W> e;
        W q;
        bool bad;
        const bool any = depo_extent<W>(a, i, &e, &q, &bad);
        if (!(any && is_large<SW>(e))) continue;  // not handed over
        int64_t off = 0;
        int ntf = 0;
        if (MODE == EMIT_PATCH) {
            const int nwf = e.w1 - e.w0 + 1;
            ntf = e.k1 - e.k0 + 1;
            off = pt.off[i];
            const bool fits = off + (int64_t)nwf * ntf <= pt.capacity_bins;
            if (lane == 0) {
                pt.w0[i] = e.w0;
                pt.t0[i] = e.k0;
                pt.nw[i] = fits ? nwf : 0;
                pt.nt[i] = fits ? ntf : 0;
                if (!fits) atomicOr(a.status, WS_DEV_PATCH_OVERFLOW);
            }
            if (!fits) continue;
        }
        const W inv_norm = window_norm<W>(a);
        const W tick = sizeof(W) == 8 ? (W)a.tick64 : (W)a.tick;
        const W pitch = sizeof(W) == 8 ? (W)a.pitch64 : (W)a.pitch;
        const W nsig = sizeof(W) == 8 ? (W)a.nsig64 : (W)a.nsig;
        const W scale = a.fluct ? (W)1 : (sizeof(W) == 8 ? (W)a.p64 : (W)a.p) * q;
        for (int kc = e.k0; kc <= e.k1; kc += kChunk) {
            const int ntc = min(kChunk, e.k1 - kc + 1);
            axis_weights<W>(e.mu_t, e.st, tick, nsig, e.point_t, kc, ntc, inv_norm, s_u[wib], s_c[wib], s_wt[wib],
                            lane);
            for (int wc = e.w0; wc <= e.w1; wc += kChunk) {
                const int nxc = min(kChunk, e.w1 - wc + 1);
                axis_weights<W>(e.mu_x, e.sx, pitch, nsig, e.point_x, wc, nxc, inv_norm, s_u[wib], s_c[wib],
                                s_wx[wib], lane);
                const int nbin = nxc * ntc;
                for (int idx = lane; idx < nbin; idx += 32) {
                    const int ia = idx / ntc, ib = idx - ia * ntc;
                    const int w = wc + ia, k = kc + ib;
                    W v;
                    if (!a.fluct) {
                        v = scale * s_wx[wib][ia] * s_wt[wib][ib];
                    } else {
                        const int N = electrons(q * s_wx[wib][ia] * s_wt[wib][ib]);
                        v = (W)binomial_bin<P>(N, a, w, k, a.depo0 + (uint32_t)i, s_recip, cdf);
                    }
                    if (MODE == EMIT_GRID) emit<P>(a, grid, (int64_t)w * a.nticks + k, v);
                    else pt.val[off + (int64_t)(w - e.w0) * ntf + (k - e.k0)] = (float)v;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            *list_count = 0u;
            *done = 0u;
            __threadfence();
        }
    }
}

// Lane per depo for patches of at most kSmallT x kSmallW bins: a warp takes
// 32 depos; lane l computes depo l's widths, clipped bin range and both erfc
// edge tables into shared memory; the warp then spreads the patches' bins
// (each with its own binomial draw when fluctuating) evenly over its lanes.
// Larger patches are appended to a list for the warp-per-depo kernel.
constexpr int kSmallWarpsPerBlock = 4;
constexpr int kSmallGroup = 32;   // depos per warp (a lane per depo)

// One axis of a lane's depo: FP32, or FP64 for the whole FP64 path and for
// axes narrower than an eighth of a bin in the compensated path.
template <int P, typename W>
__device__ __forceinline__ void lane_weights(const RasterArgs& a, W mu, W sigma, bool tick_axis, bool point, int first,
                                             int nb, W inv_norm, W* w) {
    const W delta = tick_axis ? (sizeof(W) == 8 ? (W)a.tick64 : (W)a.tick) : (sizeof(W) == 8 ? (W)a.pitch64 : (W)a.pitch);
    const W nsig = sizeof(W) == 8 ? (W)a.nsig64 : (W)a.nsig;
    if (P == 1 && !point && sigma < delta * (W)0.125) {
        lane_axis_weights<double, W>((double)mu, (double)sigma, tick_axis ? a.tick64 : a.pitch64, a.nsig64, point, first,
                                     nb, 1.0 / erf(a.nsig64 * 0.70710678118654752440), w);
        return;
    }
    lane_axis_weights<W, W>(mu, sigma, delta, nsig, point, first, nb, inv_norm, w);
}


template <int MODE, int P, int SW>
__global__ void __launch_bounds__(32 * kSmallWarpsPerBlock, 8)
raster_small_kernel(const __grid_constant__ RasterUnits U, ws_patches pt, long long* __restrict__ list,
                    unsigned* list_count, unsigned list_cap, int cdf_rows) {
    using W = typename PrecT<P>::W;
    constexpr int NW = kSmallWarpsPerBlock;
    constexpr int G = kSmallGroup;
    __shared__ W s_wt[NW][G][kSmallT + 1];
    __shared__ W s_wx[NW][G][SW + 1];
    __shared__ unsigned char s_start[NW][G];   // a round's item lane -> depo slot starting there
    __shared__ float s_recip[kExactCap + 1];
    // drawing bins of a round (at most four per lane): N and Philox word in,
    // survivor count out
    __shared__ int s_res[NW][128];
    __shared__ uint32_t s_en[NW][128];
    __shared__ uint32_t s_ew[NW][128];
    extern __shared__ float s_cdf[];     // exact-branch CDF rows 1 .. cdf_rows for unit 0's survival probability
    fill_recip(s_recip);
    const RasterArgs& a0 = U.a[0];
    if (cdf_rows > 0) fill_cdf(s_cdf, s_recip, a0, cdf_rows);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int dl = lane;                // depo slot of this lane
    const int64_t ngroups = U.gprefix[U.n];
    for (int64_t grp = (int64_t)blockIdx.x * NW + wib; grp < ngroups; grp += nwarps) {
        const int uu = find_unit64(U.gprefix, U.n, grp);
        const RasterArgs& a = U.a[uu];
        float* __restrict__ grid = U.grid[uu];
        const W inv_norm = window_norm<W>(a);
        const float* cdf = (cdf_rows > 0 && a.exact_max <= cdf_rows && a.inv_r == a0.inv_r &&
                            a.inv_base == a0.inv_base) ? s_cdf : nullptr;
        const int64_t base = (grp - U.gprefix[uu]) * G;
        const int64_t i = base + dl;
        ExtentT<W> e;
        W q = 0;
        bool bad = false, any = false;
        if (i < a.n) any = depo_extent<W>(a, i, &e, &q, &bad);
        if (bad) atomicOr(a.status, WS_DEV_BAD_DEPO);
        const bool large = any && is_large<SW>(e);
        if (large) {
            const unsigned slot = atomicAdd(list_count, 1u);
            if (slot < list_cap) list[slot] = ((long long)uu << 40) | (long long)i;
        }
        const int ntc = any ? e.k1 - e.k0 + 1 : 0;
        const int nxc = any ? e.w1 - e.w0 + 1 : 0;
        // The per-bin fluctuation into the grid walks quads (four ticks of a
        // wire sharing one Philox block) instead of bins; the same for every
        // depo of the group (one unit).
        const bool quads = MODE == EMIT_GRID && a.fluct && !a.keep_all && a.T != 0u;
        const int nqt = ntc > 0 ? (e.k1 >> 2) - (e.k0 >> 2) + 1 : 0;
        const int ncol = quads ? nqt : ntc;   // items per patch row: quads or bins
        int nb = (any && !large) ? ncol * nxc : 0;
        if (MODE == EMIT_PATCH && i < a.n && !large) {
            const int64_t off = pt.off[i];
            const bool fits = off + nb <= pt.capacity_bins;
            pt.w0[i] = any ? e.w0 : 0;
            pt.t0[i] = any ? e.k0 : 0;
            pt.nw[i] = fits ? nxc : 0;
            pt.nt[i] = fits ? ntc : 0;
            if (!fits) atomicOr(a.status, WS_DEV_PATCH_OVERFLOW);
            if (!fits) nb = 0;
        }
        if (nb > 0) {
            lane_weights<P, W>(a, e.mu_t, e.st, true, e.point_t, e.k0, ntc, inv_norm, s_wt[wib][dl]);
            lane_weights<P, W>(a, e.mu_x, e.sx, false, e.point_x, e.w0, nxc, inv_norm, s_wx[wib][dl]);
        }
        int incl = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        // this lane's depo, handed to the lanes whose items it holds by shuffles
        const int my_start = incl - nb;   // its first item
        const int my_k0 = any ? e.k0 : 0, my_w0 = any ? e.w0 : 0;
        const float my_rnt = ncol > 0 ? 1.f / (float)ncol : 0.f;
        const W my_q = a.fluct ? q : (sizeof(W) == 8 ? (W)a.p64 : (W)a.p) * q;
        __syncwarp();   // the weight tables are written
        // Round gb (every lane): item g = gb + lane lies in depo slot d, the
        // first slot whose inclusive count exceeds g: the slot holding item
        // gb (the number of slots ending at or before gb), unless a slot
        // starts at an item of the round at or before g, the last such one
        // (starts marked in a bitmask, slot numbers in a 32-entry map).  Then
        // the item's index inside that depo's patch, its (row, column) and
        // the depo's values.  Lanes with g >= total get unused values.
        struct Item {
            int d, local, ia, ib, k0, kn, w0;
            W q;
        };
        auto locate = [&](int gb) {
            Item it;
            const int d0 = __popc(__ballot_sync(0xffffffffu, incl <= gb));
            const int s = my_start - gb;
            const bool starts = nb > 0 && s > 0 && s < G;
            const unsigned smask = __reduce_or_sync(0xffffffffu, starts ? 1u << s : 0u);
            __syncwarp();   // the previous round's reads of s_start are done
            if (starts) s_start[wib][s] = (unsigned char)lane;
            __syncwarp();
            const unsigned m = smask & (0xffffffffu >> (31 - lane));
            it.d = m ? (int)s_start[wib][31 - __clz(m)] : (d0 < G ? d0 : G - 1);
            const int sd = __shfl_sync(0xffffffffu, my_start, it.d);
            const float rnt = __shfl_sync(0xffffffffu, my_rnt, it.d);
            const int nc = __shfl_sync(0xffffffffu, ncol, it.d);
            it.k0 = __shfl_sync(0xffffffffu, my_k0, it.d);
            it.kn = __shfl_sync(0xffffffffu, ntc, it.d);
            it.w0 = __shfl_sync(0xffffffffu, my_w0, it.d);
            it.q = __shfl_sync(0xffffffffu, my_q, it.d);
            it.local = gb + lane - sd;
            it.ia = (int)(((float)it.local + 0.5f) * rnt);
            it.ib = it.local - it.ia * nc;
            return it;
        };
        if (quads) {
            // Rounds of 32 quads, one per lane: the lane forms the quad's (up
            // to four) electron counts and, if any bin holds electrons, its
            // Philox block; the bins that draw are compacted with their words
            // into a per-warp list, normal-approximation bins first, so that a
            // warp runs one sampler at a time (only the entry straddling the
            // two kinds diverges).  The survivor counts go back through the
            // list to the quad's lane, which adds the quad's four bins to the
            // grid with one 16-byte atomic (rows of a multiple of four ticks
            // on a 16-byte aligned grid): the lanes of a round hold
            // consecutive quads of a few patch rows, so these atomics touch a
            // few sectors each, where adds from the compacted list would
            // scatter over as many sectors as lanes.
            const unsigned lt = (1u << lane) - 1u;
            const uint32_t qstride = (uint32_t)((a.nticks + 3) >> 2);
            const bool vec4 = P == 0 && (a.nticks & 3) == 0 && ((uintptr_t)grid & 15u) == 0;
            for (int gb = 0; gb < total; gb += 32) {
                const int g = gb + lane;
                int N[4] = {0, 0, 0, 0};
                uint32_t first = 0;
                uint4 x = make_uint4(0u, 0u, 0u, 0u);
                const Item it = locate(gb);
                if (g < total) {
                    const int d = it.d, ia = it.ia;
                    const int k0 = it.k0;
                    const int nt = it.kn;
                    const int w = it.w0 + ia;
                    const int kq = (k0 >> 2) + it.ib;          // the quad's tick group
                    const W qw = it.q * s_wx[wib][d][ia];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int b = 4 * kq + j - k0;
                        N[j] = (b >= 0 && b < nt) ? electrons(qw * s_wt[wib][d][b]) : 0;
                    }
                    first = (uint32_t)w * (uint32_t)a.nticks + (uint32_t)(4 * kq);   // grids hold < 2^31 cells
                    if ((N[0] | N[1] | N[2] | N[3]) > 0)
                        x = philox4x32_10(make_uint4(0u, (uint32_t)w * qstride + (uint32_t)kq,
                                                     a.depo0 + (uint32_t)(base + d), a.evpl), a.key0, a.key1);
                }
                unsigned nbal[4], ebal[4];
                int nbef[4], ebef[4], nn = 0, ne = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool nr = N[j] > a.exact_max;
                    nbal[j] = __ballot_sync(0xffffffffu, nr);
                    ebal[j] = __ballot_sync(0xffffffffu, N[j] > 0 && !nr);
                    nbef[j] = nn;
                    ebef[j] = ne;
                    nn += __popc(nbal[j]);
                    ne += __popc(ebal[j]);
                }
                int pos[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    pos[j] = -1;
                    if (N[j] > 0) {
                        pos[j] = N[j] > a.exact_max ? nbef[j] + __popc(nbal[j] & lt)
                                                    : nn + ebef[j] + __popc(ebal[j] & lt);
                        s_en[wib][pos[j]] = (uint32_t)N[j];
                        s_ew[wib][pos[j]] = word_of(x, j);
                    }
                }
                __syncwarp();
                // the two samplers in passes of their own: a pass never
                // runs both (a pass straddling the two kinds would)
                for (int it = lane; it < nn; it += 32)
                    s_res[wib][it] = normal_word<P>(s_ew[wib][it], (int)s_en[wib][it], a);
                const int ntot = nn + ne;
                for (int it = nn + lane; it < ntot; it += 32) {
                    const int n = (int)s_en[wib][it];
                    const uint32_t xw = s_ew[wib][it];
                    s_res[wib][it] = cdf ? invert_binomial_table(n, xw, a, cdf) : invert_binomial(n, xw, a, s_recip);
                }
                __syncwarp();
                int c[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) c[j] = pos[j] >= 0 ? s_res[wib][pos[j]] : 0;
                if ((c[0] | c[1] | c[2] | c[3]) != 0) {
                    if (vec4) {
                        atomicAdd(reinterpret_cast<float4*>(grid + first),
                                  make_float4((float)c[0], (float)c[1], (float)c[2], (float)c[3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) emit<P>(a, grid, (int64_t)first + j, (W)c[j]);
                    }
                }
                __syncwarp();
            }
        } else {
            for (int gb = 0; gb < total; gb += 32) {
                const Item it = locate(gb);
                if (gb + lane >= total) continue;
                const int d = it.d, ia = it.ia, ib = it.ib;
                const int w = it.w0 + ia, k = it.k0 + ib;
                W v = it.q * s_wx[wib][d][ia] * s_wt[wib][d][ib];
                if (a.fluct)
                    v = (W)binomial_bin<P>(electrons(v), a, w, k, a.depo0 + (uint32_t)(base + d), s_recip, cdf);
                if (MODE == EMIT_GRID) emit<P>(a, grid, (int64_t)w * a.nticks + k, v);
                else pt.val[pt.off[base + d] + it.local] = (float)v;
            }
        }
        __syncwarp();
    }
}

// ---- charge-conserving (multinomial) fluctuation, ws_params.fluctuate = 2
//
// A depo's N = floor(q + 1/2) electrons survive as K ~ Binomial(N, p)
// (Philox block (5, 0, depo, evpl), the sampler of the binomial mode), and
// the K are spread over the patch multinomially with its bin weights: over
// the in-grid wires in order by conditional binomials n_j ~ Binomial(rem,
// w_x[j] / W) (W the wire mass not yet visited, from 1, in float; block
// (4, wire, depo, evpl)), then within wire j over its in-grid ticks alike
// (block (3, wire * nticks + tick, depo, evpl)).  What is still unassigned
// after the last in-grid bin fell off the grid and is lost; when a whole
// axis window lies on the grid its last bin takes all that remain, so an
// interior depo keeps exactly K.  Lane per depo; the wire weights are
// formed edge by edge as the walk goes (one erfc per bin edge), the tick
// weights once per depo into a per-lane shared-memory row.

// Binomial(n, pr) for a float pr: float inversion (same operations as the
// binomial mode's exact branch) for n <= exact_max; else the normal
// approximation with z from words 0, 1 and the mean n pr carried exactly as
// a float pair (hi + lo, the product's rounding error by an FMA), so the
// floor sees hi's integer part exactly and adds the small remainder
// (hi - floor hi) + lo + z sd + 1/2 in float.  (No double arithmetic: this
// GPU's FP64 rate is a small fraction of its FP32 rate.)
__device__ __forceinline__ int binomial_var(int n, float pr, const RasterArgs& a, uint32_t c0, uint32_t c1,
                                            uint32_t depo, const float* recip) {
    if (n <= 0 || !(pr > 0.f)) return 0;
    if (pr >= 1.f) return n;
    const uint4 x = philox4x32_10(make_uint4(c0, c1, depo, a.evpl), a.key0, a.key1);
    if (n <= a.exact_max) {
        const int flip = pr > 0.5f;
        const float sv = flip ? __fsub_rn(1.f, pr) : pr;
        const float base = __fsub_rn(1.f, sv);
        return invert_binomial_s(n, x.x, base, __fdiv_rn(sv, base), flip, recip);
    }
    const float two_m32 = 2.3283064365386963e-10f;
    const float u1 = fmaf((float)x.x, two_m32, 0.5f * two_m32);
    const float u2 = fmaf((float)x.y, two_m32, 0.5f * two_m32);
    const float z = sqrtf(fmaxf(-2.f * __logf(u1), 0.f)) * -__cosf(6.28318530717958648f * (u2 - 0.5f));
    const float nf = (float)n;                 // n < 2^24: exact
    const float hi = nf * pr;
    const float lo = fmaf(nf, pr, -hi);        // n pr = hi + lo exactly
    const float sd = sqrtf(hi * (1.f - pr));
    const float ip = floorf(hi);
    const float kf = ip + floorf(((hi - ip) + lo) + fmaf(z, sd, 0.5f));
    return kf < 0.f ? 0 : (kf > nf ? n : (int)kf);
}

// Standardised clamped edge u and erfc(|u|) of bin edge e along an axis.
struct AxisWalk {
    float mu, inv_s2, umax, delta, inv_norm;
    bool point;
    __device__ __forceinline__ void edge(int e, float& u, float& c) const {
        u = fminf(fmaxf(((float)e * delta - mu) * inv_s2, -umax), umax);
        c = erfcf(fabsf(u));
    }
};

__device__ __forceinline__ AxisWalk axis_walk(float mu, float sigma, float delta, float nsig, bool point,
                                              float inv_norm) {
    AxisWalk w;
    w.mu = mu;
    w.point = point;
    w.delta = delta;
    w.inv_s2 = point ? 0.f : 1.f / (1.41421356237309504880f * sigma);
    w.umax = nsig * 0.70710678118654752440f;
    w.inv_norm = inv_norm;
    return w;
}

// Whether the unclipped window of the axis lies on the grid.
__device__ __forceinline__ bool window_on_grid(float mu, float sigma, float delta, float nsig, bool point,
                                               int nbins) {
    const float lo_e = point ? mu : mu - nsig * sigma;
    const float hi_e = point ? mu : mu + nsig * sigma;
    return floorf(lo_e / delta) >= 0.f && floorf(hi_e / delta) <= (float)(nbins - 1);
}

constexpr int kMultiThreads = 128;
constexpr int kMultiTicks = 32;   // tick weights a lane tabulates once per depo (wider patches: edge by edge)

template <int MODE, int P>
__global__ void __launch_bounds__(kMultiThreads)
raster_multinomial_kernel(const __grid_constant__ RasterUnits U, ws_patches pt) {
    using W = typename PrecT<P>::W;
    __shared__ float s_recip[kExactCap + 1];
    __shared__ float s_wt[kMultiThreads][kMultiTicks + 1];
    float* wtab = s_wt[threadIdx.x];
    fill_recip(s_recip);
    const int64_t total = U.dprefix[U.n];
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int u = find_unit64(U.dprefix, U.n, it);
        const int64_t i = it - U.dprefix[u];
        const RasterArgs& a = U.a[u];
        float* __restrict__ grid = U.grid[u];
        Extent e;
        float q = 0.f;
        bool bad = false;
        const bool any = depo_extent<float>(a, i, &e, &q, &bad);
        if (bad) atomicOr(a.status, WS_DEV_BAD_DEPO);
        const int ntc = any ? e.k1 - e.k0 + 1 : 0;
        const int nxc = any ? e.w1 - e.w0 + 1 : 0;
        int64_t off = 0;
        if (MODE == EMIT_PATCH) {
            off = pt.off[i];
            const bool fits = off + (int64_t)ntc * nxc <= pt.capacity_bins;
            pt.w0[i] = any ? e.w0 : 0;
            pt.t0[i] = any ? e.k0 : 0;
            pt.nw[i] = fits ? nxc : 0;
            pt.nt[i] = fits ? ntc : 0;
            if (!fits) atomicOr(a.status, WS_DEV_PATCH_OVERFLOW);
            if (!fits) continue;
        }
        if (!any) continue;
        const int N = electrons(q);
        int K = 0;
        if (N > 0 && a.T != 0u) {
            if (a.keep_all) {
                K = N;
            } else {
                const uint4 x = philox4x32_10(make_uint4(5u, 0u, a.depo0 + (uint32_t)i, a.evpl), a.key0, a.key1);
                K = N <= a.exact_max ? invert_binomial(N, x.x, a, s_recip) : normal_pair<0>(x, N, a);
            }
        }
        const float inv_norm = window_norm<float>(a);
        const AxisWalk wx = axis_walk(e.mu_x, e.sx, a.pitch, a.nsig, e.point_x, inv_norm);
        const AxisWalk wt = axis_walk(e.mu_t, e.st, a.tick, a.nsig, e.point_t, inv_norm);
        const bool xfull = window_on_grid(e.mu_x, e.sx, a.pitch, a.nsig, e.point_x, a.nwires);
        const bool tfull = window_on_grid(e.mu_t, e.st, a.tick, a.nsig, e.point_t, a.nticks);
        // the tick weights, once per depo when they fit the table
        const bool tab = ntc <= kMultiTicks;
        if (tab) {
            if (e.point_t) {
                wtab[0] = 1.f;
            } else {
                float u0, c0;
                wt.edge(e.k0, u0, c0);
                for (int k = e.k0; k <= e.k1; ++k) {
                    float u1, c1;
                    wt.edge(k + 1, u1, c1);
                    wtab[k - e.k0] = bin_mass(u0, u1, c0, c1) * inv_norm;
                    u0 = u1;
                    c0 = c1;
                }
            }
        }
        int rem = K;
        float Wx = 1.f;
        float ux0 = 0.f, cx0 = 0.f;
        if (!e.point_x) wx.edge(e.w0, ux0, cx0);
        for (int j = e.w0; j <= e.w1; ++j) {
            if (MODE == EMIT_GRID && rem <= 0) break;
            float wj = 1.f;
            if (!e.point_x) {
                float ux1, cx1;
                wx.edge(j + 1, ux1, cx1);
                wj = bin_mass(ux0, ux1, cx0, cx1) * inv_norm;
                ux0 = ux1;
                cx0 = cx1;
            }
            const float prj = (xfull && j == e.w1) ? 1.f : __fdiv_rn(wj, Wx);
            const int nj = binomial_var(rem, prj, a, 4u, (uint32_t)j, a.depo0 + (uint32_t)i, s_recip);
            rem -= nj;
            Wx = __fsub_rn(Wx, wj);
            int rem2 = nj;
            float Wt = 1.f;
            float ut0 = 0.f, ct0 = 0.f;
            if (!tab && !e.point_t) wt.edge(e.k0, ut0, ct0);
            for (int k = e.k0; k <= e.k1; ++k) {
                if (MODE == EMIT_GRID && rem2 <= 0) break;
                float wk = 1.f;
                if (tab) {
                    wk = wtab[k - e.k0];
                } else if (!e.point_t) {
                    float ut1, ct1;
                    wt.edge(k + 1, ut1, ct1);
                    wk = bin_mass(ut0, ut1, ct0, ct1) * inv_norm;
                    ut0 = ut1;
                    ct0 = ct1;
                }
                const float prk = (tfull && k == e.k1) ? 1.f : __fdiv_rn(wk, Wt);
                const int64_t bin = (int64_t)j * a.nticks + k;
                const int m = binomial_var(rem2, prk, a, 3u, (uint32_t)bin, a.depo0 + (uint32_t)i, s_recip);
                rem2 -= m;
                Wt = __fsub_rn(Wt, wk);
                if (MODE == EMIT_GRID) emit<P>(a, grid, bin, (W)m);
                else pt.val[off + (int64_t)(j - e.w0) * ntc + (k - e.k0)] = (float)m;
            }
        }
    }
}

// ---- adjoint of the expected-value raster (warp per depo)
//
// Patch = p q w_t w_x; with u = (e - mu)/sigma clamped to +-n at the window
// bounds, w = [Phi(u1) - Phi(u0)] / erf(n/sqrt 2), and an interior edge
// moves Phi by -phi(u)/sigma per unit mu and -u phi(u)/sigma per unit sigma
// (an edge on the window bound moves with it and contributes nothing).
struct GradArgs {
    const float* dS;       // dL/dS, nwires x nticks
    float* gq;
    float* gx;
    float* gt;
    double* gDL;           // accumulated (caller zeroes), may be null
    double* gDT;
    double DL, DT;
};

// Per-axis weights and their mu / sigma derivatives for bins [first, first + nb)
// (edge values: clamped u, phi(u)/sigma and erfc(|u|/sqrt 2), one per edge).
__device__ __forceinline__ void axis_weights_grad(float mu, float sigma, float delta, float nsig, bool point,
                                                  int first, int nb, float inv_norm, float* u_s, float* c_s,
                                                  float* v_s, float* w, float* dmu, float* dsig, int lane) {
    if (point) {
        for (int b = lane; b < nb; b += 32) { w[b] = 1.f; dmu[b] = 0.f; dsig[b] = 0.f; }
        __syncwarp();
        return;
    }
    const float inv_s = 1.f / sigma;
    for (int j = lane; j <= nb; j += 32) {
        const float e = (float)(first + j) * delta;
        const float u = (e - mu) * inv_s;
        const bool clamped = u <= -nsig || u >= nsig;
        const float uc = fminf(fmaxf(u, -nsig), nsig);
        u_s[j] = uc;
        // phi(u) / sigma, or 0 on a window bound
        c_s[j] = clamped ? 0.f : 0.398942280401432678f * __expf(-0.5f * uc * uc) * inv_s;
        v_s[j] = erfcf(fabsf(uc) * 0.707106781186547524f);
    }
    __syncwarp();
    for (int b = lane; b < nb; b += 32) {
        const float u0 = u_s[b], u1 = u_s[b + 1];
        const float p0 = c_s[b], p1 = c_s[b + 1];
        const float v0 = v_s[b], v1 = v_s[b + 1];
        float m;
        if (u0 >= 0.f) m = 0.5f * (v0 - v1);
        else if (u1 <= 0.f) m = 0.5f * (v1 - v0);
        else m = 1.f - 0.5f * (v0 + v1);
        w[b] = m * inv_norm;
        dmu[b] = -(p1 - p0) * inv_norm;
        dsig[b] = -(u1 * p1 - u0 * p0) * inv_norm;
    }
    __syncwarp();
}

// One more bin on each side of a non-point axis: the FP32 bin range can drop
// a sliver bin whose edge lies within rounding of the window bound; bins
// wholly outside get both edges clamped (zero weight, zero derivative), so
// the clamp test on u alone decides which side of the kink the depo is on.
__device__ __forceinline__ void widen_for_grad(const RasterArgs& a, Extent& e) {
    if (!e.point_t) { e.k0 = max(e.k0 - 1, 0); e.k1 = min(e.k1 + 1, a.nticks - 1); }
    if (!e.point_x) { e.w0 = max(e.w0 - 1, 0); e.w1 = min(e.w1 + 1, a.nwires - 1); }
}

constexpr int kGradT = kSmallT + 2;   // widened patch a lane-per-depo gradient takes
constexpr int kGradX = kSmallW + 2;
constexpr int kGradXWide = kWideW + 2;   // the same on planes binned at pitch / I

template <int GX>
__device__ __forceinline__ bool grad_is_small(const Extent& e) {
    return e.k1 - e.k0 + 1 <= kGradT && e.w1 - e.w0 + 1 <= GX;
}

// One axis of a depo's gradient tables, spread over the kGradLanes lanes of
// its group: edge values (clamped u, phi(u)/sigma, erfc(|u|/sqrt 2)) into
// ed[0..2][j], then bin b's weight and mu / sigma derivatives (as in
// axis_weights_grad) into bn[0..2][b].
constexpr int kGradLanes = 4;

template <int NE>
__device__ __forceinline__ void group_axis_grad(float mu, float sigma, float delta, float nsig, bool point, int first,
                                                int nb, float inv_norm, float (*ed)[NE], float (*bn)[NE - 1], int sub) {
    if (point) {
        if (sub == 0) { bn[0][0] = 1.f; bn[1][0] = 0.f; bn[2][0] = 0.f; }
        __syncwarp();
        return;
    }
    const float inv_s = 1.f / sigma;
    for (int j = sub; j <= nb; j += kGradLanes) {
        const float e = (float)(first + j) * delta;
        const float u = (e - mu) * inv_s;
        const bool clamped = u <= -nsig || u >= nsig;
        const float uc = fminf(fmaxf(u, -nsig), nsig);
        ed[0][j] = uc;
        ed[1][j] = clamped ? 0.f : 0.398942280401432678f * __expf(-0.5f * uc * uc) * inv_s;
        ed[2][j] = erfcf(fabsf(uc) * 0.707106781186547524f);
    }
    __syncwarp();
    for (int b = sub; b < nb; b += kGradLanes) {
        const float u0 = ed[0][b], u1 = ed[0][b + 1];
        const float c0 = ed[1][b], c1 = ed[1][b + 1];
        const float v0 = ed[2][b], v1 = ed[2][b + 1];
        float m;
        if (u0 >= 0.f) m = 0.5f * (v0 - v1);
        else if (u1 <= 0.f) m = 0.5f * (v1 - v0);
        else m = 1.f - 0.5f * (v0 + v1);
        bn[0][b] = m * inv_norm;
        bn[1][b] = -(c1 - c0) * inv_norm;
        bn[2][b] = -(u1 * c1 - u0 * c0) * inv_norm;
    }
    __syncwarp();
}

// dq, dx, dt of one depo from the five patch sums (as in depo_grad_kernel's
// last step) and its D_L, D_T terms.
__device__ __forceinline__ void finish_grad(const RasterArgs& a, const GradArgs& g, int64_t i, bool any, const Extent& e,
                                            float q, float Sq, float Smt, float Sst, float Smx, float Ssx,
                                            double& accL, double& accT) {
    const float pq = a.p * q;
    float dq = 0.f, dx = 0.f, dt = 0.f;
    if (any) {
        dq = a.p * Sq;
        dx = pq * Smx;
        dt = pq * Smt;
        const float dst = pq * Sst, dsx = pq * Ssx;
        if (!a.sig_t && e.mu_t > 0.f) {
            dt += (dst * e.st + dsx * e.sx) / (2.f * e.mu_t);
            if (g.DL > 0.0) accL += (double)dst * e.st / (2.0 * g.DL);
            if (g.DT > 0.0) accT += (double)dsx * e.sx / (2.0 * g.DT);
        }
    }
    if (g.gq) g.gq[i] = dq;
    if (g.gx) g.gx[i] = dx;
    if (g.gt) g.gt[i] = dt;
}

// kGradLanes lanes per depo (eight depos per warp): the group builds its
// depo's widened edge, weight and derivative tables in shared memory and
// splits the patch rows, gathering dL/dS; the partial sums meet by shuffles.
// Depos whose widened patch exceeds kGradT x GX go to depo_grad_kernel
// through the hand-over list.
constexpr int kGradWarps = 4;
constexpr int kGradSlots = 32 / kGradLanes;

template <int GX>
__global__ void __launch_bounds__(32 * kGradWarps)
depo_grad_small_kernel(RasterArgs a, GradArgs g, long long* __restrict__ list, unsigned* list_count,
                       unsigned list_cap) {
    __shared__ float s_te[kGradWarps][kGradSlots][3][kGradT + 1];
    __shared__ float s_tb[kGradWarps][kGradSlots][3][kGradT];
    __shared__ float s_xe[kGradWarps][kGradSlots][3][GX + 1];
    __shared__ float s_xb[kGradWarps][kGradSlots][3][GX];
    __shared__ double s_red[kGradWarps][2];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int slot = lane / kGradLanes, sub = lane % kGradLanes;
    const float inv_norm = 1.f / erff(a.nsig * 0.707106781186547524f);
    double accL = 0.0, accT = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * kGradWarps;
    for (int64_t base = ((int64_t)blockIdx.x * kGradWarps + wib) * kGradSlots; base < a.n;
         base += nwarps * kGradSlots) {
        const int64_t i = base + slot;
        Extent e;
        float q = 0.f;
        bool bad = false, any = false;
        if (i < a.n) any = depo_extent<float>(a, i, &e, &q, &bad);
        if (any) widen_for_grad(a, e);
        const bool mine = i < a.n && (!any || grad_is_small<GX>(e));
        if (sub == 0 && i < a.n && !mine) {   // hand the depo to the warp-per-depo kernel
            const unsigned s = atomicAdd(list_count, 1u);
            if (s < list_cap) list[s] = (long long)i;
        }
        const bool work = any && mine;
        const int nt = work ? e.k1 - e.k0 + 1 : 0, nx = work ? e.w1 - e.w0 + 1 : 0;
        group_axis_grad<kGradT + 1>(work ? e.mu_t : 0.f, work ? e.st : 1.f, a.tick, a.nsig, work && e.point_t,
                                    work ? e.k0 : 0, nt, inv_norm, s_te[wib][slot], s_tb[wib][slot], sub);
        group_axis_grad<GX + 1>(work ? e.mu_x : 0.f, work ? e.sx : 1.f, a.pitch, a.nsig, work && e.point_x,
                                    work ? e.w0 : 0, nx, inv_norm, s_xe[wib][slot], s_xb[wib][slot], sub);
        float Sq = 0.f, Smt = 0.f, Sst = 0.f, Smx = 0.f, Ssx = 0.f;
        const float (*tb)[kGradT] = s_tb[wib][slot];
        const float (*xb)[GX] = s_xb[wib][slot];
        for (int ia = sub; ia < nx; ia += kGradLanes) {
            const float* row = g.dS + (int64_t)(e.w0 + ia) * a.nticks + e.k0;
            float r0 = 0.f, r1 = 0.f, r2 = 0.f;   // sums over the row of gv w_t, gv dmu_t, gv dsig_t
            for (int ib = 0; ib < nt; ++ib) {
                const float gv = __ldg(row + ib);
                r0 = fmaf(gv, tb[0][ib], r0);
                r1 = fmaf(gv, tb[1][ib], r1);
                r2 = fmaf(gv, tb[2][ib], r2);
            }
            Sq = fmaf(xb[0][ia], r0, Sq);
            Smt = fmaf(xb[0][ia], r1, Smt);
            Sst = fmaf(xb[0][ia], r2, Sst);
            Smx = fmaf(xb[1][ia], r0, Smx);
            Ssx = fmaf(xb[2][ia], r0, Ssx);
        }
#pragma unroll
        for (int o = 1; o < kGradLanes; o <<= 1) {
            Sq += __shfl_xor_sync(0xffffffffu, Sq, o);
            Smt += __shfl_xor_sync(0xffffffffu, Smt, o);
            Sst += __shfl_xor_sync(0xffffffffu, Sst, o);
            Smx += __shfl_xor_sync(0xffffffffu, Smx, o);
            Ssx += __shfl_xor_sync(0xffffffffu, Ssx, o);
        }
        if (sub == 0 && mine) finish_grad(a, g, i, any, e, q, Sq, Smt, Sst, Smx, Ssx, accL, accT);
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        accL += __shfl_down_sync(0xffffffffu, accL, o);
        accT += __shfl_down_sync(0xffffffffu, accT, o);
    }
    if (lane == 0) {
        s_red[wib][0] = accL;
        s_red[wib][1] = accT;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0, T = 0.0;
        for (int w = 0; w < kGradWarps; ++w) { L += s_red[w][0]; T += s_red[w][1]; }
        if (g.gDL && L != 0.0) atomicAdd(g.gDL, L);
        if (g.gDT && T != 0.0) atomicAdd(g.gDT, T);
    }
}

// Warp per depo for the depos whose widened patch the lane-per-depo kernel
// leaves (chunks of kChunk bins per axis): the hand-over list's entries if
// they fit in it, else every depo whose widened patch is large.  The last
// block to finish resets the list counter for the next launch.
template <int GX>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
depo_grad_kernel(RasterArgs a, GradArgs g, const long long* __restrict__ list, unsigned* list_count,
                 unsigned list_cap, unsigned* done) {
    __shared__ float s_u[kWarpsPerBlock][kChunk + 1];
    __shared__ float s_c[kWarpsPerBlock][kChunk + 1];
    __shared__ float s_v[kWarpsPerBlock][kChunk + 1];
    __shared__ float s_wt[kWarpsPerBlock][3][kChunk];
    __shared__ float s_wx[kWarpsPerBlock][3][kChunk];
    __shared__ double s_red[kWarpsPerBlock][2];
    const unsigned nlist = *(volatile unsigned*)list_count;
    const bool use_list = nlist <= list_cap;
    if (use_list && nlist == 0u) return;   // nothing handed over, counters already zero
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    const float inv_norm = 1.f / erff(a.nsig * 0.707106781186547524f);
    double accL = 0.0, accT = 0.0;
    const int64_t nitems = use_list ? (int64_t)nlist : a.n;
    for (int64_t it = (int64_t)blockIdx.x * kWarpsPerBlock + wib; it < nitems; it += nwarps) {
        const int64_t i = use_list ? (int64_t)list[it] : it;
        Extent e;
        float q;
        bool bad;
        const bool any = depo_extent<float>(a, i, &e, &q, &bad);
        if (!any) continue;   // written by the lane-per-depo kernel
        widen_for_grad(a, e);
        if (grad_is_small<GX>(e)) continue;
        float Sq = 0.f, Smt = 0.f, Sst = 0.f, Smx = 0.f, Ssx = 0.f;
        for (int kc = any ? e.k0 : 1; any && kc <= e.k1; kc += kChunk) {
            const int ntc = min(kChunk, e.k1 - kc + 1);
            axis_weights_grad(e.mu_t, e.st, a.tick, a.nsig, e.point_t, kc, ntc, inv_norm, s_u[wib], s_c[wib],
                              s_v[wib], s_wt[wib][0], s_wt[wib][1], s_wt[wib][2], lane);
            for (int wc = e.w0; wc <= e.w1; wc += kChunk) {
                const int nxc = min(kChunk, e.w1 - wc + 1);
                axis_weights_grad(e.mu_x, e.sx, a.pitch, a.nsig, e.point_x, wc, nxc, inv_norm, s_u[wib],
                                  s_c[wib], s_v[wib], s_wx[wib][0], s_wx[wib][1], s_wx[wib][2], lane);
                for (int idx = lane; idx < nxc * ntc; idx += 32) {
                    const int ia = idx / ntc, ib = idx - ia * ntc;
                    const float gv = __ldg(g.dS + (int64_t)(wc + ia) * a.nticks + kc + ib);
                    const float wx = s_wx[wib][0][ia], wt = s_wt[wib][0][ib];
                    Sq = fmaf(gv, wx * wt, Sq);
                    Smt = fmaf(gv, wx * s_wt[wib][1][ib], Smt);
                    Sst = fmaf(gv, wx * s_wt[wib][2][ib], Sst);
                    Smx = fmaf(gv, s_wx[wib][1][ia] * wt, Smx);
                    Ssx = fmaf(gv, s_wx[wib][2][ia] * wt, Ssx);
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Sq += __shfl_down_sync(0xffffffffu, Sq, o);
            Smt += __shfl_down_sync(0xffffffffu, Smt, o);
            Sst += __shfl_down_sync(0xffffffffu, Sst, o);
            Smx += __shfl_down_sync(0xffffffffu, Smx, o);
            Ssx += __shfl_down_sync(0xffffffffu, Ssx, o);
        }
        if (lane == 0) finish_grad(a, g, i, any, e, q, Sq, Smt, Sst, Smx, Ssx, accL, accT);
    }
    if (lane == 0) {
        s_red[wib][0] = accL;
        s_red[wib][1] = accT;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0, T = 0.0;
        for (int w = 0; w < kWarpsPerBlock; ++w) { L += s_red[w][0]; T += s_red[w][1]; }
        if (g.gDL && L != 0.0) atomicAdd(g.gDL, L);
        if (g.gDT && T != 0.0) atomicAdd(g.gDT, T);
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            *list_count = 0u;
            *done = 0u;
            __threadfence();
        }
    }
}

__global__ void patch_sizes_kernel(RasterArgs a, int64_t* __restrict__ sizes,
                                   unsigned long long* __restrict__ total) {
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= a.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t sz = 0;
        if (i < a.n) {
            Extent e;
            float q;
            bool bad;
            if (depo_extent<float>(a, i, &e, &q, &bad)) sz = (int64_t)(e.w1 - e.w0 + 1) * (e.k1 - e.k0 + 1);
        }
        if (sizes) sizes[i] = sz;
        mine += (unsigned long long)sz;
    }
    if (total) {
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
    }
}

// ---- exclusive scan (three phases: block scan, scan of block sums, add)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* s_warp, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t before = wid > 0 ? s_warp[wid - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(int64_t* v, int64_t n, int64_t* sums) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        loc[j] = base + j < n ? v[base + j] : 0;
        sum += loc[j];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(sum, s_warp, &total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) v[base + j] = run;
        run += loc[j];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int64_t* sums, int64_t nb) {
    __shared__ int64_t s_warp[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const int64_t x = i < nb ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(x, s_warp, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void scan_add_kernel(int64_t* v, int64_t n, const int64_t* sums) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] += sums[i / kScanTile];
}

// Warp per patch: grid[w0 + a][t0 + b] += val[off + a nt + b].
__global__ void __launch_bounds__(256)
scatter_patches_kernel(ws_patches p, float* __restrict__ grid, int nwires, int nticks) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < p.n; i += nwarps) {
        const int nw = p.nw[i], nt = p.nt[i];
        if (nw <= 0 || nt <= 0) continue;
        const int w0 = p.w0[i], t0 = p.t0[i];
        const int64_t off = p.off[i];
        const int nbin = nw * nt;
        for (int idx = lane; idx < nbin; idx += 32) {
            const int ia = idx / nt, ib = idx - ia * nt;
            const int w = w0 + ia, k = t0 + ib;
            if (w < 0 || w >= nwires || k < 0 || k >= nticks) continue;
            const float v = p.val[off + idx];
            if (v != 0.f) atomicAdd(grid + (int64_t)w * nticks + k, v);
        }
    }
}

int grid_for(int64_t items, int per_block, int blocks_per_sm) {
    int64_t need = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)num_sms() * blocks_per_sm;
    if (need > cap) need = cap;
    if (need < 1) need = 1;
    return (int)need;
}

}  // namespace

// SM count of the current device, cached per device (any thread may ask).
// Only grid sizes depend on it and every kernel sized by it strides over its
// work, so if the query fails (the next launch then reports the error) one
// is returned and nothing is cached.
int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

static RasterUnits raster_units(const RasterBatch& rb) {
    RasterUnits U;
    U.n = rb.n;
    U.gprefix[0] = 0;
    U.dprefix[0] = 0;
    for (int i = 0; i < rb.n; ++i) {
        U.a[i] = rb.a[i];
        U.grid[i] = rb.grid[i];
        U.rows[i] = nullptr;
        U.cls[i] = nullptr;
        U.imp[i] = 1;
        U.gprefix[i + 1] = U.gprefix[i] + (rb.a[i].n + kSmallGroup - 1) / kSmallGroup;
        U.dprefix[i + 1] = U.dprefix[i] + rb.a[i].n;
    }
    return U;
}

template <int MODE, int P, int SW>
static cudaError_t launch_raster_pair(const RasterUnits& U, const ws_patches& p, const LargeList& L, int rows,
                                      size_t dyn, int blocks, cudaStream_t s) {
    raster_small_kernel<MODE, P, SW><<<blocks, 32 * kSmallWarpsPerBlock, dyn, s>>>(U, p, L.list, L.count, L.cap, rows);
    raster_kernel<MODE, P, SW><<<num_sms() * 2, 32 * kWarpsPerBlock, dyn, s>>>(U, p, L.list, L.count, L.cap, L.done,
                                                                           rows);
    return cudaGetLastError();
}

template <int MODE, int P>
static cudaError_t launch_raster_units(const RasterUnits& U, const ws_patches& p, const LargeList& L,
                                       cudaStream_t s) {
    if (U.dprefix[U.n] <= 0) return cudaSuccess;
    if (U.a[0].fluct == 2) {   // every unit of a call shares its fluctuation mode
        raster_multinomial_kernel<MODE, P><<<grid_for(U.dprefix[U.n], kMultiThreads, 16), kMultiThreads, 0, s>>>(U, p);
        return cudaGetLastError();
    }
    const int64_t groups = U.gprefix[U.n];
    int blocks = grid_for(groups * 32, 32 * kSmallWarpsPerBlock, 16);
    // CDF rows for the exact branch of unit 0's survival probability (rows up
    // to its exact_max), in dynamic shared memory
    const RasterArgs& a0 = U.a[0];
    const int rows = (a0.fluct && !a0.keep_all && a0.T != 0u) ? (a0.exact_max < kExactCap ? a0.exact_max : kExactCap) : 0;
    const size_t dyn = sizeof(float) * (size_t)rows * (rows + 1) / 2;
    // a launch's units are all fine-pitch (impact) planes or none is; the
    // FP64 path's tables would not fit the wide variant's shared memory (its
    // wide patches take the warp-per-depo kernel)
    if constexpr (P <= 1) {
        if (a0.wide) return launch_raster_pair<MODE, P, kWideW>(U, p, L, rows, dyn, blocks, s);
    }
    return launch_raster_pair<MODE, P, kSmallW>(U, p, L, rows, dyn, blocks, s);
}

cudaError_t launch_raster_scatter_batch(const RasterBatch& rb, const LargeList& L, cudaStream_t s) {
    ws_patches none{};
    switch (rb.prec) {
        case WS_PREC_FP32_COMP: return launch_raster_units<EMIT_GRID, 1>(raster_units(rb), none, L, s);
        case WS_PREC_FP64: return launch_raster_units<EMIT_GRID, 2>(raster_units(rb), none, L, s);
        default: return launch_raster_units<EMIT_GRID, 0>(raster_units(rb), none, L, s);
    }
}

cudaError_t launch_raster_scatter(const RasterArgs& a, float* grid, const LargeList& L, cudaStream_t s) {
    RasterBatch rb;
    rb.n = 1;
    rb.prec = a.prec;
    rb.a[0] = a;
    rb.grid[0] = grid;
    return launch_raster_scatter_batch(rb, L, s);
}

cudaError_t launch_patch_sizes(const RasterArgs& a, int64_t* sizes, unsigned long long* total, cudaStream_t s) {
    patch_sizes_kernel<<<grid_for(a.n + 1, 256, 8), 256, 0, s>>>(a, sizes, total);
    return cudaGetLastError();
}

cudaError_t launch_scan_inplace(int64_t* v, int64_t n, int64_t* scratch, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kScanScratch) return cudaErrorInvalidValue;
    scan_tiles_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(v, n, scratch);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(scratch, nb);
    scan_add_kernel<<<grid_for(n, 256, 8), 256, 0, s>>>(v, n, scratch);
    return cudaGetLastError();
}

cudaError_t launch_raster_patches(const RasterArgs& a, const ws_patches& p, const LargeList& L, cudaStream_t s) {
    RasterBatch rb;
    rb.n = 1;
    rb.prec = WS_PREC_FP32;
    rb.a[0] = a;
    rb.grid[0] = nullptr;
    return launch_raster_units<EMIT_PATCH, 0>(raster_units(rb), p, L, s);
}

cudaError_t launch_scatter_patches(const ws_patches& p, float* grid, int nwires, int nticks, cudaStream_t s) {
    if (p.n <= 0) return cudaSuccess;
    scatter_patches_kernel<<<grid_for(p.n, 8, 8), 256, 0, s>>>(p, grid, nwires, nticks);
    return cudaGetLastError();
}

// Zero every unit's grid (float4 stores; grids are 16-byte aligned and a
// multiple of 4 floats, else the tail is done with scalar stores).
__global__ void zero_grids_kernel(const __grid_constant__ RasterUnits U, const __grid_constant__ ZeroSizes Z) {
    for (int u = 0; u < U.n; ++u) {
        float* g = U.grid[u];
        const int64_t n = Z.count[u];
        const int64_t n4 = ((uintptr_t)g % 16 == 0) ? n / 4 : 0;
        float4* g4 = reinterpret_cast<float4*>(g);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
            g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            g[i] = 0.f;
    }
}

cudaError_t launch_zero_grids(const RasterBatch& rb, const int64_t* counts, cudaStream_t s) {
    RasterUnits U = raster_units(rb);
    ZeroSizes Z;
    for (int i = 0; i < rb.n; ++i) Z.count[i] = counts[i];
    zero_grids_kernel<<<num_sms() * 4, 256, 0, s>>>(U, Z);
    return cudaGetLastError();
}

// Active rows, step 1: every depo marks the wire rows [w0 - 1, w1 + 1] of its
// clipped pitch-axis range (the raster's own extent, computed the same way,
// widened by one wire against rounding differences between the two
// kernels) with the new epoch, base + 1.  On an impact plane (pitch axis
// binned at pitch / I) the range is in fine bins: widened by one fine bin,
// it marks the wires w0 / I .. w1 / I that hold those bins.  Block (x, u) takes unit u's depos
// x, x + gridDim.x, ... (256 at a time) with the unit's parameters staged in
// shared memory.  Depos along a track share rows, and many threads storing
// to the same few words serialise in L2, so a warp merges its lanes' ranges
// when they fall within 32 rows and stores each of their rows once.  Block
// (0, 0) stores the epoch; `base` is not written while this kernel runs.
struct MarkUnit {
    const float* x;
    const float* t;
    const float* sig_x;   // null: widths from diffusion
    int64_t n;
    float two_DT, pitch, nsig;
    int nwires;   // bins of the pitch axis (wires x impact positions)
    int imp;      // bins per marked row
    mark_t* rows;
};

__device__ __forceinline__ MarkUnit mark_unit(const RasterUnits& U, int u) {
    const RasterArgs& a = U.a[u];
    return MarkUnit{a.x, a.t, a.sig_t ? a.sig_x : nullptr, a.n, a.two_DT, a.pitch, a.nsig, a.nwires, U.imp[u],
                    U.rows[u]};
}

__global__ void __launch_bounds__(256)
mark_rows_kernel(const __grid_constant__ RasterUnits U, const mark_t* base_epoch, mark_t* epoch) {
    __shared__ MarkUnit mu;
    const mark_t e = read_epoch(base_epoch) + 1ull;
    if (threadIdx.x == 0) mu = mark_unit(U, blockIdx.y);
    __syncthreads();
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *epoch = e;
    if (!mu.rows) return;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together (the merge below needs every lane)
    for (int64_t wbase = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); wbase < mu.n; wbase += stride) {
        const int64_t i = wbase + lane;
        int lo = 0, hi = -1;
        if (i < mu.n) {
            const float x = __ldg(mu.x + i);
            float sx;
            if (mu.sig_x) {
                sx = __ldg(mu.sig_x + i);
            } else {
                const float t = __ldg(mu.t + i);
                sx = sqrtf(mu.two_DT * (t > 0.f ? t : 0.f));
            }
            bool point = false;
            axis_range<float>(x, sx, mu.pitch, mu.nsig, mu.nwires, &lo, &hi, &point);
            lo = lo - 1 > 0 ? lo - 1 : 0;
            hi = hi + 1 < mu.nwires - 1 ? hi + 1 : mu.nwires - 1;
            if (mu.imp > 1 && lo <= hi) {
                lo /= mu.imp;
                hi /= mu.imp;
            }
        }
        const bool has = lo <= hi;
        const int mlo = __reduce_min_sync(0xffffffffu, has ? lo : INT_MAX);
        const int mhi = __reduce_max_sync(0xffffffffu, has ? hi : -1);
        if (mhi < 0) continue;   // no lane marks anything
        if (mhi - mlo < 32) {
            const uint32_t mine =
                has ? (uint32_t)((2ull << (hi - mlo)) - 1ull) & ~((1u << (lo - mlo)) - 1u) : 0u;
            if ((__reduce_or_sync(0xffffffffu, mine) >> lane) & 1u) mu.rows[mlo + lane] = e;
        } else if (has) {
            for (int w = lo; w <= hi; ++w) mu.rows[w] = e;
        }
    }
}

// Active rows, step 2: clear the marked rows of unit u's grid (and of its
// compensated low-part grid), a warp per row, or the whole grid of a unit
// without marks; with marks, also write every row's class (ROW_MARKED,
// ROW_NEEDED: a marked row in [w - kw + 1, w + K - 1], ROW_LIVE: a marked
// row in [w + c - kw + 1, w + c]) from the marks of rows w - (kw - 1) ..
// w + 32 + 31 - (kw - 1), two per lane (kw, K <= 21, so the widest window,
// kw + K - 1 rows, fits in 64).  On an impact plane a marked wire's I fine
// rows are cleared (a warp each).  Block (0, 0) hands the
// epoch on to the next call's marking kernel (`base`; the marking kernel is
// not running).
struct ZeroUnit {
    float* grid;
    float* lo;
    const mark_t* rows;   // null: every row
    uint32_t* cls;
    int nwires, nticks;   // marked rows (wires) and ticks per grid row
    int imp;              // grid rows per marked row (a warp clears one)
};

__global__ void __launch_bounds__(256)
zero_marked_rows_kernel(const __grid_constant__ RasterUnits U, const mark_t* epoch, mark_t* base, int kw,
                        int center) {
    __shared__ ZeroUnit zu;
    const mark_t cur = read_epoch(epoch);
    if (threadIdx.x == 0) {
        const int u = blockIdx.y;
        const int imp = U.rows[u] ? U.imp[u] : 1;   // without marks: every fine row on its own
        zu = ZeroUnit{U.grid[u], U.a[u].lo, U.rows[u], U.cls[u], U.a[u].nwires / imp, U.a[u].nticks, imp};
    }
    __syncthreads();
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && base) *base = cur;
    const int lane = threadIdx.x & 31;
    const int nt = zu.nticks, nw = zu.nwires, imp = zu.imp;
    // item (w, piece): grid row w * imp + piece, cleared if wire w is marked
    for (int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < nw * imp;
         item += gridDim.x * (blockDim.x >> 5)) {
        const int w = item / imp, piece = item - w * imp;
        bool marked = true;
        if (zu.rows) {
            const int r0 = w - (kw - 1) + lane, r1 = r0 + 32;
            const bool m0 = r0 >= 0 && r0 < nw && zu.rows[r0] == cur;
            const bool m1 = r1 >= 0 && r1 < nw && zu.rows[r1] == cur;
            const unsigned long long mm =
                (unsigned long long)__ballot_sync(0xffffffffu, m0) | ((unsigned long long)__ballot_sync(0xffffffffu, m1) << 32);
            marked = (mm >> (kw - 1)) & 1ull;
            const bool needed = (mm & ((2ull << (kw - 1 + kMaxRespWires - 1)) - 1ull)) != 0ull;
            const bool live = ((mm >> center) & ((1ull << kw) - 1ull)) != 0ull;
            if (lane == 0 && piece == 0)
                zu.cls[w] = (marked ? ROW_MARKED : 0u) | (needed ? ROW_NEEDED : 0u) | (live ? ROW_LIVE : 0u);
        }
        if (!marked) continue;
        for (int g = 0; g < 2; ++g) {
            float* row = g == 0 ? zu.grid : zu.lo;
            if (!row) continue;
            row += (int64_t)item * nt;
            if ((uintptr_t)row % 16 == 0 && nt % 4 == 0) {
                float4* r4 = reinterpret_cast<float4*>(row);
                for (int j = lane; j < nt / 4; j += 32) r4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                for (int j = lane; j < nt; j += 32) row[j] = 0.f;
            }
        }
    }
}

cudaError_t launch_mark_rows(const RasterBatch& rb, const RowMarks& m, cudaStream_t s) {
    if (rb.n <= 0) return cudaSuccess;
    RasterUnits U = raster_units(rb);
    int64_t maxn = 0;
    for (int i = 0; i < rb.n; ++i) {
        U.rows[i] = m.rows[i];
        U.imp[i] = m.impacts[i] > 1 ? m.impacts[i] : 1;
        if (rb.a[i].nwires % U.imp[i] != 0) return cudaErrorInvalidValue;
        maxn = std::max<int64_t>(maxn, rb.a[i].n);
    }
    // at least one block per unit (block (0, 0) stores the epoch)
    const int bx = (int)std::max<int64_t>(1, std::min<int64_t>((maxn + 255) / 256, 256));
    mark_rows_kernel<<<dim3(bx, rb.n), 256, 0, s>>>(U, m.base, m.epoch);
    return cudaGetLastError();
}

cudaError_t launch_zero_marked_rows(const RasterBatch& rb, const RowMarks& m, cudaStream_t s) {
    if (rb.n <= 0) return cudaSuccess;
    if (m.kw < 1 || m.kw > 32 || m.center < 0 || m.center >= m.kw) return cudaErrorInvalidValue;
    RasterUnits U = raster_units(rb);
    int maxw = 1;
    for (int i = 0; i < rb.n; ++i) {
        U.rows[i] = m.rows[i];
        U.cls[i] = m.rows[i] ? m.cls[i] : nullptr;
        U.imp[i] = m.impacts[i] > 1 ? m.impacts[i] : 1;
        if (m.rows[i] && !m.cls[i]) return cudaErrorInvalidValue;
        if (rb.a[i].nwires % U.imp[i] != 0) return cudaErrorInvalidValue;
        maxw = std::max(maxw, rb.a[i].nwires);   // grid rows (a warp each)
    }
    const int bx = (maxw + 7) / 8;   // a warp per row
    zero_marked_rows_kernel<<<dim3(bx, rb.n), 256, 0, s>>>(U, m.epoch, m.base, m.kw, m.center);
    return cudaGetLastError();
}

cudaError_t launch_depo_grads(const RasterArgs& a, const float* dS, float* gq, float* gx, float* gt, double* gDL,
                              double* gDT, double DL, double DT, const LargeList& L, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    GradArgs g{dS, gq, gx, gt, gDL, gDT, DL, DT};
    const int blocks = grid_for((a.n + kGradSlots - 1) / kGradSlots, kGradWarps, 8);
    if (a.wide) {   // impact planes: up to kWideW fine wire bins per patch
        depo_grad_small_kernel<kGradXWide><<<blocks, 32 * kGradWarps, 0, s>>>(a, g, L.list, L.count, L.cap);
        depo_grad_kernel<kGradXWide><<<num_sms() * 2, 32 * kWarpsPerBlock, 0, s>>>(a, g, L.list, L.count, L.cap,
                                                                                    L.done);
    } else {
        depo_grad_small_kernel<kGradX><<<blocks, 32 * kGradWarps, 0, s>>>(a, g, L.list, L.count, L.cap);
        depo_grad_kernel<kGradX><<<num_sms() * 2, 32 * kWarpsPerBlock, 0, s>>>(a, g, L.list, L.count, L.cap,
                                                                                L.done);
    }
    return cudaGetLastError();
}

}  // namespace ws
