// FFT convolution of a wire x tick grid with the detector response (Eq. 2).
//
// The 2D transform of Eq. 2 is split by axis:
//   1. fwd_rows   real FFT of every wire row along ticks (length L_t, zero
//                 padded), two real rows packed into one complex transform;
//   2. wire_conv  in the tick-frequency domain the wire direction is a short
//                 convolution (K_w <= 21 taps) with the response's per-row
//                 tick spectra, done directly with register blocking: this
//                 is Eq. 2's product R_hat * S_hat with the wire-axis
//                 transform carried out as the equivalent sum, so no
//                 nwires x L_t response spectrum has to be streamed from HBM;
//   3. inv_rows   inverse real FFT of every row, cropped to the grid.
// Transforms are mixed-radix Stockham autosort passes in shared memory with
// radices up to 25 (composites done as two register-level stages with
// compile-time twiddles) and a per-pass table of inter-pass twiddles.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "ws_internal.cuh"

namespace ws {
namespace {

// ---------------------------------------------------------------- helpers
// Compile-time unrolled loop: f(integral_constant<int, i>) for i in [0, N).
template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// cos and sin of 2 pi m / n in double at compile time: exact octant
// reduction of the rational angle, then Taylor series on |a| <= pi/4.
constexpr double kPi = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double cx_sin_small(double a) {
    double a2 = a * a, term = a, sum = a;
    for (int i = 1; i < 14; ++i) { term *= -a2 / ((2.0 * i) * (2.0 * i + 1.0)); sum += term; }
    return sum;
}
__host__ __device__ constexpr double cx_cos_small(double a) {
    double a2 = a * a, term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) { term *= -a2 / ((2.0 * i - 1.0) * (2.0 * i)); sum += term; }
    return sum;
}
// Returns cos (want_sin = false) or sin of 2 pi m / n.
__host__ __device__ constexpr double cx_trig2pi(long m, long n, bool want_sin) {
    long t = (8 * (m % n) + 8 * n) % (8 * n);   // angle in units of pi/(4n)
    long o = t / n, r = t - o * n;               // octant and remainder
    double a = 0.0;
    long q = 0;
    if (o % 2 == 0) { a = (kPi / 4.0) * (double)r / (double)n; q = o / 2; }
    else { a = -(kPi / 4.0) * (double)(n - r) / (double)n; q = (o + 1) / 2; }
    double c = cx_cos_small(a), s = cx_sin_small(a);
    double cc = c, ss = s;
    switch (q % 4) {
        case 0: cc = c; ss = s; break;
        case 1: cc = -s; ss = c; break;
        case 2: cc = -c; ss = -s; break;
        default: cc = s; ss = -c; break;
    }
    return want_sin ? ss : cc;
}

// Complex arithmetic on float2 (FP32 path) or double2 (FP64 path).
template <typename S> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename S> using cplx = typename CplxOf<S>::type;

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { return mkc(a.x * s, a.y * s); }
// a * w (forward) or a * conj(w) (inverse)
template <bool INV, typename C>
__device__ __forceinline__ C cmul_tw(C a, C w) {
    if (INV) w.y = -w.y;
    return mkc(fmx(a.x, w.x, -a.y * w.y), fmx(a.x, w.y, a.y * w.x));
}
// -i*a (forward) or +i*a (inverse)
template <bool INV, typename C>
__device__ __forceinline__ C mul_mi(C a) {
    return INV ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}

// x * e^{-+2 pi i M / N} with M, N compile-time.
template <int N, int M, bool INV, typename C>
__device__ __forceinline__ C rot(C x) {
    using S = decltype(x.x);
    constexpr int m = M % N;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (2 * m == N) {
        return mkc(-x.x, -x.y);
    } else if constexpr (4 * m == N) {
        return mul_mi<INV>(x);
    } else if constexpr (4 * m == 3 * N) {
        return mul_mi<!INV>(x);
    } else {
        constexpr S c = (S)cx_trig2pi(m, N, false);
        constexpr S s = INV ? (S)cx_trig2pi(m, N, true) : -(S)cx_trig2pi(m, N, true);
        return mkc(fmx(x.x, c, -x.y * s), fmx(x.x, s, x.y * c));
    }
}

// ------------------------------------------------------------ small DFTs
// y_m = sum_n x_n e^{-+2 pi i m n / R}, in place, natural order.
template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<2, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV, typename C> struct Dft<3, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        using S = decltype(v[0].x);
        const S s3 = (S)0.866025403784438646763723170752936183;  // sin(2 pi / 3)
        C t1 = cadd(v[1], v[2]);
        C t2 = csub(v[1], v[2]);
        C a = mkc(fmx((S)-0.5, t1.x, v[0].x), fmx((S)-0.5, t1.y, v[0].y));
        C b = mul_mi<INV>(cscale(t2, s3));
        v[0] = cadd(v[0], t1);
        v[1] = cadd(a, b);
        v[2] = csub(a, b);
    }
};

template <bool INV, typename C> struct Dft<4, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        C s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <bool INV, typename C> struct Dft<5, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        using S = decltype(v[0].x);
        const S c1 = (S)0.309016994374947424102293417182819059;   // cos(2 pi / 5)
        const S c2 = (S)-0.809016994374947424102293417182819059;  // cos(4 pi / 5)
        const S s1 = (S)0.951056516295153572116439333379382143;   // sin(2 pi / 5)
        const S s2 = (S)0.587785252292473129168705954639072769;   // sin(4 pi / 5)
        C t1 = cadd(v[1], v[4]), t3 = csub(v[1], v[4]);
        C t2 = cadd(v[2], v[3]), t4 = csub(v[2], v[3]);
        C x0 = v[0];
        C a1 = mkc(fmx(c1, t1.x, fmx(c2, t2.x, x0.x)), fmx(c1, t1.y, fmx(c2, t2.y, x0.y)));
        C a2 = mkc(fmx(c2, t1.x, fmx(c1, t2.x, x0.x)), fmx(c2, t1.y, fmx(c1, t2.y, x0.y)));
        C b1 = mkc(fmx(s1, t3.x, s2 * t4.x), fmx(s1, t3.y, s2 * t4.y));
        C b2 = mkc(fmx(s2, t3.x, -s1 * t4.x), fmx(s2, t3.y, -s1 * t4.y));
        b1 = mul_mi<INV>(b1);
        b2 = mul_mi<INV>(b2);
        v[0] = cadd(x0, cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

// Composite N = N1 N2 (Cooley-Tukey in registers): with n = N2 n1 + n2 and
// k = k1 + N1 k2, X[k] = sum_n2 W_N2^(n2 k2) W_N^(n2 k1) sum_n1 x[n] W_N1^(n1 k1).
template <int N1, int N2, bool INV, typename C>
__device__ __forceinline__ void dft_composite(C* v) {
    constexpr int N = N1 * N2;
    sfor<N2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        C t[N1];
        sfor<N1>([&](auto n1c) { t[decltype(n1c)::value] = v[N2 * decltype(n1c)::value + n2]; });
        Dft<N1, INV, C>::run(t);
        sfor<N1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            v[N2 * k1 + n2] = rot<N, n2 * k1, INV>(t[k1]);
        });
    });
    C out[N];
    sfor<N1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        C t[N2];
        sfor<N2>([&](auto n2c) { t[decltype(n2c)::value] = v[N2 * k1 + decltype(n2c)::value]; });
        Dft<N2, INV, C>::run(t);
        sfor<N2>([&](auto k2c) { out[k1 + N1 * decltype(k2c)::value] = t[decltype(k2c)::value]; });
    });
    sfor<N>([&](auto ic) { v[decltype(ic)::value] = out[decltype(ic)::value]; });
}

#define WS_COMPOSITE(R, A, B)                                                             \
    template <bool INV, typename C> struct Dft<R, INV, C> {                                \
        __device__ __forceinline__ static void run(C* v) { dft_composite<A, B, INV>(v); } \
    };
WS_COMPOSITE(6, 3, 2)
WS_COMPOSITE(8, 4, 2)
WS_COMPOSITE(9, 3, 3)
WS_COMPOSITE(10, 5, 2)
WS_COMPOSITE(12, 4, 3)
WS_COMPOSITE(15, 5, 3)
WS_COMPOSITE(16, 4, 4)
WS_COMPOSITE(20, 5, 4)
WS_COMPOSITE(25, 5, 5)
#undef WS_COMPOSITE

// ------------------------------------------------------- Stockham passes
constexpr int kRowThreads = 256;

// Unit owning global block b: the last u with prefix[u] <= b.
__device__ __forceinline__ int find_unit(const int* prefix, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ noise
// Standard normals z1, z2 from two Philox words by Box-Muller: u = (m + 1/2)
// 2^-23 with m the word's top 23 bits (exact in float and double), z1 =
// sqrt(-2 ln u1) cos(2 pi u2), z2 = sqrt(-2 ln u1) sin(2 pi u2).  In single
// precision the hardware logarithm, sine, cosine and reciprocal square root
// (absolute errors ~2^-21 on these ranges: ~1e-6 of a typical normal) keep
// the noise well inside the FP32 path's 1e-5; cos(2 pi u) = -cos(2 pi (u -
// 1/2)) puts the argument in [-pi, pi].
__device__ __forceinline__ void normal_pair(uint32_t a, uint32_t b, float& z1, float& z2) {
    const float u1 = ((float)(a >> 9) + 0.5f) * 1.1920928955078125e-7f;
    const float u2 = ((float)(b >> 9) + 0.5f) * 1.1920928955078125e-7f;
    const float t = -2.0f * __logf(u1);   // > 0: u1 < 1
    const float rad = t * rsqrtf(t);
    const float ang = 6.28318530717958648f * (u2 - 0.5f);
    z1 = -rad * __cosf(ang);
    z2 = -rad * __sinf(ang);
}
__device__ __forceinline__ void normal_pair(uint32_t a, uint32_t b, double& z1, double& z2) {
    const double u1 = ((double)(a >> 9) + 0.5) * 1.1920928955078125e-7;
    const double u2 = ((double)(b >> 9) + 0.5) * 1.1920928955078125e-7;
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    z1 = rad * cs;
    z2 = rad * sn;
}

// xi from words 2h, 2h + 1 of block x: (z1 + i z2) / sqrt 2, or z1 on the
// real bins (k = 0, k = L/2).
template <typename C>
__device__ __forceinline__ C noise_xi(const uint4& x, int h, bool edge) {
    using S = decltype(C{}.x);
    S z1, z2;
    normal_pair(h ? x.z : x.x, h ? x.w : x.y, z1, z2);
    if (edge) return mkc(z1, (S)0);
    const S r = (S)0.70710678118654752440;
    return mkc(z1 * r, z2 * r);
}

// Noise term of Eq. 1 added to the spectra Y (between the wire convolution
// and the inverse transform; Y carries the 1/L of the unnormalised
// inverse): thread = one bin k of one unit and a block of kNoiseRows wires,
// taken in pairs (one Philox block serves a pair's incoherent draws); the
// coherent draw of a group is made once per run of the group's wires in the
// block and reused.
constexpr int kNoiseRows = 8;
constexpr int kNoiseCols = 128;

template <typename C>
__global__ void __launch_bounds__(kNoiseCols)
add_noise_kernel(const __grid_constant__ NoiseUnits U, int nfreq, int L, int64_t stride) {
    using S = decltype(C{}.x);
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.y);
    const int k = blockIdx.x * kNoiseCols + threadIdx.x;
    if (k >= nfreq) return;
    const NoiseUnit& nz = U.noise[u];
    C* __restrict__ Y = static_cast<C*>(U.Y[u]);
    const int w0 = ((int)blockIdx.y - U.prefix[u]) * kNoiseRows;   // even
    const int nr = min(kNoiseRows, U.nwires[u] - w0);
    // the block's spectra first (independent loads in flight), then the draws
    C yv[kNoiseRows];
#pragma unroll
    for (int i = 0; i < kNoiseRows; ++i)
        if (i < nr) yv[i] = Y[(int64_t)(w0 + i) * stride + k];
    const bool edge = k == 0 || 2 * k == L;
    const S a = (S)__ldg(nz.amp + k) * (S)nz.scale;
    const S c = nz.coh ? (S)__ldg(nz.coh + k) * (S)nz.scale : (S)0;
    // the pairs' incoherent blocks first (independent Philox chains in flight)
    uint4 xs[kNoiseRows / 2];
#pragma unroll
    for (int i = 0; i < kNoiseRows; i += 2)
        if (i < nr) xs[i / 2] = philox4x32_10(make_uint4(1u, (uint32_t)k, (uint32_t)((w0 + i) >> 1), nz.evpl), U.key0,
                                              U.key1);
#pragma unroll
    for (int i = 0; i < kNoiseRows; ++i) {
        if (i < nr) {
            const C v = noise_xi<C>(xs[i / 2], i & 1, edge);
            yv[i].x += a * v.x;
            yv[i].y += a * v.y;
        }
    }
    if (nz.coh) {
        // the block's wires span groups g_first .. g_last (usually one)
        int gr[kNoiseRows];
#pragma unroll
        for (int i = 0; i < kNoiseRows; ++i) gr[i] = (w0 + i) / nz.group;
        for (int g = gr[0]; g <= gr[nr - 1]; ++g) {
            const uint4 y = philox4x32_10(make_uint4(2u, (uint32_t)k, (uint32_t)(g >> 1), nz.evpl), U.key0, U.key1);
            const C xg = noise_xi<C>(y, g & 1, edge);
#pragma unroll
            for (int i = 0; i < kNoiseRows; ++i) {
                if (i < nr && gr[i] == g) {
                    yv[i].x += c * xg.x;
                    yv[i].y += c * xg.y;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kNoiseRows; ++i)
        if (i < nr) Y[(int64_t)(w0 + i) * stride + k] = yv[i];
}

template <typename C>
static cudaError_t add_noise_t(const NoiseBatch& nb, int nfreq, int L, int64_t stride, cudaStream_t s) {
    NoiseUnits U;
    U.n = 0;
    U.prefix[0] = 0;
    U.key0 = nb.key0;
    U.key1 = nb.key1;
    for (int i = 0; i < nb.n; ++i) {
        if (!nb.noise[i].amp) continue;
        const int j = U.n++;
        U.Y[j] = nb.Y[i];
        U.nwires[j] = nb.nwires[i];
        U.noise[j] = nb.noise[i];
        U.prefix[j + 1] = U.prefix[j] + (nb.nwires[i] + kNoiseRows - 1) / kNoiseRows;
    }
    if (U.n == 0 || U.prefix[U.n] == 0 || nfreq <= 0) return cudaSuccess;
    dim3 grid((nfreq + kNoiseCols - 1) / kNoiseCols, U.prefix[U.n]);
    add_noise_kernel<C><<<grid, kNoiseCols, 0, s>>>(U, nfreq, L, stride);
    return cudaGetLastError();
}

// One Stockham pass of radix R over a length-L sequence: butterfly j reads
// src[j + r L/R], multiplies input r by w^r with w = e^{-+2 pi i (j mod Ns) /
// (Ns R)} (w from the pass's table of Ns base twiddles, its powers by a
// multiply tree of depth <= 5), and writes dst[(j - j mod Ns) R + j mod Ns +
// r Ns].
template <int R, bool INV, typename C>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst,
                                              int L, int Ns, const C* __restrict__ tw) {
    const int nb = L / R;
    for (int j = threadIdx.x; j < nb; j += kRowThreads) {
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
        if (Ns > 1) {
            C wp[R];
            wp[1] = tw[k];
            if (INV) wp[1].y = -wp[1].y;
#pragma unroll
            for (int r = 2; r < R; ++r) wp[r] = cmul_tw<false>(wp[r / 2], wp[r - r / 2]);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul_tw<false>(v[r], wp[r]);
        }
        Dft<R, INV, C>::run(v);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[d + r * Ns] = v[r];
    }
}

// Full transform in shared memory; returns the buffer holding the result.
template <bool INV, typename C>
__device__ C* fft_smem(const FftPlan& plan, C* a, C* b, const C* __restrict__ tw) {
    C* src = a;
    C* dst = b;
    for (int p = 0; p < plan.npass; ++p) {
        const int Ns = plan.ns[p];
        const C* t = tw + plan.twoff[p];
        switch (plan.radix[p]) {
            case 2: stockham_pass<2, INV>(src, dst, plan.L, Ns, t); break;
            case 3: stockham_pass<3, INV>(src, dst, plan.L, Ns, t); break;
            case 4: stockham_pass<4, INV>(src, dst, plan.L, Ns, t); break;
            case 5: stockham_pass<5, INV>(src, dst, plan.L, Ns, t); break;
            case 6: stockham_pass<6, INV>(src, dst, plan.L, Ns, t); break;
            case 8: stockham_pass<8, INV>(src, dst, plan.L, Ns, t); break;
            case 9: stockham_pass<9, INV>(src, dst, plan.L, Ns, t); break;
            case 10: stockham_pass<10, INV>(src, dst, plan.L, Ns, t); break;
            case 12: stockham_pass<12, INV>(src, dst, plan.L, Ns, t); break;
            case 15: stockham_pass<15, INV>(src, dst, plan.L, Ns, t); break;
            case 16: stockham_pass<16, INV>(src, dst, plan.L, Ns, t); break;
            case 20: stockham_pass<20, INV>(src, dst, plan.L, Ns, t); break;
            default: stockham_pass<25, INV>(src, dst, plan.L, Ns, t); break;
        }
        __syncthreads();
        C* tmp = src; src = dst; dst = tmp;
    }
    return src;
}

// Pass twiddles: for pass p, tw[twoff[p] + k] = e^{-2 pi i k / (Ns R)}, k < Ns.
template <typename C>
__global__ void pass_twiddles_kernel(C* tw, FftPlan plan) {
    for (int p = 0; p < plan.npass; ++p) {
        const int Ns = plan.ns[p], R = plan.radix[p];
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += gridDim.x * blockDim.x) {
            double s, c;
            sincospi(-2.0 * (double)k / (double)((long long)Ns * R), &s, &c);
            tw[plan.twoff[p] + k] = mkc((decltype(tw[0].x))c, (decltype(tw[0].x))s);
        }
    }
}

// Two real rows of unit u as one complex transform z = a + i b, then
// A_k = (Z_k + conj Z_{L-k}) / 2, B_k = (Z_k - conj Z_{L-k}) / 2i.  Input rows
// are TIN (float, or double for the FP64 path); with U.in2 set (float
// inputs) a row is in + in2 (the compensated hi + lo pair).
template <typename S, typename TIN>
__global__ void __launch_bounds__(kRowThreads, sizeof(S) == 4 ? 2 : 1)
fwd_rows_kernel(FftPlan plan, const cplx<S>* __restrict__ tw, const __grid_constant__ RowUnits U, int ncols,
                int64_t in_stride, int64_t out_stride, int nfreq, float scale, int vec4) {
    using C = cplx<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int L = plan.L;
    C* a = smem;
    C* b = smem + ((L + 1) & ~1);  // both buffers 16-byte aligned
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.x);
    const TIN* __restrict__ in = static_cast<const TIN*>(U.in[u]);
    const float* __restrict__ in2 = static_cast<const float*>(U.in2[u]);
    C* __restrict__ out = static_cast<C*>(U.out[u]);
    const int nrows = U.nrows[u];
    const int r0 = 2 * ((int)blockIdx.x - U.prefix[u]);
    const bool has_b = r0 + 1 < nrows;
    const TIN* pa = in + (int64_t)r0 * in_stride;
    const TIN* pb = has_b ? pa + in_stride : pa;
    const int nload = ncols < L ? ncols : L;
    if (std::is_same<S, float>::value && std::is_same<TIN, float>::value && vec4 && !in2) {
        // rows are 16-byte aligned and nload % 4 == 0
        const float4* qa = reinterpret_cast<const float4*>(pa);
        const float4* qb = reinterpret_cast<const float4*>(pb);
        float4* a4 = reinterpret_cast<float4*>(a);
        for (int n4 = threadIdx.x; n4 < nload / 4; n4 += kRowThreads) {
            const float4 xa = __ldg(qa + n4);
            float4 xb = __ldg(qb + n4);
            if (!has_b) xb = make_float4(0.f, 0.f, 0.f, 0.f);
            a4[2 * n4] = make_float4(xa.x, xb.x, xa.y, xb.y);
            a4[2 * n4 + 1] = make_float4(xa.z, xb.z, xa.w, xb.w);
        }
        for (int n = nload + threadIdx.x; n < L; n += kRowThreads) a[n] = mkc((S)0, (S)0);
    } else {
        const float* la = in2 ? in2 + (int64_t)r0 * in_stride : nullptr;
        const float* lb = (in2 && has_b) ? la + in_stride : la;
        for (int n = threadIdx.x; n < L; n += kRowThreads) {
            S xa = 0, xb = 0;
            if (n < nload) {
                xa = (S)pa[n];
                if (has_b) xb = (S)pb[n];
                if (in2) {
                    xa += (S)la[n];
                    if (has_b) xb += (S)lb[n];
                }
            }
            a[n] = mkc(xa, xb);
        }
    }
    __syncthreads();
    const C* z = fft_smem<false>(plan, a, b, tw);
    C* oa = out + (int64_t)r0 * out_stride;
    C* ob = oa + out_stride;
    const S h = (S)0.5 * (S)scale;
    for (int k = threadIdx.x; k < nfreq; k += kRowThreads) {
        const C zk = z[k];
        const C zm = z[k == 0 ? 0 : L - k];
        oa[k] = mkc(h * (zk.x + zm.x), h * (zk.y - zm.y));
        if (has_b) ob[k] = mkc(h * (zk.y + zm.y), h * (zm.x - zk.x));
    }
}

// Two half spectra A (row r0) and B (row r0+1) -> Z = A + iB over the full
// Hermitian extension, inverse transform, real part row r0, imaginary r0+1,
// stored as float.
template <typename S>
__global__ void __launch_bounds__(kRowThreads, sizeof(S) == 4 ? 2 : 1)
inv_rows_kernel(FftPlan plan, const cplx<S>* __restrict__ tw, const __grid_constant__ RowUnits U,
                int64_t in_stride, int nfreq, int ncols, int64_t out_stride, int vec4) {
    using C = cplx<S>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int L = plan.L;
    C* a = smem;
    C* b = smem + ((L + 1) & ~1);  // both buffers 16-byte aligned
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.x);
    const C* __restrict__ in = static_cast<const C*>(U.in[u]);
    float* __restrict__ out = static_cast<float*>(U.out[u]);
    const int nrows = U.nrows[u];
    const int r0 = 2 * ((int)blockIdx.x - U.prefix[u]);
    const bool has_b = r0 + 1 < nrows;
    const C* ya = in + (int64_t)r0 * in_stride;
    const C* yb = has_b ? ya + in_stride : ya;
    const bool even = (L & 1) == 0;
    for (int k = threadIdx.x; k < L; k += kRowThreads) {
        const bool upper = k >= nfreq;
        const int kk = upper ? L - k : k;
        C A = ya[kk];
        C B = has_b ? yb[kk] : mkc((S)0, (S)0);
        if (kk == 0 || (even && 2 * kk == L)) { A.y = 0; B.y = 0; }
        if (upper) { A.y = -A.y; B.y = -B.y; }
        a[k] = mkc(A.x - B.y, A.y + B.x);
    }
    __syncthreads();
    const C* z = fft_smem<true>(plan, a, b, tw);
    float* oa = out + (int64_t)r0 * out_stride;
    float* ob = oa + out_stride;
    const int nst = ncols < L ? ncols : L;
    if (std::is_same<S, float>::value && vec4) {
        const float4* z4 = reinterpret_cast<const float4*>(z);
        for (int n4 = threadIdx.x; n4 < nst / 4; n4 += kRowThreads) {
            const float4 u4 = z4[2 * n4], w4 = z4[2 * n4 + 1];
            reinterpret_cast<float4*>(oa)[n4] = make_float4(u4.x, u4.z, w4.x, w4.z);
            if (has_b) reinterpret_cast<float4*>(ob)[n4] = make_float4(u4.y, u4.w, w4.y, w4.w);
        }
    } else {
        for (int n = threadIdx.x; n < nst; n += kRowThreads) {
            const C v = z[n];
            oa[n] = (float)v.x;
            if (has_b) ob[n] = (float)v.y;
        }
    }
}

// ------------------------------------------- row transforms of fixed shape
// For the common transform lengths the radix sequence, L and every pass's
// Ns are template constants: index arithmetic folds, each kernel holds only
// its own passes (the generic kernels above carry all thirteen radices and
// their code outgrows the instruction cache when edge passes are fused), and
// the edge passes are fused with the row I/O:
//   forward: pass 0 reads the two input rows (fetched into shared memory by
//            bulk copies when the launch has a status word, else loaded by
//            every thread); the last pass pairs butterflies j and Ns - j so
//            that each thread holds Z_k and Z_{L-k} and writes the split
//            spectra A_k, B_k to global memory;
//   inverse: pass 0 reads the Hermitian extension of both half spectra
//            (fetched the same way); the last pass stores the real and
//            imaginary rows.
template <int NT, int... Rs>
struct Shape {
    static constexpr int threads = NT;
    static constexpr int npass = sizeof...(Rs);
    static constexpr int radix[npass] = {Rs...};
    static constexpr int L = (Rs * ...);
    static constexpr int ns(int p) {
        int n = 1;
        for (int i = 0; i < p; ++i) n *= radix[i];
        return n;
    }
    // one middle pass whose butterflies fit one per thread runs in place
    // (inputs held in registers across a barrier): one shared buffer
    static constexpr bool inplace = npass == 3 && L / radix[npass == 3 ? 1 : 0] <= NT;
    static constexpr int buffers = inplace ? 1 : 2;
    // CTAs per SM: one 50 KB buffer lets four 256-thread CTAs share an SM
    // (64 registers each; the inverse measured faster so, the forward at 320
    // threads keeps three)
    static constexpr int ctas = inplace ? (NT <= 256 ? 4 : 3) : 2;
    // A half spectrum rounded up to 16 bytes, and a buffer that holds either
    // L complex values or two such half spectra (the rows fetched by bulk
    // copies before the first pass).
    static constexpr int nfe = ((L / 2 + 1) + 1) & ~1;
    static constexpr int buf = ((L + 1) & ~1) > 2 * nfe ? ((L + 1) & ~1) : 2 * nfe;
    // the first pass has one butterfly per thread, so it can read its inputs
    // from the buffer it then overwrites
    static constexpr bool first_inplace = L / radix[0] <= NT;
};

template <int R, bool INV, typename C>
__device__ __forceinline__ void twiddle_inputs(C* v, C w) {
    C wp[R];
    wp[1] = w;
    if (INV) wp[1].y = -wp[1].y;
#pragma unroll
    for (int r = 2; r < R; ++r) wp[r] = cmul_tw<false>(wp[r / 2], wp[r - r / 2]);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul_tw<false>(v[r], wp[r]);
}

// One Stockham pass (same butterfly as stockham_pass) reading ld(i) and
// writing st(i, value).
template <int R, int Ns, int L, int NT, bool INV, typename C, typename Ld, typename St>
__device__ __forceinline__ void io_pass(const C* __restrict__ tw, Ld ld, St st) {
    constexpr int nb = L / R;
#pragma unroll 1
    for (int j = threadIdx.x; j < nb; j += NT) {
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * nb);
        if (Ns > 1) twiddle_inputs<R, INV>(v, tw[k]);
        Dft<R, INV, C>::run(v);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) st(d + r * Ns, v[r]);
    }
}

// Last forward pass (Ns R = L: butterfly j yields Z[j + r Ns]).  Z[L - k]
// for k = j + r Ns is output R-1-r of butterfly Ns - j, or output (R-r) mod R
// of butterfly 0 when j = 0; out(k, Z_k, Z_{L-k}) for every k < nfreq.
template <int R, int Ns, int L, int NT, typename C, typename Ld, typename Out>
__device__ __forceinline__ void fwd_last_pass(const C* __restrict__ tw, Ld ld, int nfreq, Out out) {
    static_assert(Ns * R == L, "last pass");
    constexpr int ntask = Ns / 2 + 1;
#pragma unroll 1
    for (int j = threadIdx.x; j < ntask; j += NT) {
        const int jm = Ns - j;
        const bool two = j > 0 && jm != j;
        C v[R], w[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * Ns);
        if (Ns > 1) twiddle_inputs<R, false>(v, tw[j]);
        Dft<R, false, C>::run(v);
        if (two) {
#pragma unroll
            for (int r = 0; r < R; ++r) w[r] = ld(jm + r * Ns);
            twiddle_inputs<R, false>(w, tw[jm]);
            Dft<R, false, C>::run(w);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = j + r * Ns;
            if (k < nfreq) out(k, v[r], j == 0 ? v[(R - r) % R] : (two ? w[R - 1 - r] : v[R - 1 - r]));
        }
        if (two) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = jm + r * Ns;
                if (k < nfreq) out(k, w[r], v[R - 1 - r]);
            }
        }
    }
}

// Passes 1 .. npass-2 of shape SH in shared memory, pass p reading buf[(p-1)&1]
// and writing buf[p&1].
template <typename SH, bool INV, typename C>
__device__ __forceinline__ void shape_middle(const FftPlan& plan, C* buf0, C* buf1, const C* __restrict__ tw) {
    if constexpr (SH::inplace) {
        constexpr int R = SH::radix[1], Ns = SH::ns(1), nb = SH::L / R;
        const int j = threadIdx.x;
        const int k = j % Ns;
        C v[R];
        if (j < nb) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = buf0[j + r * nb];
            if (Ns > 1) twiddle_inputs<R, INV>(v, tw[plan.twoff[1] + k]);
            Dft<R, INV, C>::run(v);
        }
        __syncthreads();   // every input read before any output lands
        if (j < nb) {
            const int d = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf0[d + r * Ns] = v[r];
        }
        __syncthreads();
        return;
    }
    sfor<SH::npass>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        if constexpr (p > 0 && p + 1 < SH::npass) {
            constexpr int R = SH::radix[p], Ns = SH::ns(p);
            C* src = (p - 1) & 1 ? buf1 : buf0;
            C* dst = p & 1 ? buf1 : buf0;
            io_pass<R, Ns, SH::L, SH::threads, INV>(tw + plan.twoff[p], [&](int i) { return src[i]; },
                                       [&](int i, C v) { dst[i] = v; });
            __syncthreads();
        }
    });
}

// First pass with Ns = 1 (no twiddles) from inputs in shared memory into the
// same buffer: one butterfly per thread reads its R inputs into registers,
// every thread passes a barrier, then the outputs land at j R + r.
template <typename SH, bool INV, typename Ld>
__device__ __forceinline__ void first_pass_inplace(float2* buf, Ld ld) {
    constexpr int R = SH::radix[0], nb = SH::L / R;
    static_assert(SH::first_inplace, "one butterfly per thread");
    const int j = threadIdx.x;
    float2 v[R];
    if (j < nb) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * nb);
    }
    __syncthreads();   // every input read before any output lands
    if (j < nb) {
        Dft<R, INV, float2>::run(v);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[j * R + r] = v[r];
    }
    __syncthreads();
}

// Fetch `bytes0` from src0 (and bytes1 from src1 if non-null) into shared
// memory with bulk copies on one mbarrier; false (after flagging
// WS_DEV_TIMEOUT and letting a late copy drain) if they never land.
__device__ __forceinline__ bool bulk_fetch_rows(void* dst0, const void* src0, uint32_t bytes0, void* dst1,
                                                const void* src1, uint32_t bytes1, uint64_t* bar, uint32_t* status) {
    if (threadIdx.x == 0) {
        mbar_init(bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_expect(bar, bytes0 + (src1 ? bytes1 : 0u));
        bulk_load(dst0, src0, bytes0, bar);
        if (src1) bulk_load(dst1, src1, bytes1, bar);
    }
    const bool ok = mbar_wait(bar, 0u);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(status, WS_DEV_TIMEOUT);
        mbar_wait(bar, 0u);
        return false;
    }
    return true;
}

template <typename SH, bool BULK>
__global__ void __launch_bounds__(SH::threads, SH::ctas)
fwd_rows_shape_kernel(FftPlan plan, const float2* __restrict__ tw, const __grid_constant__ RowUnits U, int ncols,
                      int64_t in_stride, int64_t out_stride, int nfreq, float scale) {
    using C = float2;
    constexpr int L = SH::L, last = SH::npass - 1;
    static_assert(SH::npass >= 2, "edge passes");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + SH::buf;
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.x);
    const float* __restrict__ in = static_cast<const float*>(U.in[u]);
    const float* __restrict__ in2 = static_cast<const float*>(U.in2[u]);
    const int r0 = 2 * ((int)blockIdx.x - U.prefix[u]);
    const bool has_b = r0 + 1 < U.nrows[u];
    C* oa = static_cast<C*>(U.out[u]) + (int64_t)r0 * out_stride;
    C* ob = oa + out_stride;
    // active rows: an unmarked row of S is zero (and was not cleared, so it
    // is not read); a pair with no marked row has zero spectra, written only
    // if a live row's wire convolution may read them
    bool use_a = true, use_b = has_b;
    if (const uint32_t* cls = U.rows[u]) {
        const int dv = U.rdiv[u];
        const uint32_t ca = cls[r0 / dv], cb = has_b ? cls[(r0 + 1) / dv] : 0u;
        use_a = (ca & ROW_MARKED) != 0u;
        use_b = (cb & ROW_MARKED) != 0u;
        if (!use_a && !use_b) {
            if ((ca | cb) & ROW_NEEDED) {
                for (int k = threadIdx.x; k < nfreq; k += SH::threads) {
                    oa[k] = make_float2(0.f, 0.f);
                    if (has_b) ob[k] = make_float2(0.f, 0.f);
                }
            }
            return;
        }
    }
    const float* __restrict__ pa = in + (int64_t)r0 * in_stride;
    const float* __restrict__ pb = has_b ? pa + in_stride : pa;
    const float* __restrict__ la = in2 ? in2 + (int64_t)r0 * in_stride : nullptr;
    const float* __restrict__ lb = (in2 && has_b) ? la + in_stride : la;
    const int nload = ncols < L ? ncols : L;
    if constexpr (BULK) {
        // the pair's rows in use (nload floats each, a multiple of 4) by bulk copies
        __shared__ __align__(8) uint64_t bar;
        float* sa = reinterpret_cast<float*>(buf0);
        float* sb = sa + nload;
        const uint32_t bytes = (uint32_t)nload * 4u;
        const bool ok = use_a ? bulk_fetch_rows(sa, pa, bytes, sb, use_b ? pb : nullptr, bytes, &bar, U.status)
                              : bulk_fetch_rows(sb, pb, bytes, nullptr, nullptr, 0u, &bar, U.status);
        if (!ok) return;
        first_pass_inplace<SH, false>(buf0, [&](int n) {
            return n < nload ? make_float2(use_a ? sa[n] : 0.f, use_b ? sb[n] : 0.f) : make_float2(0.f, 0.f);
        });
    } else {
        io_pass<SH::radix[0], 1, L, SH::threads, false>(tw, [&](int n) {
            float xa = 0.f, xb = 0.f;
            if (n < nload) {
                if (use_a) xa = __ldg(pa + n);
                if (use_b) xb = __ldg(pb + n);
                if (in2) {
                    if (use_a) xa += __ldg(la + n);
                    if (use_b) xb += __ldg(lb + n);
                }
            }
            return make_float2(xa, xb);
        }, [&](int i, C v) { buf0[i] = v; });
        __syncthreads();
    }
    shape_middle<SH, false>(plan, buf0, buf1, tw);
    const C* z = (!SH::inplace && ((last - 1) & 1)) ? buf1 : buf0;
    const float h = 0.5f * scale;
    fwd_last_pass<SH::radix[last], SH::ns(last), L, SH::threads>(tw + plan.twoff[last], [&](int i) { return z[i]; }, nfreq,
                                                    [&](int k, C zk, C zm) {
        oa[k] = make_float2(h * (zk.x + zm.x), h * (zk.y - zm.y));
        if (has_b) ob[k] = make_float2(h * (zk.y + zm.y), h * (zm.x - zk.x));
    });
}

template <typename SH, bool BULK>
__global__ void __launch_bounds__(SH::threads, SH::ctas)
inv_rows_shape_kernel(FftPlan plan, const float2* __restrict__ tw, const __grid_constant__ RowUnits U,
                      int64_t in_stride, int nfreq, int ncols, int64_t out_stride) {
    using C = float2;
    constexpr int L = SH::L, last = SH::npass - 1;
    static_assert(SH::npass >= 2, "edge passes");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + SH::buf;
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.x);
    const int r0 = 2 * ((int)blockIdx.x - U.prefix[u]);
    const bool has_b = r0 + 1 < U.nrows[u];
    float* oa = static_cast<float*>(U.out[u]) + (int64_t)r0 * out_stride;
    float* ob = oa + out_stride;
    const int nst = ncols < L ? ncols : L;
    // active rows: a row whose wire-convolution window holds no marked row
    // is zero (its spectrum, possibly never written, is not read); a pair of
    // such rows is stored as zeros without a transform
    bool live_a = true, live_b = has_b;
    if (const uint32_t* cls = U.rows[u]) {
        live_a = (cls[r0] & ROW_LIVE) != 0u;
        live_b = has_b && (cls[r0 + 1] & ROW_LIVE) != 0u;
        if (!live_a && !live_b) {
            for (int n = threadIdx.x; n < nst; n += SH::threads) {
                oa[n] = 0.f;
                if (has_b) ob[n] = 0.f;
            }
            return;
        }
    }
    const C* __restrict__ ya = static_cast<const C*>(U.in[u]) + (int64_t)r0 * in_stride;
    const C* __restrict__ yb = has_b ? ya + in_stride : ya;
    // Z = A + iB over the Hermitian extension of both half spectra (global
    // spectra through the read-only path, or their copies in shared memory)
    auto hermitian = [&](const C* a, const C* b, int k) {
        const bool upper = k >= nfreq;
        const int kk = upper ? L - k : k;
        C A = live_a ? (BULK ? a[kk] : __ldg(a + kk)) : make_float2(0.f, 0.f);
        C B = live_b ? (BULK ? b[kk] : __ldg(b + kk)) : make_float2(0.f, 0.f);
        if (kk == 0 || (L % 2 == 0 && 2 * kk == L)) { A.y = 0.f; B.y = 0.f; }
        if (upper) { A.y = -A.y; B.y = -B.y; }
        return make_float2(A.x - B.y, A.y + B.x);
    };
    if constexpr (BULK) {
        // the live half spectra (nfreq <= SH::nfe values each) by bulk copies
        __shared__ __align__(8) uint64_t bar;
        C* sA = buf0;
        C* sB = buf0 + SH::nfe;
        const uint32_t bytes = (uint32_t)SH::nfe * (uint32_t)sizeof(C);
        const bool ok = live_a ? bulk_fetch_rows(sA, ya, bytes, sB, live_b ? yb : nullptr, bytes, &bar, U.status)
                               : bulk_fetch_rows(sB, yb, bytes, nullptr, nullptr, 0u, &bar, U.status);
        if (!ok) return;
        first_pass_inplace<SH, true>(buf0, [&](int k) { return hermitian(sA, sB, k); });
    } else {
        io_pass<SH::radix[0], 1, L, SH::threads, true>(tw, [&](int k) { return hermitian(ya, yb, k); },
                                                     [&](int i, C v) { buf0[i] = v; });
        __syncthreads();
    }
    shape_middle<SH, true>(plan, buf0, buf1, tw);
    const C* z = (!SH::inplace && ((last - 1) & 1)) ? buf1 : buf0;
    io_pass<SH::radix[last], SH::ns(last), L, SH::threads, true>(tw + plan.twoff[last], [&](int i) { return z[i]; },
                                                    [&](int n, C v) {
        if (n < nst) {
            oa[n] = v.x;
            if (has_b) ob[n] = v.y;
        }
    });
}

// Register-blocked wire convolution in the tick-frequency domain.  A CTA
// owns 128 frequency columns x B output wires; it stages the B + K - 1 input
// rows those outputs need in shared memory with 16-byte loads (zeros outside
// the grid in linear mode, wrapped rows in circular mode), then each thread
// keeps its column's K taps and B accumulators in registers.
constexpr int kConvCols = 128;

// KARATSUBA: with r = c + i d (tap) and x = a + i b (input), r x =
// [c (a + b) - b (c + d)] + i [c (a + b) + a (d - c)]: three real products
// per tap into three accumulators instead of four.
template <int K, int B, bool KARATSUBA, typename S>
__global__ void __launch_bounds__(kConvCols)
wire_conv_kernel(const __grid_constant__ ConvUnits U, int nfreq, int64_t stride, int kw, int center, int circular) {
    using C = cplx<S>;
    constexpr int ROWS = B + K - 1;
    __shared__ __align__(16) C tile[ROWS][kConvCols];
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.y);
    const C* __restrict__ X = static_cast<const C*>(U.X[u]);
    C* __restrict__ Y = static_cast<C*>(U.Y[u]);
    const C* __restrict__ Rt = static_cast<const C*>(U.Rt[u]);
    const int nwires = U.nwires[u];
    const int k0 = blockIdx.x * kConvCols;
    const int w0 = ((int)blockIdx.y - U.prefix[u]) * B;
    const int ibase = w0 + center - (K - 1);
    // active rows: a tile none of whose output rows is live is never read
    if (const mark_t* marks = U.rows[u])
        if (!cta_any_marked(marks, read_epoch(U.epoch), w0 + center - kw + 1, w0 + B - 1 + center, nwires)) return;
    constexpr int PER = std::is_same<S, float>::value ? 2 : 1;   // complex values per 16-byte load
    for (int e = threadIdx.x; e < ROWS * (kConvCols / PER); e += kConvCols) {
        const int uu = e / (kConvCols / PER), c2 = e - uu * (kConvCols / PER);
        int i = ibase + uu;
        const int kk = k0 + PER * c2;
        bool ok = kk < stride;
        if (circular) {
            i %= nwires;
            if (i < 0) i += nwires;
        } else {
            ok = ok && i >= 0 && i < nwires;
        }
        if constexpr (PER == 2) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) v = __ldg(reinterpret_cast<const float4*>(X + (int64_t)i * stride + kk));
            reinterpret_cast<float4*>(&tile[uu][0])[c2] = v;
        } else {
            C v = mkc((S)0, (S)0);
            if (ok) v = X[(int64_t)i * stride + kk];
            tile[uu][c2] = v;
        }
    }
    __syncthreads();
    const int k = k0 + threadIdx.x;
    if (k >= nfreq) return;
    if constexpr (KARATSUBA) {
        S cc[K], cm[K], cp[K];   // c, d - c, c + d
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const C t = r < kw ? Rt[(int64_t)r * stride + k] : mkc((S)0, (S)0);
            cc[r] = t.x;
            cm[r] = t.y - t.x;
            cp[r] = t.x + t.y;
        }
        S k1[B], k2[B], k3[B];
#pragma unroll
        for (int b = 0; b < B; ++b) k1[b] = k2[b] = k3[b] = 0;
#pragma unroll
        for (int uu = 0; uu < ROWS; ++uu) {
            const C x = tile[uu][threadIdx.x];
            const S sab = x.x + x.y;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int r = b + K - 1 - uu;
                if (r >= 0 && r < K) {
                    k1[b] = fmx(cc[r], sab, k1[b]);
                    k2[b] = fmx(cm[r], x.x, k2[b]);
                    k3[b] = fmx(cp[r], x.y, k3[b]);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (w0 + b < nwires) Y[(int64_t)(w0 + b) * stride + k] = mkc(k1[b] - k3[b], k1[b] + k2[b]);
    } else {
        C c[K];
#pragma unroll
        for (int r = 0; r < K; ++r) c[r] = r < kw ? Rt[(int64_t)r * stride + k] : mkc((S)0, (S)0);
        C acc[B];
#pragma unroll
        for (int b = 0; b < B; ++b) acc[b] = mkc((S)0, (S)0);
#pragma unroll
        for (int uu = 0; uu < ROWS; ++uu) {
            const C x = tile[uu][threadIdx.x];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int r = b + K - 1 - uu;
                if (r >= 0 && r < K) {
                    acc[b].x = fmx(c[r].x, x.x, fmx(-c[r].y, x.y, acc[b].x));
                    acc[b].y = fmx(c[r].x, x.y, fmx(c[r].y, x.x, acc[b].y));
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (w0 + b < nwires) Y[(int64_t)(w0 + b) * stride + k] = acc[b];
    }
}

// Wire convolution over sub-pitch impact positions: a CTA owns 128 columns
// x B output wires; for each impact i it stages the B + K - 1 input wires'
// rows of that impact (fine rows wire * impacts + i) in shared memory and
// adds that impact's K-tap sum (Karatsuba taps in registers) into the same
// accumulators.
template <int K, int B>
__global__ void __launch_bounds__(kConvCols)
wire_conv_impacts_kernel(const float2* __restrict__ X, float2* __restrict__ Y, const float2* __restrict__ Rt,
                         int nwires, int impacts, int nfreq, int64_t stride, int kw, int center, int circular) {
    constexpr int ROWS = B + K - 1;
    __shared__ __align__(16) float2 tile[ROWS][kConvCols];
    const int k0 = blockIdx.x * kConvCols;
    const int w0 = blockIdx.y * B;
    const int ibase = w0 + center - (K - 1);
    const int k = k0 + threadIdx.x;
    float k1[B], k2[B], k3[B];
#pragma unroll
    for (int b = 0; b < B; ++b) k1[b] = k2[b] = k3[b] = 0.f;
    for (int im = 0; im < impacts; ++im) {
        __syncthreads();   // the previous impact's tile is read
        for (int e = threadIdx.x; e < ROWS * (kConvCols / 2); e += kConvCols) {
            const int uu = e / (kConvCols / 2), c2 = e - uu * (kConvCols / 2);
            int wi = ibase + uu;
            const int kk = k0 + 2 * c2;
            bool ok = kk < stride;
            if (circular) {
                wi %= nwires;
                if (wi < 0) wi += nwires;
            } else {
                ok = ok && wi >= 0 && wi < nwires;
            }
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) v = __ldg(reinterpret_cast<const float4*>(X + ((int64_t)wi * impacts + im) * stride + kk));
            reinterpret_cast<float4*>(&tile[uu][0])[c2] = v;
        }
        __syncthreads();
        if (k < nfreq) {
            float cc[K], cm[K], cp[K];
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const float2 t = r < kw ? __ldg(&Rt[((int64_t)im * kw + r) * stride + k]) : make_float2(0.f, 0.f);
                cc[r] = t.x;
                cm[r] = t.y - t.x;
                cp[r] = t.x + t.y;
            }
#pragma unroll
            for (int uu = 0; uu < ROWS; ++uu) {
                const float2 x = tile[uu][threadIdx.x];
                const float sab = x.x + x.y;
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int r = b + K - 1 - uu;
                    if (r >= 0 && r < K) {
                        k1[b] = fmaf(cc[r], sab, k1[b]);
                        k2[b] = fmaf(cm[r], x.x, k2[b]);
                        k3[b] = fmaf(cp[r], x.y, k3[b]);
                    }
                }
            }
        }
    }
    if (k >= nfreq) return;
#pragma unroll
    for (int b = 0; b < B; ++b)
        if (w0 + b < nwires) Y[(int64_t)(w0 + b) * stride + k] = make_float2(k1[b] - k3[b], k1[b] + k2[b]);
}

template <int B, bool KS, typename S>
void launch_wc(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, int circular, cudaStream_t s) {
    constexpr int K = kMaxRespWires;
    ConvUnits U;
    U.n = cb.n;
    U.prefix[0] = 0;
    for (int i = 0; i < cb.n; ++i) {
        U.X[i] = cb.X[i];
        U.Y[i] = cb.Y[i];
        U.Rt[i] = cb.Rt[i];
        U.nwires[i] = cb.nwires[i];
        U.rows[i] = std::is_same<S, float>::value ? cb.rows[i] : nullptr;
        U.prefix[i + 1] = U.prefix[i] + (cb.nwires[i] + B - 1) / B;
    }
    U.epoch = cb.epoch;
    dim3 grid((nfreq + kConvCols - 1) / kConvCols, U.prefix[cb.n]);
    wire_conv_kernel<K, B, KS, S><<<grid, kConvCols, 0, s>>>(U, nfreq, stride, kw, center, circular);
}

// Adjoint coefficients: the wire correlation sum_r conj(Rt[r]) X[w + r - c]
// is the wire convolution with taps A[kw-1-r] = conj(Rt[r]) and centre
// kw-1-c.
__global__ void adj_coeffs_kernel(const float2* __restrict__ Rt, float2* __restrict__ A, int kw, int64_t stride,
                                  int nfreq) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)kw * nfreq;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / nfreq), k = (int)(e - (int64_t)r * nfreq);
        const float2 v = Rt[(int64_t)r * stride + k];
        A[(int64_t)(kw - 1 - r) * stride + k] = make_float2(v.x, -v.y);
    }
}

// Response-gradient spectra: A[r][k] += scale * sum_w conj(XS[w - (r - c)][k])
// XG[w][k] over this block's chunk of wires (XS zero outside the grid, or
// wrapped), accumulated into A with atomics.  Each thread walks its column
// down the chunk keeping the K rows of XS that the current wire needs in a
// register window (row w + c - K + 1 + j in slot (step + j) mod K), so every
// element of XS and XG is read once per chunk.
constexpr int kRespGradRows = 32;
constexpr int kRespGradThreads = 64;

__global__ void __launch_bounds__(kRespGradThreads)
resp_grad_kernel(const float2* __restrict__ XG, const float2* __restrict__ XS, float2* __restrict__ A, int nwires,
                 int nfreq, int64_t stride, int kw, int center, int circular, float scale) {
    constexpr int K = kMaxRespWires;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nfreq) return;
    const int w0 = blockIdx.y * kRespGradRows;
    const int w1 = min(nwires, w0 + kRespGradRows);
    auto xs_row = [&](int row) -> float2 {
        if (circular) {
            row %= nwires;
            if (row < 0) row += nwires;
        } else if (row < 0 || row >= nwires) {
            return make_float2(0.f, 0.f);
        }
        return __ldg(&XS[(int64_t)row * stride + k]);
    };
    float2 win[K];
    float2 acc[K];
#pragma unroll
    for (int r = 0; r < K; ++r) acc[r] = make_float2(0.f, 0.f);
    // window of the first wire: rows w0 + c - K + 1 + j, j = 0 .. K - 2 (row
    // j = K - 1 is loaded by the first step)
#pragma unroll
    for (int j = 0; j < K - 1; ++j) win[j] = xs_row(w0 + center - K + 1 + j);
    for (int wb = w0; wb < w1; wb += K) {
#pragma unroll
        for (int jj = 0; jj < K; ++jj) {
            const int w = wb + jj;
            if (w < w1) {
                win[(jj + K - 1) % K] = xs_row(w + center);
                const float2 xg = __ldg(&XG[(int64_t)w * stride + k]);
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    // XS row w - (r - c) = w + c - K + 1 + j with j = K - 1 - r
                    const float2 xs = win[(jj + K - 1 - r) % K];
                    acc[r].x = fmaf(xs.x, xg.x, fmaf(xs.y, xg.y, acc[r].x));
                    acc[r].y = fmaf(xs.x, xg.y, fmaf(-xs.y, xg.x, acc[r].y));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        if (r >= kw) break;
        atomicAdd(&A[(int64_t)r * stride + k].x, scale * acc[r].x);
        atomicAdd(&A[(int64_t)r * stride + k].y, scale * acc[r].y);
    }
}

}  // namespace

cudaError_t launch_adj_coeffs(const float2* Rt, float2* A, int kw, int64_t stride, int nfreq, cudaStream_t s) {
    adj_coeffs_kernel<<<(kw * nfreq + 255) / 256, 256, 0, s>>>(Rt, A, kw, stride, nfreq);
    return cudaGetLastError();
}

cudaError_t launch_resp_grad(const float2* XG, const float2* XS, float2* A, int nwires, int nfreq, int64_t stride,
                             int kw, int center, int circular, float scale, cudaStream_t s) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    dim3 grid((nfreq + kRespGradThreads - 1) / kRespGradThreads, (nwires + kRespGradRows - 1) / kRespGradRows);
    resp_grad_kernel<<<grid, kRespGradThreads, 0, s>>>(XG, XS, A, nwires, nfreq, stride, kw, center, circular, scale);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(float2* tw, const FftPlan& plan, cudaStream_t s) {
    pass_twiddles_kernel<float2><<<(plan.L + 255) / 256, 256, 0, s>>>(tw, plan);
    return cudaGetLastError();
}

cudaError_t launch_twiddles64(double2* tw, const FftPlan& plan, cudaStream_t s) {
    pass_twiddles_kernel<double2><<<(plan.L + 255) / 256, 256, 0, s>>>(tw, plan);
    return cudaGetLastError();
}

static cudaError_t set_smem(const void* fn, int bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

static RowUnits row_units(const RowBatch& rb, bool* aligned16) {
    RowUnits U;
    U.n = rb.n;
    U.prefix[0] = 0;
    U.status = rb.status;
    *aligned16 = true;
    for (int i = 0; i < rb.n; ++i) {
        U.in[i] = rb.in[i];
        U.in2[i] = rb.in2[i];
        U.out[i] = rb.out[i];
        U.nrows[i] = rb.nrows[i];
        U.rows[i] = rb.rows[i];
        U.rdiv[i] = rb.rdiv[i] > 1 ? rb.rdiv[i] : 1;
        U.prefix[i + 1] = U.prefix[i] + (rb.nrows[i] + 1) / 2;
        *aligned16 = *aligned16 && ((uintptr_t)rb.in[i] % 16 == 0) && ((uintptr_t)rb.out[i] % 16 == 0);
    }
    return U;
}

// Fixed-shape kernels for the FP32 transforms (greedy radix plans of the
// lengths below); other plans run the generic kernels.
using FwdShapeFn = void (*)(FftPlan, const float2*, const RowUnits, int, int64_t, int64_t, int, float);
using InvShapeFn = void (*)(FftPlan, const float2*, const RowUnits, int64_t, int, int, int64_t);
struct ShapeKernels {
    int npass;
    int radix[4];
    FwdShapeFn fwd, fwd_bulk;    // first-pass rows by loads / by bulk copies
    int fwd_threads, fwd_buffers, fwd_buf;
    InvShapeFn inv, inv_bulk;
    int inv_threads, inv_buffers, inv_buf;
};
constexpr int kFwdShapeThreads = 320;
constexpr int kInvShapeThreads = 256;
#define WS_SHAPE3(A, B, C)                                                                                  \
    {3, {A, B, C}, fwd_rows_shape_kernel<Shape<kFwdShapeThreads, A, B, C>, false>,                          \
     fwd_rows_shape_kernel<Shape<kFwdShapeThreads, A, B, C>, true>, kFwdShapeThreads,                       \
     Shape<kFwdShapeThreads, A, B, C>::buffers, Shape<kFwdShapeThreads, A, B, C>::buf,                      \
     inv_rows_shape_kernel<Shape<kInvShapeThreads, A, B, C>, false>,                                         \
     inv_rows_shape_kernel<Shape<kInvShapeThreads, A, B, C>, true>, kInvShapeThreads,                        \
     Shape<kInvShapeThreads, A, B, C>::buffers, Shape<kInvShapeThreads, A, B, C>::buf}
static const ShapeKernels kShapes[] = {
    WS_SHAPE3(25, 25, 10),  // 6250: linear convolution of 6000 ticks with a 200-tick response
    WS_SHAPE3(25, 16, 15),  // 6000: circular convolution of 6000 ticks
    WS_SHAPE3(25, 16, 16),  // 6400
    WS_SHAPE3(25, 16, 8),   // 3200
    WS_SHAPE3(25, 16, 3),   // 1200
};
#undef WS_SHAPE3

static const ShapeKernels* shape_kernels(const FftPlan& plan) {
    for (const ShapeKernels& k : kShapes) {
        bool eq = k.npass == plan.npass;
        for (int p = 0; eq && p < plan.npass; ++p) eq = k.radix[p] == plan.radix[p];
        if (eq) return &k;
    }
    return nullptr;
}

bool row_fft_fixed_shape(const FftPlan& plan) { return shape_kernels(plan) != nullptr; }

template <typename S, typename TIN>
static cudaError_t fwd_rows_t(const FftPlan& plan, const cplx<S>* tw, const RowBatch& rb, int ncols,
                              int64_t in_stride, int64_t out_stride, int nfreq, float scale, cudaStream_t s) {
    if (rb.n <= 0) return cudaSuccess;
    if constexpr (std::is_same<S, float>::value && std::is_same<TIN, float>::value) {
        if (const ShapeKernels* k = shape_kernels(plan)) {
            bool al = false;
            const RowUnits U = row_units(rb, &al);
            if (U.prefix[rb.n] <= 0) return cudaSuccess;
            // bulk copies need 16-byte rows and a status word to report a copy that never lands
            bool bulk = rb.status != nullptr && al && in_stride % 4 == 0 && (ncols < plan.L ? ncols : plan.L) % 4 == 0;
            for (int i = 0; i < rb.n; ++i) bulk = bulk && rb.in2[i] == nullptr;
            const FwdShapeFn fn = bulk ? k->fwd_bulk : k->fwd;
            const int smem = k->fwd_buffers * k->fwd_buf * (int)sizeof(float2);
            cudaError_t e = set_smem((const void*)fn, smem);
            if (e != cudaSuccess) return e;
            fn<<<U.prefix[rb.n], k->fwd_threads, smem, s>>>(plan, tw, U, ncols, in_stride, out_stride, nfreq, scale);
            return cudaGetLastError();
        }
    }
    // active-row marks are honoured by the fixed-shape kernels only
    for (int i = 0; i < rb.n; ++i)
        if (rb.rows[i]) return cudaErrorInvalidValue;
    const int smem = 2 * ((plan.L + 1) & ~1) * (int)sizeof(cplx<S>);
    cudaError_t e = set_smem((const void*)fwd_rows_kernel<S, TIN>, smem);
    if (e != cudaSuccess) return e;
    bool al = false;
    const RowUnits U = row_units(rb, &al);
    if (U.prefix[rb.n] <= 0) return cudaSuccess;
    const int nload = ncols < plan.L ? ncols : plan.L;
    const int vec4 = al && (in_stride % 4 == 0) && (nload % 4 == 0);
    fwd_rows_kernel<S, TIN><<<U.prefix[rb.n], kRowThreads, smem, s>>>(plan, tw, U, ncols, in_stride, out_stride,
                                                                      nfreq, scale, vec4);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t inv_rows_t(const FftPlan& plan, const cplx<S>* tw, const RowBatch& rb, int64_t in_stride,
                              int nfreq, int ncols, int64_t out_stride, cudaStream_t s) {
    if (rb.n <= 0) return cudaSuccess;
    if constexpr (std::is_same<S, float>::value) {
        if (const ShapeKernels* k = shape_kernels(plan)) {
            bool al = true;
            const RowUnits U = row_units(rb, &al);
            if (U.prefix[rb.n] <= 0) return cudaSuccess;
            bool in16 = in_stride % 2 == 0 && nfreq == plan.L / 2 + 1;
            for (int i = 0; i < rb.n; ++i) in16 = in16 && (uintptr_t)rb.in[i] % 16 == 0;
            const bool bulk = rb.status != nullptr && in16;
            const InvShapeFn fn = bulk ? k->inv_bulk : k->inv;
            const int smem = k->inv_buffers * k->inv_buf * (int)sizeof(float2);
            cudaError_t e = set_smem((const void*)fn, smem);
            if (e != cudaSuccess) return e;
            fn<<<U.prefix[rb.n], k->inv_threads, smem, s>>>(plan, tw, U, in_stride, nfreq, ncols, out_stride);
            return cudaGetLastError();
        }
    }
    for (int i = 0; i < rb.n; ++i)
        if (rb.rows[i]) return cudaErrorInvalidValue;
    const int smem = 2 * ((plan.L + 1) & ~1) * (int)sizeof(cplx<S>);
    cudaError_t e = set_smem((const void*)inv_rows_kernel<S>, smem);
    if (e != cudaSuccess) return e;
    bool al = false;
    const RowUnits U = row_units(rb, &al);
    if (U.prefix[rb.n] <= 0) return cudaSuccess;
    const int nst = ncols < plan.L ? ncols : plan.L;
    const int vec4 = al && (out_stride % 4 == 0) && (nst % 4 == 0);
    inv_rows_kernel<S><<<U.prefix[rb.n], kRowThreads, smem, s>>>(plan, tw, U, in_stride, nfreq, ncols, out_stride,
                                                                 vec4);
    return cudaGetLastError();
}

static RowBatch one_row(const void* in, const void* in2, void* out, int nrows) {
    RowBatch rb;
    rb.n = 1;
    rb.in[0] = in;
    rb.in2[0] = in2;
    rb.out[0] = out;
    rb.nrows[0] = nrows;
    return rb;
}

cudaError_t launch_fwd_rows_batch(const FftPlan& plan, const float2* tw, const RowBatch& rb, int ncols,
                                  int64_t in_stride, int64_t out_stride, int nfreq, float scale, cudaStream_t s) {
    return fwd_rows_t<float, float>(plan, tw, rb, ncols, in_stride, out_stride, nfreq, scale, s);
}

cudaError_t launch_fwd_rows(const FftPlan& plan, const float2* tw, const float* in, int nrows,
                            int ncols, int64_t in_stride, float2* out, int64_t out_stride,
                            int nfreq, float scale, cudaStream_t s, uint32_t* status) {
    if (nrows <= 0) return cudaSuccess;
    RowBatch rb = one_row(in, nullptr, out, nrows);
    rb.status = status;
    return launch_fwd_rows_batch(plan, tw, rb, ncols, in_stride, out_stride, nfreq, scale, s);
}

cudaError_t launch_fwd_rows_comp(const FftPlan& plan, const float2* tw, const float* hi, const float* lo, int nrows,
                                 int ncols, int64_t in_stride, float2* out, int64_t out_stride, int nfreq,
                                 cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    return fwd_rows_t<float, float>(plan, tw, one_row(hi, lo, out, nrows), ncols, in_stride, out_stride, nfreq,
                                    1.0f, s);
}

cudaError_t launch_fwd_rows64(const FftPlan& plan, const double2* tw, const void* in, bool in_double, int nrows,
                              int ncols, int64_t in_stride, double2* out, int64_t out_stride, int nfreq, float scale,
                              cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    const RowBatch rb = one_row(in, nullptr, out, nrows);
    if (in_double) return fwd_rows_t<double, double>(plan, tw, rb, ncols, in_stride, out_stride, nfreq, scale, s);
    return fwd_rows_t<double, float>(plan, tw, rb, ncols, in_stride, out_stride, nfreq, scale, s);
}

cudaError_t launch_inv_rows_batch(const FftPlan& plan, const float2* tw, const RowBatch& rb, int64_t in_stride,
                                  int nfreq, int ncols, int64_t out_stride, cudaStream_t s) {
    return inv_rows_t<float>(plan, tw, rb, in_stride, nfreq, ncols, out_stride, s);
}

cudaError_t launch_inv_rows(const FftPlan& plan, const float2* tw, const float2* in, int nrows,
                            int64_t in_stride, int nfreq, float* out, int ncols,
                            int64_t out_stride, cudaStream_t s, uint32_t* status) {
    if (nrows <= 0) return cudaSuccess;
    RowBatch rb = one_row(in, nullptr, out, nrows);
    rb.status = status;
    return launch_inv_rows_batch(plan, tw, rb, in_stride, nfreq, ncols, out_stride, s);
}

cudaError_t launch_inv_rows64(const FftPlan& plan, const double2* tw, const double2* in, int nrows, int64_t in_stride,
                              int nfreq, float* out, int ncols, int64_t out_stride, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    return inv_rows_t<double>(plan, tw, one_row(in, nullptr, out, nrows), in_stride, nfreq, ncols, out_stride, s);
}

cudaError_t launch_wire_conv_batch(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, int circular,
                                   cudaStream_t s, int variant, uint32_t* status) {
    if (cb.n <= 0 || nfreq <= 0) return cudaSuccess;
    if (variant >= 4) {
        if (circular || !status) return cudaErrorInvalidValue;
        return launch_wire_conv_tma(cb, nfreq, stride, kw, center, variant - 4, status, s);
    }
    switch (variant) {
        case 1: launch_wc<16, true, float>(cb, nfreq, stride, kw, center, circular, s); break;
        case 2: launch_wc<8, false, float>(cb, nfreq, stride, kw, center, circular, s); break;
        case 3: launch_wc<8, true, float>(cb, nfreq, stride, kw, center, circular, s); break;
        default: launch_wc<16, false, float>(cb, nfreq, stride, kw, center, circular, s); break;
    }
    return cudaGetLastError();
}

static ConvBatch one_conv(const void* X, void* Y, const void* Rt, int nwires) {
    ConvBatch cb;
    cb.n = 1;
    cb.X[0] = X;
    cb.Y[0] = Y;
    cb.Rt[0] = Rt;
    cb.nwires[0] = nwires;
    return cb;
}

cudaError_t launch_wire_conv(const float2* X, float2* Y, const float2* Rt, int nwires, int nfreq,
                             int64_t stride, int kw, int center, int circular, cudaStream_t s, int variant,
                             uint32_t* status) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    return launch_wire_conv_batch(one_conv(X, Y, Rt, nwires), nfreq, stride, kw, center, circular, s, variant,
                                  status);
}

cudaError_t launch_wire_conv_impacts(const float2* X, float2* Y, const float2* Rt, int nwires, int impacts,
                                     int nfreq, int64_t stride, int kw, int center, int circular, cudaStream_t s) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    constexpr int B = 16;
    dim3 grid((nfreq + kConvCols - 1) / kConvCols, (nwires + B - 1) / B);
    wire_conv_impacts_kernel<kMaxRespWires, B><<<grid, kConvCols, 0, s>>>(X, Y, Rt, nwires, impacts, nfreq, stride, kw,
                                                                          center, circular);
    return cudaGetLastError();
}

cudaError_t launch_add_noise(const NoiseBatch& nb, int nfreq, int L, int64_t stride, cudaStream_t s) {
    return add_noise_t<float2>(nb, nfreq, L, stride, s);
}

cudaError_t launch_add_noise64(const NoiseBatch& nb, int nfreq, int L, int64_t stride, cudaStream_t s) {
    return add_noise_t<double2>(nb, nfreq, L, stride, s);
}

// The FP64 path of impact planes (a reference-precision path): a thread per
// output (wire w, frequency k) sums the I x K_w complex products of
// Y[w][k] = sum_i sum_r Rt[i kw + r][k] X[(w + c - r) I + i][k] straight
// from global memory (coalesced over k; rows outside the wires are zero, or
// wrap in circular mode).
__global__ void wire_conv_impacts64_kernel(const double2* __restrict__ X, double2* __restrict__ Y,
                                           const double2* __restrict__ Rt, int nwires, int impacts, int nfreq,
                                           int64_t stride, int kw, int center, int circular) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (k >= nfreq) return;
    double re = 0.0, im = 0.0;
    for (int r = 0; r < kw; ++r) {
        int wi = w + center - r;
        if (circular) {
            wi %= nwires;
            if (wi < 0) wi += nwires;
        } else if (wi < 0 || wi >= nwires) {
            continue;
        }
        for (int i = 0; i < impacts; ++i) {
            const double2 t = Rt[((int64_t)i * kw + r) * stride + k];
            const double2 x = X[((int64_t)wi * impacts + i) * stride + k];
            re = fma(t.x, x.x, fma(-t.y, x.y, re));
            im = fma(t.x, x.y, fma(t.y, x.x, im));
        }
    }
    Y[(int64_t)w * stride + k] = make_double2(re, im);
}

cudaError_t launch_wire_conv_impacts64(const double2* X, double2* Y, const double2* Rt, int nwires, int impacts,
                                       int nfreq, int64_t stride, int kw, int center, int circular, cudaStream_t s) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    if (nwires > 65535 || impacts < 1) return cudaErrorInvalidValue;
    wire_conv_impacts64_kernel<<<dim3((nfreq + 127) / 128, nwires), 128, 0, s>>>(X, Y, Rt, nwires, impacts, nfreq,
                                                                               stride, kw, center, circular);
    return cudaGetLastError();
}

cudaError_t launch_wire_conv64(const double2* X, double2* Y, const double2* Rt, int nwires, int nfreq, int64_t stride,
                               int kw, int center, int circular, cudaStream_t s) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    launch_wc<4, false, double>(one_conv(X, Y, Rt, nwires), nfreq, stride, kw, center, circular, s);
    return cudaGetLastError();
}

}  // namespace ws
