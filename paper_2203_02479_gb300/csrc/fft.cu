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

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * w (forward) or a * conj(w) (inverse)
template <bool INV>
__device__ __forceinline__ float2 cmul_tw(float2 a, float2 w) {
    if (INV) w.y = -w.y;
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// -i*a (forward) or +i*a (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// x * e^{-+2 pi i M / N} with M, N compile-time.
template <int N, int M, bool INV>
__device__ __forceinline__ float2 rot(float2 x) {
    constexpr int m = M % N;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (2 * m == N) {
        return make_float2(-x.x, -x.y);
    } else if constexpr (4 * m == N) {
        return mul_mi<INV>(x);
    } else if constexpr (4 * m == 3 * N) {
        return mul_mi<!INV>(x);
    } else {
        constexpr float c = (float)cx_trig2pi(m, N, false);
        constexpr float s = INV ? (float)cx_trig2pi(m, N, true) : -(float)cx_trig2pi(m, N, true);
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    }
}

// ------------------------------------------------------------ small DFTs
// y_m = sum_n x_n e^{-+2 pi i m n / R}, in place, natural order.
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV> struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float s3 = 0.866025403784438647f;  // sin(2 pi / 3)
        float2 t1 = cadd(v[1], v[2]);
        float2 t2 = csub(v[1], v[2]);
        float2 a = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
        float2 b = mul_mi<INV>(cscale(t2, s3));
        v[0] = cadd(v[0], t1);
        v[1] = cadd(a, b);
        v[2] = csub(a, b);
    }
};

template <bool INV> struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <bool INV> struct Dft<5, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float c1 = 0.309016994374947424f;   // cos(2 pi / 5)
        const float c2 = -0.809016994374947424f;  // cos(4 pi / 5)
        const float s1 = 0.951056516295153572f;   // sin(2 pi / 5)
        const float s2 = 0.587785252292473129f;   // sin(4 pi / 5)
        float2 t1 = cadd(v[1], v[4]), t3 = csub(v[1], v[4]);
        float2 t2 = cadd(v[2], v[3]), t4 = csub(v[2], v[3]);
        float2 x0 = v[0];
        float2 a1 = make_float2(fmaf(c1, t1.x, fmaf(c2, t2.x, x0.x)), fmaf(c1, t1.y, fmaf(c2, t2.y, x0.y)));
        float2 a2 = make_float2(fmaf(c2, t1.x, fmaf(c1, t2.x, x0.x)), fmaf(c2, t1.y, fmaf(c1, t2.y, x0.y)));
        float2 b1 = make_float2(fmaf(s1, t3.x, s2 * t4.x), fmaf(s1, t3.y, s2 * t4.y));
        float2 b2 = make_float2(fmaf(s2, t3.x, -s1 * t4.x), fmaf(s2, t3.y, -s1 * t4.y));
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
template <int N1, int N2, bool INV>
__device__ __forceinline__ void dft_composite(float2* v) {
    constexpr int N = N1 * N2;
    sfor<N2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        float2 t[N1];
        sfor<N1>([&](auto n1c) { t[decltype(n1c)::value] = v[N2 * decltype(n1c)::value + n2]; });
        Dft<N1, INV>::run(t);
        sfor<N1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            v[N2 * k1 + n2] = rot<N, n2 * k1, INV>(t[k1]);
        });
    });
    float2 out[N];
    sfor<N1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        float2 t[N2];
        sfor<N2>([&](auto n2c) { t[decltype(n2c)::value] = v[N2 * k1 + decltype(n2c)::value]; });
        Dft<N2, INV>::run(t);
        sfor<N2>([&](auto k2c) { out[k1 + N1 * decltype(k2c)::value] = t[decltype(k2c)::value]; });
    });
    sfor<N>([&](auto ic) { v[decltype(ic)::value] = out[decltype(ic)::value]; });
}

#define WS_COMPOSITE(R, A, B)                                                          \
    template <bool INV> struct Dft<R, INV> {                                            \
        __device__ __forceinline__ static void run(float2* v) { dft_composite<A, B, INV>(v); } \
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

// One Stockham pass of radix R over a length-L sequence: butterfly j reads
// src[j + r L/R], multiplies input r by w^r with w = e^{-+2 pi i (j mod Ns) /
// (Ns R)} (w from the pass's table of Ns base twiddles, its powers by a
// multiply tree of depth <= 5), and writes dst[(j - j mod Ns) R + j mod Ns +
// r Ns].
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ src, float2* __restrict__ dst,
                                              int L, int Ns, const float2* __restrict__ tw) {
    const int nb = L / R;
    for (int j = threadIdx.x; j < nb; j += kRowThreads) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
        if (Ns > 1) {
            float2 wp[R];
            wp[1] = __ldg(&tw[k]);
            if (INV) wp[1].y = -wp[1].y;
#pragma unroll
            for (int r = 2; r < R; ++r) wp[r] = cmul_tw<false>(wp[r / 2], wp[r - r / 2]);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul_tw<false>(v[r], wp[r]);
        }
        Dft<R, INV>::run(v);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[d + r * Ns] = v[r];
    }
}

// Full transform in shared memory; returns the buffer holding the result.
template <bool INV>
__device__ float2* fft_smem(const FftPlan& plan, float2* a, float2* b, const float2* __restrict__ tw) {
    float2* src = a;
    float2* dst = b;
    for (int p = 0; p < plan.npass; ++p) {
        const int Ns = plan.ns[p];
        const float2* t = tw + plan.twoff[p];
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
        float2* tmp = src; src = dst; dst = tmp;
    }
    return src;
}

// Pass twiddles: for pass p, tw[twoff[p] + k] = e^{-2 pi i k / (Ns R)}, k < Ns.
__global__ void pass_twiddles_kernel(float2* tw, FftPlan plan) {
    for (int p = 0; p < plan.npass; ++p) {
        const int Ns = plan.ns[p], R = plan.radix[p];
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += gridDim.x * blockDim.x) {
            double s, c;
            sincospi(-2.0 * (double)k / (double)((long long)Ns * R), &s, &c);
            tw[plan.twoff[p] + k] = make_float2((float)c, (float)s);
        }
    }
}

// Two real rows (2 blockIdx.x, 2 blockIdx.x + 1) as one complex transform
// z = a + i b; then A_k = (Z_k + conj Z_{L-k}) / 2, B_k = (Z_k - conj Z_{L-k}) / 2i.
__global__ void __launch_bounds__(kRowThreads, 2)
fwd_rows_kernel(FftPlan plan, const float2* __restrict__ tw, const __grid_constant__ RowUnits U, int ncols,
                int64_t in_stride, int64_t out_stride, int nfreq, float scale, int vec4) {
    extern __shared__ __align__(16) float2 smem[];
    const int L = plan.L;
    float2* a = smem;
    float2* b = smem + ((L + 1) & ~1);  // both buffers 16-byte aligned
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.x);
    const float* __restrict__ in = static_cast<const float*>(U.in[u]);
    float2* __restrict__ out = static_cast<float2*>(U.out[u]);
    const int nrows = U.nrows[u];
    const int r0 = 2 * ((int)blockIdx.x - U.prefix[u]);
    const bool has_b = r0 + 1 < nrows;
    const float* pa = in + (int64_t)r0 * in_stride;
    const float* pb = has_b ? pa + in_stride : pa;
    const int nload = ncols < L ? ncols : L;
    if (vec4) {
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
        for (int n = nload + threadIdx.x; n < L; n += kRowThreads) a[n] = make_float2(0.f, 0.f);
    } else {
        for (int n = threadIdx.x; n < L; n += kRowThreads) {
            float xa = 0.f, xb = 0.f;
            if (n < nload) {
                xa = __ldg(pa + n);
                if (has_b) xb = __ldg(pb + n);
            }
            a[n] = make_float2(xa, xb);
        }
    }
    __syncthreads();
    const float2* z = fft_smem<false>(plan, a, b, tw);
    float2* oa = out + (int64_t)r0 * out_stride;
    float2* ob = oa + out_stride;
    const float h = 0.5f * scale;
    for (int k = threadIdx.x; k < nfreq; k += kRowThreads) {
        const float2 zk = z[k];
        const float2 zm = z[k == 0 ? 0 : L - k];
        oa[k] = make_float2(h * (zk.x + zm.x), h * (zk.y - zm.y));
        if (has_b) ob[k] = make_float2(h * (zk.y + zm.y), h * (zm.x - zk.x));
    }
}

// Two half spectra A (row r0) and B (row r0+1) -> Z = A + iB over the full
// Hermitian extension, inverse transform, real part row r0, imaginary r0+1.
__global__ void __launch_bounds__(kRowThreads, 2)
inv_rows_kernel(FftPlan plan, const float2* __restrict__ tw, const __grid_constant__ RowUnits U,
                int64_t in_stride, int nfreq, int ncols, int64_t out_stride, int vec4) {
    extern __shared__ __align__(16) float2 smem[];
    const int L = plan.L;
    float2* a = smem;
    float2* b = smem + ((L + 1) & ~1);  // both buffers 16-byte aligned
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.x);
    const float2* __restrict__ in = static_cast<const float2*>(U.in[u]);
    float* __restrict__ out = static_cast<float*>(U.out[u]);
    const int nrows = U.nrows[u];
    const int r0 = 2 * ((int)blockIdx.x - U.prefix[u]);
    const bool has_b = r0 + 1 < nrows;
    const float2* ya = in + (int64_t)r0 * in_stride;
    const float2* yb = has_b ? ya + in_stride : ya;
    const bool even = (L & 1) == 0;
    for (int k = threadIdx.x; k < L; k += kRowThreads) {
        const bool upper = k >= nfreq;
        const int kk = upper ? L - k : k;
        float2 A = __ldg(ya + kk);
        float2 B = has_b ? __ldg(yb + kk) : make_float2(0.f, 0.f);
        if (kk == 0 || (even && 2 * kk == L)) { A.y = 0.f; B.y = 0.f; }
        if (upper) { A.y = -A.y; B.y = -B.y; }
        a[k] = make_float2(A.x - B.y, A.y + B.x);
    }
    __syncthreads();
    const float2* z = fft_smem<true>(plan, a, b, tw);
    float* oa = out + (int64_t)r0 * out_stride;
    float* ob = oa + out_stride;
    const int nst = ncols < L ? ncols : L;
    if (vec4) {
        const float4* z4 = reinterpret_cast<const float4*>(z);
        for (int n4 = threadIdx.x; n4 < nst / 4; n4 += kRowThreads) {
            const float4 u = z4[2 * n4], w = z4[2 * n4 + 1];
            reinterpret_cast<float4*>(oa)[n4] = make_float4(u.x, u.z, w.x, w.z);
            if (has_b) reinterpret_cast<float4*>(ob)[n4] = make_float4(u.y, u.w, w.y, w.w);
        }
    } else {
        for (int n = threadIdx.x; n < nst; n += kRowThreads) {
            const float2 v = z[n];
            oa[n] = v.x;
            if (has_b) ob[n] = v.y;
        }
    }
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
template <int K, int B, bool KARATSUBA>
__global__ void __launch_bounds__(kConvCols)
wire_conv_kernel(const __grid_constant__ ConvUnits U, int nfreq, int64_t stride, int kw, int center, int circular) {
    constexpr int ROWS = B + K - 1;
    __shared__ float4 tile[ROWS][kConvCols / 2];
    const int u = find_unit(U.prefix, U.n, (int)blockIdx.y);
    const float2* __restrict__ X = U.X[u];
    float2* __restrict__ Y = U.Y[u];
    const float2* __restrict__ Rt = U.Rt[u];
    const int nwires = U.nwires[u];
    const int k0 = blockIdx.x * kConvCols;
    const int w0 = ((int)blockIdx.y - U.prefix[u]) * B;
    const int ibase = w0 + center - (K - 1);
    for (int e = threadIdx.x; e < ROWS * (kConvCols / 2); e += kConvCols) {
        const int u = e / (kConvCols / 2), c2 = e - u * (kConvCols / 2);
        int i = ibase + u;
        const int kk = k0 + 2 * c2;
        bool ok = kk < stride;
        if (circular) {
            i %= nwires;
            if (i < 0) i += nwires;
        } else {
            ok = ok && i >= 0 && i < nwires;
        }
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) v = __ldg(reinterpret_cast<const float4*>(X + (int64_t)i * stride + kk));
        tile[u][c2] = v;
    }
    __syncthreads();
    const int k = k0 + threadIdx.x;
    if (k >= nfreq) return;
    const float2* col = reinterpret_cast<const float2*>(&tile[0][0]) + threadIdx.x;
    if constexpr (KARATSUBA) {
        float cc[K], cm[K], cp[K];   // c, d - c, c + d
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const float2 t = r < kw ? __ldg(&Rt[(int64_t)r * stride + k]) : make_float2(0.f, 0.f);
            cc[r] = t.x;
            cm[r] = t.y - t.x;
            cp[r] = t.x + t.y;
        }
        float k1[B], k2[B], k3[B];
#pragma unroll
        for (int b = 0; b < B; ++b) k1[b] = k2[b] = k3[b] = 0.f;
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const float2 x = col[u * kConvCols];
            const float sab = x.x + x.y;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int r = b + K - 1 - u;
                if (r >= 0 && r < K) {
                    k1[b] = fmaf(cc[r], sab, k1[b]);
                    k2[b] = fmaf(cm[r], x.x, k2[b]);
                    k3[b] = fmaf(cp[r], x.y, k3[b]);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (w0 + b < nwires) Y[(int64_t)(w0 + b) * stride + k] = make_float2(k1[b] - k3[b], k1[b] + k2[b]);
    } else {
        float2 c[K];
#pragma unroll
        for (int r = 0; r < K; ++r) c[r] = r < kw ? __ldg(&Rt[(int64_t)r * stride + k]) : make_float2(0.f, 0.f);
        float2 acc[B];
#pragma unroll
        for (int b = 0; b < B; ++b) acc[b] = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < ROWS; ++u) {
            const float2 x = col[u * kConvCols];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int r = b + K - 1 - u;
                if (r >= 0 && r < K) {
                    acc[b].x = fmaf(c[r].x, x.x, fmaf(-c[r].y, x.y, acc[b].x));
                    acc[b].y = fmaf(c[r].x, x.y, fmaf(c[r].y, x.x, acc[b].y));
                }
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (w0 + b < nwires) Y[(int64_t)(w0 + b) * stride + k] = acc[b];
    }
}

template <int B, bool KS>
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
        U.prefix[i + 1] = U.prefix[i] + (cb.nwires[i] + B - 1) / B;
    }
    dim3 grid((nfreq + kConvCols - 1) / kConvCols, U.prefix[cb.n]);
    wire_conv_kernel<K, B, KS><<<grid, kConvCols, 0, s>>>(U, nfreq, stride, kw, center, circular);
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
// XG[w][k] over this thread's chunk of wires (XS zero outside the grid, or
// wrapped), accumulated into A with atomics.
constexpr int kRespGradRows = 64;

__global__ void __launch_bounds__(128)
resp_grad_kernel(const float2* __restrict__ XG, const float2* __restrict__ XS, float2* __restrict__ A, int nwires,
                 int nfreq, int64_t stride, int kw, int center, int circular, float scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nfreq) return;
    const int w0 = blockIdx.y * kRespGradRows;
    const int w1 = min(nwires, w0 + kRespGradRows);
    float2 acc[kMaxRespWires];
#pragma unroll
    for (int r = 0; r < kMaxRespWires; ++r) acc[r] = make_float2(0.f, 0.f);
    for (int w = w0; w < w1; ++w) {
        const float2 xg = __ldg(&XG[(int64_t)w * stride + k]);
#pragma unroll
        for (int r = 0; r < kMaxRespWires; ++r) {
            if (r >= kw) break;
            int ws = w - (r - center);
            if (circular) {
                ws %= nwires;
                if (ws < 0) ws += nwires;
            } else if (ws < 0 || ws >= nwires) {
                continue;
            }
            const float2 xs = __ldg(&XS[(int64_t)ws * stride + k]);
            // conj(xs) * xg
            acc[r].x = fmaf(xs.x, xg.x, fmaf(xs.y, xg.y, acc[r].x));
            acc[r].y = fmaf(xs.x, xg.y, fmaf(-xs.y, xg.x, acc[r].y));
        }
    }
#pragma unroll
    for (int r = 0; r < kMaxRespWires; ++r) {
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
    dim3 grid((nfreq + 127) / 128, (nwires + kRespGradRows - 1) / kRespGradRows);
    resp_grad_kernel<<<grid, 128, 0, s>>>(XG, XS, A, nwires, nfreq, stride, kw, center, circular, scale);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(float2* tw, const FftPlan& plan, cudaStream_t s) {
    pass_twiddles_kernel<<<(plan.L + 255) / 256, 256, 0, s>>>(tw, plan);
    return cudaGetLastError();
}

static cudaError_t set_smem(const void* fn, int bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

static RowUnits row_units(const RowBatch& rb, bool* aligned16) {
    RowUnits U;
    U.n = rb.n;
    U.prefix[0] = 0;
    *aligned16 = true;
    for (int i = 0; i < rb.n; ++i) {
        U.in[i] = rb.in[i];
        U.out[i] = rb.out[i];
        U.nrows[i] = rb.nrows[i];
        U.prefix[i + 1] = U.prefix[i] + (rb.nrows[i] + 1) / 2;
        *aligned16 = *aligned16 && ((uintptr_t)rb.in[i] % 16 == 0) && ((uintptr_t)rb.out[i] % 16 == 0);
    }
    return U;
}

cudaError_t launch_fwd_rows_batch(const FftPlan& plan, const float2* tw, const RowBatch& rb, int ncols,
                                  int64_t in_stride, int64_t out_stride, int nfreq, float scale, cudaStream_t s) {
    if (rb.n <= 0) return cudaSuccess;
    const int smem = 2 * ((plan.L + 1) & ~1) * (int)sizeof(float2);
    cudaError_t e = set_smem((const void*)fwd_rows_kernel, smem);
    if (e != cudaSuccess) return e;
    bool al = false;
    const RowUnits U = row_units(rb, &al);
    if (U.prefix[rb.n] <= 0) return cudaSuccess;
    const int nload = ncols < plan.L ? ncols : plan.L;
    const int vec4 = al && (in_stride % 4 == 0) && (nload % 4 == 0);
    fwd_rows_kernel<<<U.prefix[rb.n], kRowThreads, smem, s>>>(plan, tw, U, ncols, in_stride, out_stride, nfreq,
                                                              scale, vec4);
    return cudaGetLastError();
}

cudaError_t launch_fwd_rows(const FftPlan& plan, const float2* tw, const float* in, int nrows,
                            int ncols, int64_t in_stride, float2* out, int64_t out_stride,
                            int nfreq, float scale, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    RowBatch rb;
    rb.n = 1;
    rb.in[0] = in;
    rb.out[0] = out;
    rb.nrows[0] = nrows;
    return launch_fwd_rows_batch(plan, tw, rb, ncols, in_stride, out_stride, nfreq, scale, s);
}

cudaError_t launch_inv_rows_batch(const FftPlan& plan, const float2* tw, const RowBatch& rb, int64_t in_stride,
                                  int nfreq, int ncols, int64_t out_stride, cudaStream_t s) {
    if (rb.n <= 0) return cudaSuccess;
    const int smem = 2 * ((plan.L + 1) & ~1) * (int)sizeof(float2);
    cudaError_t e = set_smem((const void*)inv_rows_kernel, smem);
    if (e != cudaSuccess) return e;
    bool al = false;
    const RowUnits U = row_units(rb, &al);
    if (U.prefix[rb.n] <= 0) return cudaSuccess;
    const int nst = ncols < plan.L ? ncols : plan.L;
    const int vec4 = al && (out_stride % 4 == 0) && (nst % 4 == 0);
    inv_rows_kernel<<<U.prefix[rb.n], kRowThreads, smem, s>>>(plan, tw, U, in_stride, nfreq, ncols, out_stride,
                                                              vec4);
    return cudaGetLastError();
}

cudaError_t launch_inv_rows(const FftPlan& plan, const float2* tw, const float2* in, int nrows,
                            int64_t in_stride, int nfreq, float* out, int ncols,
                            int64_t out_stride, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    RowBatch rb;
    rb.n = 1;
    rb.in[0] = in;
    rb.out[0] = out;
    rb.nrows[0] = nrows;
    return launch_inv_rows_batch(plan, tw, rb, in_stride, nfreq, ncols, out_stride, s);
}

cudaError_t launch_wire_conv_batch(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, int circular,
                                   cudaStream_t s, int variant) {
    if (cb.n <= 0 || nfreq <= 0) return cudaSuccess;
    switch (variant) {
        case 1: launch_wc<16, true>(cb, nfreq, stride, kw, center, circular, s); break;
        case 2: launch_wc<8, false>(cb, nfreq, stride, kw, center, circular, s); break;
        case 3: launch_wc<8, true>(cb, nfreq, stride, kw, center, circular, s); break;
        default: launch_wc<16, false>(cb, nfreq, stride, kw, center, circular, s); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_wire_conv(const float2* X, float2* Y, const float2* Rt, int nwires, int nfreq,
                             int64_t stride, int kw, int center, int circular, cudaStream_t s, int variant) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    ConvBatch cb;
    cb.n = 1;
    cb.X[0] = X;
    cb.Y[0] = Y;
    cb.Rt[0] = Rt;
    cb.nwires[0] = nwires;
    return launch_wire_conv_batch(cb, nfreq, stride, kw, center, circular, s, variant);
}

}  // namespace ws
