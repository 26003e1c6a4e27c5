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
// Transforms are mixed-radix (2, 3, 4, 5) Stockham autosort passes in shared
// memory with a table of L-th roots of unity.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.cuh"

namespace ws {
namespace {

__global__ void twiddle_kernel(float2* tw, int L) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < L; q += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)q / (double)L, &s, &c);
        tw[q] = make_float2((float)c, (float)s);
    }
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

// Small DFTs, y_m = sum_n x_n e^{-+2 pi i m n / R}, in place.
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

// One Stockham pass of radix R over a length-L sequence: butterfly j reads
// src[j + r L/R], twiddles by w^(r (j mod Ns)) with w the (Ns R)-th root,
// and writes dst[(j - j mod Ns) R + j mod Ns + r Ns].
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ src, float2* __restrict__ dst,
                                              int L, int Ns, const float2* __restrict__ tw) {
    const int nb = L / R;
    const int step = L / (Ns * R);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = src[j + r * nb];
            if (r > 0) x = cmul_tw<INV>(x, __ldg(&tw[k * r * step]));
            v[r] = x;
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
    int Ns = 1;
    for (int p = 0; p < plan.npass; ++p) {
        const int R = plan.radix[p];
        switch (R) {
            case 2: stockham_pass<2, INV>(src, dst, plan.L, Ns, tw); break;
            case 3: stockham_pass<3, INV>(src, dst, plan.L, Ns, tw); break;
            case 4: stockham_pass<4, INV>(src, dst, plan.L, Ns, tw); break;
            default: stockham_pass<5, INV>(src, dst, plan.L, Ns, tw); break;
        }
        __syncthreads();
        float2* t = src; src = dst; dst = t;
        Ns *= R;
    }
    return src;
}

constexpr int kRowThreads = 512;

// Two real rows (2 blockIdx.x, 2 blockIdx.x + 1) as one complex transform
// z = a + i b; then A_k = (Z_k + conj Z_{L-k}) / 2, B_k = (Z_k - conj Z_{L-k}) / 2i.
__global__ void __launch_bounds__(kRowThreads)
fwd_rows_kernel(FftPlan plan, const float2* __restrict__ tw, const float* __restrict__ in,
                int nrows, int ncols, int64_t in_stride, float2* __restrict__ out,
                int64_t out_stride, int nfreq, float scale) {
    extern __shared__ float2 smem[];
    const int L = plan.L;
    float2* a = smem;
    float2* b = smem + L;
    const int r0 = 2 * blockIdx.x;
    const bool has_b = r0 + 1 < nrows;
    const float* pa = in + (int64_t)r0 * in_stride;
    const float* pb = pa + in_stride;
    const int nload = ncols < L ? ncols : L;
    for (int n = threadIdx.x; n < L; n += blockDim.x) {
        float xa = 0.f, xb = 0.f;
        if (n < nload) {
            xa = __ldg(pa + n);
            if (has_b) xb = __ldg(pb + n);
        }
        a[n] = make_float2(xa, xb);
    }
    __syncthreads();
    const float2* z = fft_smem<false>(plan, a, b, tw);
    float2* oa = out + (int64_t)r0 * out_stride;
    float2* ob = oa + out_stride;
    const float h = 0.5f * scale;
    for (int k = threadIdx.x; k < nfreq; k += blockDim.x) {
        const float2 zk = z[k];
        const float2 zm = z[k == 0 ? 0 : L - k];
        // conj(zm) = (zm.x, -zm.y)
        oa[k] = make_float2(h * (zk.x + zm.x), h * (zk.y - zm.y));
        if (has_b) ob[k] = make_float2(h * (zk.y + zm.y), h * (zm.x - zk.x));
    }
}

// Two half spectra A (row r0) and B (row r0+1) -> Z = A + iB over the full
// Hermitian extension, inverse transform, real part row r0, imaginary r0+1.
__global__ void __launch_bounds__(kRowThreads)
inv_rows_kernel(FftPlan plan, const float2* __restrict__ tw, const float2* __restrict__ in,
                int nrows, int64_t in_stride, int nfreq, float* __restrict__ out, int ncols,
                int64_t out_stride) {
    extern __shared__ float2 smem[];
    const int L = plan.L;
    float2* a = smem;
    float2* b = smem + L;
    const int r0 = 2 * blockIdx.x;
    const bool has_b = r0 + 1 < nrows;
    const float2* ya = in + (int64_t)r0 * in_stride;
    const float2* yb = ya + in_stride;
    const bool even = (L & 1) == 0;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
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
    for (int n = threadIdx.x; n < nst; n += blockDim.x) {
        const float2 v = z[n];
        oa[n] = v.x;
        if (has_b) ob[n] = v.y;
    }
}

// Register-blocked wire convolution in the tick-frequency domain.  Thread
// (k, block of B wires) keeps the K taps of column k in registers and
// streams the B + K - 1 input rows its outputs need once each.
template <int K, int B>
__global__ void __launch_bounds__(128)
wire_conv_kernel(const float2* __restrict__ X, float2* __restrict__ Y, const float2* __restrict__ Rt,
                 int nwires, int nfreq, int64_t stride, int kw, int center, int circular) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int w0 = blockIdx.y * B;
    if (k >= nfreq) return;
    float2 c[K];
#pragma unroll
    for (int r = 0; r < K; ++r) c[r] = r < kw ? __ldg(&Rt[(int64_t)r * stride + k]) : make_float2(0.f, 0.f);
    float2 acc[B];
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = make_float2(0.f, 0.f);
    const int ibase = w0 + center - (K - 1);
#pragma unroll
    for (int u = 0; u < B + K - 1; ++u) {
        int i = ibase + u;
        float2 x = make_float2(0.f, 0.f);
        if (circular) {
            i %= nwires;
            if (i < 0) i += nwires;
            x = __ldg(&X[(int64_t)i * stride + k]);
        } else if (i >= 0 && i < nwires) {
            x = __ldg(&X[(int64_t)i * stride + k]);
        }
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

}  // namespace

cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t s) {
    twiddle_kernel<<<(L + 255) / 256, 256, 0, s>>>(tw, L);
    return cudaGetLastError();
}

static cudaError_t set_smem(const void* fn, int bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_fwd_rows(const FftPlan& plan, const float2* tw, const float* in, int nrows,
                            int ncols, int64_t in_stride, float2* out, int64_t out_stride,
                            int nfreq, float scale, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    const int smem = 2 * plan.L * (int)sizeof(float2);
    cudaError_t e = set_smem((const void*)fwd_rows_kernel, smem);
    if (e != cudaSuccess) return e;
    fwd_rows_kernel<<<(nrows + 1) / 2, kRowThreads, smem, s>>>(plan, tw, in, nrows, ncols, in_stride,
                                                               out, out_stride, nfreq, scale);
    return cudaGetLastError();
}

cudaError_t launch_inv_rows(const FftPlan& plan, const float2* tw, const float2* in, int nrows,
                            int64_t in_stride, int nfreq, float* out, int ncols,
                            int64_t out_stride, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    const int smem = 2 * plan.L * (int)sizeof(float2);
    cudaError_t e = set_smem((const void*)inv_rows_kernel, smem);
    if (e != cudaSuccess) return e;
    inv_rows_kernel<<<(nrows + 1) / 2, kRowThreads, smem, s>>>(plan, tw, in, nrows, in_stride, nfreq,
                                                               out, ncols, out_stride);
    return cudaGetLastError();
}

cudaError_t launch_wire_conv(const float2* X, float2* Y, const float2* Rt, int nwires, int nfreq,
                             int64_t stride, int kw, int center, int circular, cudaStream_t s) {
    if (nwires <= 0 || nfreq <= 0) return cudaSuccess;
    constexpr int K = kMaxRespWires, B = 16;
    dim3 grid((nfreq + 127) / 128, (nwires + B - 1) / B);
    wire_conv_kernel<K, B><<<grid, 128, 0, s>>>(X, Y, Rt, nwires, nfreq, stride, kw, center, circular);
    return cudaGetLastError();
}

}  // namespace ws
