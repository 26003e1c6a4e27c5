// Wire convolution fed by the tensor memory accelerator (linear mode).
//
// Same sum as wire_conv_kernel in fft.cu (Y[w][k] = sum_r Rt[r][k]
// X[w + c - r][k], the wire axis of Eq. 2's product in the tick-frequency
// domain), but the (B + K - 1) x 128-column input tiles arrive by 2D TMA
// copies (cp.async.bulk.tensor) that complete on shared-memory mbarriers:
// persistent CTAs double-buffer, issuing tile t + 1 while computing tile t.
// Rows outside the grid come back as zeros from the copy engine's
// out-of-bounds fill, which is exactly linear mode's zero padding.
//
// Every mbarrier wait is bounded: if a copy never lands, the CTA sets
// WS_DEV_TIMEOUT in the plane's status word, waits (bounded) for its other
// copy in flight and returns; it never spins forever.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "ws_internal.cuh"

namespace ws {
namespace {

constexpr int kCols = 128;                 // complex columns per tile (one thread each)

struct TmaConvUnits {
    CUtensorMap map[kMaxUnits];            // X of each unit: {2 * stride floats, nwires rows}
    int n;
    int prefix[kMaxUnits + 1];             // cumulative tiles
    int nwires[kMaxUnits];
    void* Y[kMaxUnits];
    const void* Rt[kMaxUnits];
    const mark_t* rows[kMaxUnits];         // active-row marks, or null (every tile computed)
    const mark_t* epoch;
};

// 2D tile copy of the box at (x, y) into dst, completing on bar.
__device__ __forceinline__ void tma_load_tile(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                              uint32_t bytes) {
    const uint32_t b = smem_addr(bar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(b)
        : "memory");
}

template <int K, int B, bool KARATSUBA>
__global__ void __launch_bounds__(kCols)
wire_conv_tma_kernel(const __grid_constant__ TmaConvUnits U, int nfreq, int64_t stride, int kw, int center,
                     int nkblocks, uint32_t* status) {
    constexpr int ROWS = B + K - 1;
    constexpr uint32_t TILE_BYTES = ROWS * kCols * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    auto buf = [&](int st) { return reinterpret_cast<float2*>(smem + (st ? TILE_BYTES : 0u)); };
    const int total = U.prefix[U.n];
    // tiles run wire block fastest, so a CTA's consecutive tiles share their
    // column block (the taps stay in registers) and overlap in halo rows
    auto tile_of = [&](int t, int& u, int& k0, int& w0) {
        int lo = 0, hi = U.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (U.prefix[mid] <= t) lo = mid; else hi = mid - 1;
        }
        u = lo;
        const int tt = t - U.prefix[u];
        const int nwb = (U.nwires[u] + B - 1) / B;
        k0 = (tt / nwb) * kCols;
        w0 = (tt % nwb) * B;
    };
    auto issue = [&](int t, int st) {
        int u, k0, w0;
        tile_of(t, u, k0, w0);
        tma_load_tile(buf(st), &U.map[u], 2 * k0, w0 + center - (K - 1), &bar[st], TILE_BYTES);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // each CTA takes a contiguous run of tiles
    const int t_end = (int)((int64_t)total * (blockIdx.x + 1) / gridDim.x);
    int t = (int)((int64_t)total * blockIdx.x / gridDim.x);
    if (t < t_end && threadIdx.x == 0) issue(t, 0);
    uint32_t parity[2] = {0u, 0u};
    bool inflight_next = false;
    int cur_u = -1, cur_k = -1;
    float cc[K], cm[K], cp[K];   // taps of the current column block (Karatsuba form)
    float2 c[K];                 // the same, plain form
    for (int i = 0; t < t_end; ++i, ++t) {
        const int st = i & 1;
        const int tn = t + 1;
        inflight_next = tn < t_end;
        if (inflight_next && threadIdx.x == 0) issue(tn, st ^ 1);
        const bool ok = mbar_wait(&bar[st], parity[st]);
        parity[st] ^= 1u;
        if (__syncthreads_or(!ok)) {
            // A copy never landed: flag it, let the other copy (if any) drain,
            // and leave without touching the buffers again.
            if (threadIdx.x == 0) atomicOr(status, WS_DEV_TIMEOUT);
            if (inflight_next) mbar_wait(&bar[st ^ 1], parity[st ^ 1]);
            return;
        }
        int u, k0, w0;
        tile_of(t, u, k0, w0);
        const int k = k0 + threadIdx.x;
        const int nwires = U.nwires[u];
        // active rows: a tile none of whose output rows is live is never
        // read (the barrier inside also frees buffer st for the next copy)
        if (U.rows[u] &&
            !cta_any_marked(U.rows[u], read_epoch(U.epoch), w0 + center - kw + 1, w0 + B - 1 + center, nwires))
            continue;
        float2* __restrict__ Y = static_cast<float2*>(U.Y[u]);
        const float2* __restrict__ Rt = static_cast<const float2*>(U.Rt[u]);
        const float2* col = buf(st) + threadIdx.x;
        if (u != cur_u || k0 != cur_k) {
            cur_u = u;
            cur_k = k0;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const float2 v =
                    (r < kw && k < nfreq) ? __ldg(&Rt[(int64_t)r * stride + k]) : make_float2(0.f, 0.f);
                if constexpr (KARATSUBA) {
                    cc[r] = v.x;
                    cm[r] = v.y - v.x;
                    cp[r] = v.x + v.y;
                } else {
                    c[r] = v;
                }
            }
        }
        if (k < nfreq) {
            if constexpr (KARATSUBA) {
                float k1[B], k2[B], k3[B];
#pragma unroll
                for (int b = 0; b < B; ++b) k1[b] = k2[b] = k3[b] = 0.f;
#pragma unroll
                for (int uu = 0; uu < ROWS; ++uu) {
                    const float2 x = col[uu * kCols];
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
#pragma unroll
                for (int b = 0; b < B; ++b)
                    if (w0 + b < nwires) Y[(int64_t)(w0 + b) * stride + k] = make_float2(k1[b] - k3[b], k1[b] + k2[b]);
            } else {
                float2 acc[B];
#pragma unroll
                for (int b = 0; b < B; ++b) acc[b] = make_float2(0.f, 0.f);
#pragma unroll
                for (int uu = 0; uu < ROWS; ++uu) {
                    const float2 x = col[uu * kCols];
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const int r = b + K - 1 - uu;
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
        __syncthreads();   // buffer st is free for the copy issued next iteration
    }
}

// Ring-fed variant: a CTA walks a run of consecutive wire blocks of one
// column block, and the input rows arrive once per run in chunks of
// kRingRows rows (one TMA copy each) into a ring of kRingSlots chunk
// buffers, instead of one (B + K - 1)-row tile per output block: the
// window of tile i of a run (rows ybase + 16 i .. + 35) is chunks i, i + 1
// and the head of i + 2, so each further tile fetches only its 16 new rows.
// Chunk i + 3 (for tile i + 1) is issued into chunk i's slot as soon as the
// window's first 16 rows have been read, half-way through tile i.  48 KB of
// shared memory per CTA lets four CTAs (16 warps) share an SM.
constexpr int kRingRows = 16;
constexpr int kRingSlots = 3;

template <int K, bool KARATSUBA>
__global__ void __launch_bounds__(kCols, 4)
wire_conv_ring_kernel(const __grid_constant__ TmaConvUnits U, int nfreq, int64_t stride, int kw, int center,
                      uint32_t* status) {
    constexpr int B = kRingRows;
    constexpr int ROWS = B + K - 1;
    static_assert(ROWS > 2 * kRingRows && ROWS <= kRingSlots * kRingRows, "window spans three chunks");
    constexpr uint32_t CHUNK_BYTES = kRingRows * kCols * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[kRingSlots];
    auto slot_buf = [&](int sl) { return reinterpret_cast<const float2*>(smem + sl * CHUNK_BYTES); };
    const int total = U.prefix[U.n];
    auto tile_of = [&](int t, int& u, int& k0, int& wb, int& nwb) {
        int lo = 0, hi = U.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (U.prefix[mid] <= t) lo = mid; else hi = mid - 1;
        }
        u = lo;
        const int tt = t - U.prefix[u];
        nwb = (U.nwires[u] + B - 1) / B;
        k0 = (tt / nwb) * kCols;
        wb = tt % nwb;
    };
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRingSlots; ++i) mbar_init(&bar[i]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0u, pending = 0u;   // per slot: parity of its next completion; copy in flight
    // Give up on a copy: flag it, drain the others (bounded) and report.
    auto fail = [&]() {
        if (threadIdx.x == 0) atomicOr(status, WS_DEV_TIMEOUT);
        for (int sl = 0; sl < kRingSlots; ++sl)
            if (pending & (1u << sl)) mbar_wait(&bar[sl], (phase >> sl) & 1u);
    };
    auto wait_slot = [&](int sl) -> bool {
        if (!(pending & (1u << sl))) return true;
        const bool ok = mbar_wait(&bar[sl], (phase >> sl) & 1u);
        if (__syncthreads_or(!ok)) return false;
        phase ^= 1u << sl;
        pending &= ~(1u << sl);
        return true;
    };
    const int t_end = (int)((int64_t)total * (blockIdx.x + 1) / gridDim.x);
    int t = (int)((int64_t)total * blockIdx.x / gridDim.x);
    float cc[K], cm[K], cp[K];   // taps of the run's column block (Karatsuba form)
    float2 c[K];                 // the same, plain form
    __shared__ unsigned long long s_live;   // live tiles of the current run (bit i: tile i), with marks
    while (t < t_end) {
        int u, k0, wb, nwb;
        tile_of(t, u, k0, wb, nwb);
        const int run = min(t_end - t, nwb - wb);   // tiles in this run
        int n = run;
        // live tiles of the (trimmed) run with marks, bit i for tile i;
        // per_tile: runs over 64 tiles test each tile on its own
        unsigned long long tiles_live = ~0ull;
        bool per_tile = false;
        // active rows: trim the run to its first .. last live tile (a tile is
        // live if a marked row lies in [w0 + c - K_w + 1, w0 + B - 1 + c]),
        // so the chunks of dead tiles at either end are never fetched
        if (const mark_t* marks = U.rows[u]) {
            const mark_t cur = read_epoch(U.epoch);
            const int nw = U.nwires[u];
            if (threadIdx.x == 0) s_live = 0ull;
            __syncthreads();
            const int lo = wb * B + center - kw + 1, hi = (wb + run) * B - 1 + center;
            unsigned long long mine = 0ull;
            for (int r = max(lo, 0) + (int)threadIdx.x; r <= min(hi, nw - 1); r += kCols) {
                if (marks[r] != cur) continue;
                // tiles i whose window holds row r: w0_i + c - kw + 1 <= r <= w0_i + B - 1 + c
                const int ia = max(0, (r - center - (B - 1) - wb * B + B - 1) / B);
                const int ib = min(run - 1, (r - center + kw - 1 - wb * B) / B);
                for (int i = ia; i <= ib && i < 64; ++i) mine |= 1ull << i;
            }
            if (mine) atomicOr(&s_live, mine);
            __syncthreads();
            const unsigned long long live = s_live;
            __syncthreads();   // s_live read by every thread before the next run resets it
            if (run <= 64) {
                if (live == 0ull) {
                    t += run;
                    continue;
                }
                const int first = __ffsll((long long)live) - 1;
                const int last = 63 - __clzll((long long)live);
                wb += first;
                n = last - first + 1;
                tiles_live = live >> first;
            } else {
                per_tile = true;
            }
        }
        const int ybase = wb * B + center - (K - 1);
        const CUtensorMap* map = &U.map[u];
        auto issue = [&](int j) {   // chunk j of the run into slot j % 3 (thread 0 copies, all track)
            const int sl = j % kRingSlots;
            if (threadIdx.x == 0) tma_load_tile(smem + sl * CHUNK_BYTES, map, 2 * k0, ybase + kRingRows * j, &bar[sl],
                                                CHUNK_BYTES);
            pending |= 1u << sl;
        };
        for (int j = 0; j < kRingSlots; ++j) issue(j);
        const int k = k0 + threadIdx.x;
        const int nwires = U.nwires[u];
        float2* __restrict__ Y = static_cast<float2*>(U.Y[u]);
        const float2* __restrict__ Rt = static_cast<const float2*>(U.Rt[u]);
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const float2 v = (r < kw && k < nfreq) ? __ldg(&Rt[(int64_t)r * stride + k]) : make_float2(0.f, 0.f);
            if constexpr (KARATSUBA) {
                cc[r] = v.x;
                cm[r] = v.y - v.x;
                cp[r] = v.x + v.y;
            } else {
                c[r] = v;
            }
        }
        for (int i = 0; i < n; ++i) {
            const int s0 = i % kRingSlots, s1 = (i + 1) % kRingSlots, s2 = (i + 2) % kRingSlots;
            if (!wait_slot(s0) || !wait_slot(s1) || !wait_slot(s2)) {
                fail();
                return;
            }
            const float2* col0 = slot_buf(s0) + threadIdx.x;
            const float2* col1 = slot_buf(s1) + threadIdx.x;
            const float2* col2 = slot_buf(s2) + threadIdx.x;
            const int w0 = (wb + i) * B;
            // active rows: skip the sums of a tile none of whose output rows
            // is live (its chunks still stream through the ring), from the
            // run's bitmask (no loads or barrier per tile)
            const bool live_tile = !U.rows[u] ? true
                                   : per_tile ? cta_any_marked(U.rows[u], read_epoch(U.epoch), w0 + center - kw + 1,
                                                               w0 + B - 1 + center, nwires)
                                              : ((tiles_live >> i) & 1ull) != 0ull;   // i < 64 here
            float k1[B], k2[B], k3[B];
            float2 acc[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                k1[b] = k2[b] = k3[b] = 0.f;
                acc[b] = make_float2(0.f, 0.f);
            }
            // window row uu: input row ybase + 16 i + uu, read by outputs b = uu - (K - 1) + r
            auto row = [&](const float2 x, const int uu) {
                if constexpr (KARATSUBA) {
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
                } else {
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const int r = b + K - 1 - uu;
                        if (r >= 0 && r < K) {
                            acc[b].x = fmaf(c[r].x, x.x, fmaf(-c[r].y, x.y, acc[b].x));
                            acc[b].y = fmaf(c[r].x, x.y, fmaf(c[r].y, x.x, acc[b].y));
                        }
                    }
                }
            };
            const bool live = k < nfreq && live_tile;
            if (live) {
#pragma unroll
                for (int uu = 0; uu < kRingRows; ++uu) row(col0[uu * kCols], uu);
            }
            __syncthreads();   // chunk i read by every thread: its slot takes chunk i + 3
            if (i + 1 < n) issue(i + 3);
            if (live) {
#pragma unroll
                for (int uu = kRingRows; uu < ROWS; ++uu)
                    row(uu < 2 * kRingRows ? col1[(uu - kRingRows) * kCols] : col2[(uu - 2 * kRingRows) * kCols], uu);
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    if (w0 + b < nwires) {
                        if constexpr (KARATSUBA)
                            Y[(int64_t)(w0 + b) * stride + k] = make_float2(k1[b] - k3[b], k1[b] + k2[b]);
                        else
                            Y[(int64_t)(w0 + b) * stride + k] = acc[b];
                    }
                }
            }
        }
        __syncthreads();   // the run's last chunks read before the next run reuses the slots
        t += run;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <int B, bool KS>
cudaError_t launch_tma(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, uint32_t* status,
                       cudaStream_t s) {
    constexpr int K = kMaxRespWires;
    constexpr int ROWS = B + K - 1;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    TmaConvUnits U;
    const int nkblocks = (nfreq + kCols - 1) / kCols;
    U.n = cb.n;
    U.prefix[0] = 0;
    for (int i = 0; i < cb.n; ++i) {
        const cuuint64_t dims[2] = {(cuuint64_t)(2 * stride), (cuuint64_t)cb.nwires[i]};
        const cuuint64_t strides[1] = {(cuuint64_t)(2 * stride * sizeof(float))};
        const cuuint32_t box[2] = {2 * kCols, ROWS};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&U.map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(cb.X[i]), dims,
                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        U.nwires[i] = cb.nwires[i];
        U.Y[i] = cb.Y[i];
        U.Rt[i] = cb.Rt[i];
        U.rows[i] = cb.rows[i];
        U.prefix[i + 1] = U.prefix[i] + nkblocks * ((cb.nwires[i] + B - 1) / B);
    }
    U.epoch = cb.epoch;
    const int total = U.prefix[cb.n];
    if (total <= 0) return cudaSuccess;
    const int smem = 2 * ROWS * kCols * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute((const void*)wire_conv_tma_kernel<K, B, KS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wire_conv_tma_kernel<K, B, KS>, kCols, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms() * per_sm;
    if (grid > total) grid = total;
    wire_conv_tma_kernel<K, B, KS><<<grid, kCols, smem, s>>>(U, nfreq, stride, kw, center, nkblocks, status);
    return cudaGetLastError();
}

template <bool KS>
cudaError_t launch_ring(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, uint32_t* status,
                        cudaStream_t s) {
    constexpr int K = kMaxRespWires;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    TmaConvUnits U;
    const int nkblocks = (nfreq + kCols - 1) / kCols;
    U.n = cb.n;
    U.prefix[0] = 0;
    for (int i = 0; i < cb.n; ++i) {
        const cuuint64_t dims[2] = {(cuuint64_t)(2 * stride), (cuuint64_t)cb.nwires[i]};
        const cuuint64_t strides[1] = {(cuuint64_t)(2 * stride * sizeof(float))};
        const cuuint32_t box[2] = {2 * kCols, kRingRows};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&U.map[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(cb.X[i]), dims,
                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        U.nwires[i] = cb.nwires[i];
        U.Y[i] = cb.Y[i];
        U.Rt[i] = cb.Rt[i];
        U.rows[i] = cb.rows[i];
        U.prefix[i + 1] = U.prefix[i] + nkblocks * ((cb.nwires[i] + kRingRows - 1) / kRingRows);
    }
    U.epoch = cb.epoch;
    const int total = U.prefix[cb.n];
    if (total <= 0) return cudaSuccess;
    const int smem = kRingSlots * kRingRows * kCols * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute((const void*)wire_conv_ring_kernel<K, KS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wire_conv_ring_kernel<K, KS>, kCols, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms() * per_sm;
    if (grid > total) grid = total;
    wire_conv_ring_kernel<K, KS><<<grid, kCols, smem, s>>>(U, nfreq, stride, kw, center, status);
    return cudaGetLastError();
}

// Wire convolution over sub-pitch impact positions (fine rows w * I + i of
// each unit's X), fed by TMA, over the units of a launch: persistent CTAs
// claim tiles (a column block of kCols frequencies x B output wires of one
// unit) from a counter and walk each tile's units of work (tile, impact),
// double-buffering the (B + K - 1)-row tile of the next one while computing
// the current one; impact i of unit u comes through tensor map u * I + i
// (base row i, row pitch I rows), and one set of accumulators per tile sums
// the impacts before Y is stored.  With active-row marks (U.rows[u], one per
// wire) a claimed tile none of whose outputs is live (no marked wire in
// [w0 + c - K_w + 1, w0 + B - 1 + c]) is dropped at once and its Y rows are
// left for the inverse transform to write as zeros; claiming tiles one by
// one over all units keeps the SMs evenly loaded when the live tiles
// cluster.  The CTA claims its next tile before computing the current
// tile's second-to-last impact.  sched[0] is the claim counter and sched[1]
// counts finished CTAs; the last CTA to finish sets both back to zero (they
// start at zero).  Waits are bounded as in the other TMA kernels.
template <int K, int B, int C>
__global__ void __launch_bounds__(C)
wire_conv_impacts_tma_kernel(const __grid_constant__ TmaConvUnits U, int impacts, int nfreq, int64_t stride, int kw,
                             int center, unsigned* sched, uint32_t* status) {
    constexpr int ROWS = B + K - 1;
    constexpr uint32_t TILE_BYTES = ROWS * C * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_claim;
    auto buf = [&](int st) { return reinterpret_cast<const float2*>(smem + (st ? TILE_BYTES : 0u)); };
    const mark_t cur = U.epoch ? read_epoch(U.epoch) : 0ull;
    const int ntiles = U.prefix[U.n];
    struct Tile {
        int u, k0, w0;
    };
    auto decode = [&](int t) {
        int u = 0;
        while (u + 1 < U.n && U.prefix[u + 1] <= t) ++u;
        const int tt = t - U.prefix[u];
        const int nwb = (U.nwires[u] + B - 1) / B;
        return Tile{u, (tt / nwb) * C, (tt % nwb) * B};
    };
    auto issue = [&](int t, int im, int st) {
        const Tile T = decode(t);
        tma_load_tile(smem + (st ? TILE_BYTES : 0u), &U.map[T.u * impacts + im], 2 * T.k0, T.w0 + center - (K - 1),
                      &bar[st], TILE_BYTES);
    };
    // the next live tile (-1: none left); every thread calls it
    auto claim = [&]() -> int {
        for (;;) {
            if (threadIdx.x == 0) s_claim = (int)atomicAdd(&sched[0], 1u);
            __syncthreads();
            const int t = s_claim;
            __syncthreads();   // s_claim read by every thread before the next claim
            if (t >= ntiles) return -1;
            const Tile T = decode(t);
            const mark_t* marks = U.rows[T.u];
            if (!marks) return t;
            if (cta_any_marked(marks, cur, T.w0 + center - kw + 1, T.w0 + B - 1 + center, U.nwires[T.u])) return t;
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    int st = 0;   // buffer of the current unit of work
    float k1[B], k2[B], k3[B];
    int tile = claim(), next = -1;
    if (tile >= 0 && threadIdx.x == 0) issue(tile, 0, st);
    for (int im = 0; tile >= 0;) {
        if (im == (impacts > 1 ? impacts - 2 : 0)) next = claim();
        const int tn = im + 1 < impacts ? tile : next;
        const int imn = im + 1 < impacts ? im + 1 : 0;
        const bool inflight_next = tn >= 0;
        if (inflight_next && threadIdx.x == 0) issue(tn, imn, st ^ 1);
        const Tile T = decode(tile);
        const int k = T.k0 + threadIdx.x;
        const float2* __restrict__ Rt = static_cast<const float2*>(U.Rt[T.u]);
        // this impact's taps (loaded while the tile lands)
        float cc[K], cm[K], cp[K];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const float2 v = (r < kw && k < nfreq) ? __ldg(&Rt[((int64_t)im * kw + r) * stride + k])
                                                   : make_float2(0.f, 0.f);
            cc[r] = v.x;
            cm[r] = v.y - v.x;
            cp[r] = v.x + v.y;
        }
        if (im == 0) {
#pragma unroll
            for (int b = 0; b < B; ++b) k1[b] = k2[b] = k3[b] = 0.f;
        }
        const bool ok = mbar_wait(&bar[st], parity[st]);
        parity[st] ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(status, WS_DEV_TIMEOUT);
            if (inflight_next) mbar_wait(&bar[st ^ 1], parity[st ^ 1]);
            break;
        }
        const float2* col = buf(st) + threadIdx.x;
        if (k < nfreq) {
#pragma unroll
            for (int uu = 0; uu < ROWS; ++uu) {
                const float2 x = col[uu * C];
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
            if (im == impacts - 1) {
                float2* __restrict__ Y = static_cast<float2*>(U.Y[T.u]);
                const int nw = U.nwires[T.u];
#pragma unroll
                for (int b = 0; b < B; ++b)
                    if (T.w0 + b < nw) Y[(int64_t)(T.w0 + b) * stride + k] = make_float2(k1[b] - k3[b], k1[b] + k2[b]);
            }
        }
        __syncthreads();   // buffer st is free for the copy issued next iteration
        st ^= 1;
        tile = tn;
        im = imn;
    }
    // the last CTA out resets the claim counter for the next launch (every
    // CTA has made its final claim before it counts itself out)
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&sched[1], 1u) == gridDim.x - 1) {
            sched[0] = 0u;
            sched[1] = 0u;
            __threadfence();
        }
    }
}

// The bounded-wait path on its own: one CTA waits on an mbarrier that
// expects an arrival nobody makes; after `iters` attempts it gives up,
// records WS_DEV_TIMEOUT and returns (cycles spent into *cycles).
__global__ void bounded_wait_selftest_kernel(uint32_t* status, int iters, unsigned long long* cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long t0 = clock64();
    const bool ok = mbar_wait(&bar, 0u, iters);
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(status, WS_DEV_TIMEOUT);
        if (cycles) *cycles = (unsigned long long)(t1 - t0);
    }
}

}  // namespace

bool tma_available() { return encode_fn() != nullptr; }

// One launch over units [u0, u1) of cb (at most kMaxUnits / I of them, one
// tensor map per unit and impact).
template <int B, int C>
static cudaError_t launch_impacts_tma(const ConvBatch& cb, int u0, int u1, int impacts, int nfreq, int64_t stride,
                                      int kw, int center, unsigned* sched, uint32_t* status, cudaStream_t s) {
    constexpr int K = kMaxRespWires;
    constexpr int ROWS = B + K - 1;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    TmaConvUnits U;
    U.n = u1 - u0;
    U.prefix[0] = 0;
    U.epoch = cb.epoch;
    const int nkblocks = (nfreq + C - 1) / C;
    for (int j = 0; j < U.n; ++j) {
        const int u = u0 + j;
        const int nwires = cb.nwires[u];
        if (nwires <= 0) return cudaErrorInvalidValue;
        U.nwires[j] = nwires;
        U.Y[j] = cb.Y[u];
        U.Rt[j] = cb.Rt[u];
        U.rows[j] = cb.rows[u];
        U.prefix[j + 1] = U.prefix[j] + nkblocks * ((nwires + B - 1) / B);
        for (int i = 0; i < impacts; ++i) {
            // impact i: fine rows i, i + I, i + 2I, ... (one per wire)
            const cuuint64_t dims[2] = {(cuuint64_t)(2 * stride), (cuuint64_t)nwires};
            const cuuint64_t strides[1] = {(cuuint64_t)(2 * stride * sizeof(float)) * (cuuint64_t)impacts};
            const cuuint32_t box[2] = {2 * C, ROWS};
            const cuuint32_t estr[2] = {1, 1};
            const CUresult r = enc(&U.map[j * impacts + i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                   const_cast<float2*>(static_cast<const float2*>(cb.X[u])) + (int64_t)i * stride,
                                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    const int ntiles = U.prefix[U.n];
    if (ntiles <= 0) return cudaSuccess;
    const int smem = 2 * ROWS * C * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute((const void*)wire_conv_impacts_tma_kernel<K, B, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wire_conv_impacts_tma_kernel<K, B, C>, C, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms() * per_sm;
    if (grid > ntiles) grid = ntiles;
    wire_conv_impacts_tma_kernel<K, B, C><<<grid, C, smem, s>>>(U, impacts, nfreq, stride, kw, center, sched,
                                                                 status);
    return cudaGetLastError();
}

cudaError_t launch_wire_conv_impacts_tma(const ConvBatch& cb, int impacts, int nfreq, int64_t stride, int kw,
                                         int center, unsigned* sched, uint32_t* status, cudaStream_t s, int variant) {
    if (impacts < 1 || impacts > kMaxUnits || nfreq <= 0 || variant < 0 || variant >= kImpactConvVariants ||
        !sched || !status || cb.n < 0 || cb.n > kMaxUnits)
        return cudaErrorInvalidValue;
    for (int u = 0; u < cb.n; ++u)
        if (cb.rows[u] && !cb.epoch) return cudaErrorInvalidValue;
    const int per_launch = kMaxUnits / impacts;   // tensor maps of a launch: units x impacts
    for (int u0 = 0; u0 < cb.n; u0 += per_launch) {
        const int u1 = u0 + per_launch < cb.n ? u0 + per_launch : cb.n;
        auto run = [&](auto launch) { return launch(cb, u0, u1, impacts, nfreq, stride, kw, center, sched, status, s); };
        cudaError_t e;
        switch (variant) {
            case 1: e = run(launch_impacts_tma<32, 128>); break;
            case 2: e = run(launch_impacts_tma<16, 64>); break;
            case 3: e = run(launch_impacts_tma<32, 64>); break;
            default: e = run(launch_impacts_tma<16, 128>);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bounded_wait_selftest(uint32_t* status, int iters, unsigned long long* cycles, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(status, iters, cycles);
    return cudaGetLastError();
}

cudaError_t launch_wire_conv_tma(const ConvBatch& cb, int nfreq, int64_t stride, int kw, int center, int variant,
                                 uint32_t* status, cudaStream_t s) {
    if (cb.n <= 0 || nfreq <= 0) return cudaSuccess;
    switch (variant) {
        case 1: return launch_tma<16, true>(cb, nfreq, stride, kw, center, status, s);
        case 2: return launch_tma<8, false>(cb, nfreq, stride, kw, center, status, s);
        case 3: return launch_tma<8, true>(cb, nfreq, stride, kw, center, status, s);
        case 4: return launch_ring<false>(cb, nfreq, stride, kw, center, status, s);
        case 5: return launch_ring<true>(cb, nfreq, stride, kw, center, status, s);
        default: return launch_tma<16, false>(cb, nfreq, stride, kw, center, status, s);
    }
}

}  // namespace ws
