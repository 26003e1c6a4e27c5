// ws_convolve_noalloc: the convolution for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running inside another framework's allocator, plug-ins loaded into a
// process whose memory is reserved up front, or setups that forbid any new
// device allocation after start-up.  This entry point needs nothing but the
// caller's input and output buffers: its scratch (twiddles, response
// spectrum and the two row spectra) lives in one file-scope __device__ array
// of kStaticScratchBytes, which every GPU that loads the library holds until
// the process exits.
//
// The array's name is only a host-side stand-in in host code, so the first
// call on each device (with that device current) looks up its device address
// with cudaGetSymbolAddress and caches it; that first call should therefore
// come before any stream capture.  All calls share the one array and it
// keeps the last call's contents; calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ws_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of g_scratch on the current device (looked up once).
ws_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ws::record_cuda_error(e, "ws_convolve_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return WS_ERR_UNSUPPORTED_SIZE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return ws::record_cuda_error(e, "ws_convolve_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return WS_OK;
}

}  // namespace

extern "C" ws_status ws_convolve_noalloc(const ws_plane_desc* desc, const float* response_dev,
                                         const float* grid_dev, float* out_dev, void* stream) {
    if (!desc || !response_dev || !grid_dev || !out_dev) return WS_ERR_INVALID_ARG;
    if (((uintptr_t)response_dev | (uintptr_t)grid_dev | (uintptr_t)out_dev) & 3) return WS_ERR_INVALID_ARG;
    if (desc->impacts > 1) return WS_ERR_UNSUPPORTED_SIZE;   // one response for the whole pitch only
    ws::FftPlan plan;
    int nfreq = 0, fstride = 0;
    ws_status st = ws::conv_plan(desc, &plan, &nfreq, &fstride);
    if (st != WS_OK) return st;
    const size_t tw_bytes = align256(sizeof(float2) * (size_t)plan.L);
    const size_t rt_bytes = align256(sizeof(float2) * (size_t)desc->resp_nwires * fstride);
    const size_t sp_bytes = align256(sizeof(float2) * (size_t)desc->nwires * fstride);
    if (tw_bytes + rt_bytes + 2 * sp_bytes > kStaticScratchBytes) return WS_ERR_WORKSPACE;
    void* base = nullptr;
    st = scratch_address(&base);
    if (st != WS_OK) return st;
    char* b = (char*)base;
    float2* tw = (float2*)b;
    float2* Rt = (float2*)(b + tw_bytes);
    float2* X = (float2*)(b + tw_bytes + rt_bytes);
    float2* Y = (float2*)(b + tw_bytes + rt_bytes + sp_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = ws::launch_twiddles(tw, plan, s);
    if (e == cudaSuccess)
        e = ws::launch_fwd_rows(plan, tw, response_dev, desc->resp_nwires, desc->resp_nticks, desc->resp_nticks, Rt,
                                fstride, nfreq, 1.0f / (float)plan.L, s);
    if (e == cudaSuccess)
        e = ws::launch_fwd_rows(plan, tw, grid_dev, desc->nwires, desc->nticks, desc->nticks, X, fstride, nfreq,
                                1.0f, s);
    if (e == cudaSuccess)
        e = ws::launch_wire_conv(X, Y, Rt, desc->nwires, nfreq, fstride, desc->resp_nwires, desc->resp_wire_center,
                                 desc->conv_mode == WS_CONV_CIRCULAR, s);
    if (e == cudaSuccess)
        e = ws::launch_inv_rows(plan, tw, Y, desc->nwires, fstride, nfreq, out_dev, desc->nticks, desc->nticks, s);
    if (e != cudaSuccess) return ws::record_cuda_error(e, "ws_convolve_noalloc");
    return WS_OK;
}
