// GroupNorm+SiLU for callers that cannot allocate device memory.
//
// tok_groupnorm_silu needs a small scratch buffer (per-chunk partial
// statistics and the per-group mean / 1/std) that the caller normally passes
// in. Some callers cannot provide one: code running where cudaMalloc is not
// allowed or not wanted, such as a host callback, a real-time thread that must
// not take the allocator's locks or risk a synchronising allocation, or an
// embedding whose memory budget is fixed up front. For them this file keeps
// the scratch in a fixed-size array in device global memory, declared at file
// scope, which every GPU that loads the library holds until the process exits.
//
// The array's name, used in host code, is only a host-side stand-in for the
// symbol, not a device address: passing it to a kernel would fault or, where
// the GPU can reach host memory, silently use the wrong memory. So the first
// call on each device looks up the real device address with
// cudaGetSymbolAddress (with that device current) and caches it.
//
// The kernels fully overwrite the part of the scratch they read in the same
// call (every partial triple and every group's statistics are written before
// they are read), so nothing has to be cleared between calls. All calls share
// the one array: two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it and may return wrong
// results; serialise them on one stream.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tok.h"
#include "launchers.h"

namespace {

static __device__ __align__(256) unsigned char g_gn_scratch[TOK_GN_NOALLOC_MAX_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_gn_scratch on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOK_EDEVICE;
    if (dev < 0 || dev >= kMaxDevices) return TOK_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gn_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return TOK_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return TOK_OK;
}

}  // namespace

extern "C" int tok_groupnorm_silu_noalloc(int precision, const void* x, int64_t frames, int64_t HW, int C, int G,
                                          const float* gamma, const float* beta, float eps, void* y,
                                          void* stream) {
    if (!x || !y || frames < 1 || HW < 1 || C < 1 || G < 1 || !(eps >= 0.f)) return TOK_EINVAL;
    if (precision != TOK_BF16 && precision != TOK_FP32) return TOK_EINVAL;
    const int V = precision == TOK_BF16 ? 8 : 4;
    const int vpv = C / V;
    if (C % V || C % G || C / G < 2 || G > 64 || vpv > 256 || (vpv & (vpv - 1))) return TOK_ESHAPE;
    const int cg = C / G;
    if (!(cg % V == 0 || V % cg == 0)) return TOK_ESHAPE;
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOK_EDEVICE;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // Problems whose scratch exceeds the fixed array are refused.
    if (tok::gn_scratch_bytes(frames, HW, C, G, nsm, V) > (size_t)TOK_GN_NOALLOC_MAX_SCRATCH_BYTES)
        return TOK_ENOMEM;
    void* scratch = nullptr;
    const int e0 = scratch_address(&scratch);
    if (e0 != TOK_OK) return e0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int e;
    if (precision == TOK_BF16)
        e = tok::launch_gn_silu<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(x), static_cast<__nv_bfloat16*>(y),
                                               frames, HW, C, G, gamma, beta, eps, scratch, nsm, true, s);
    else
        e = tok::launch_gn_silu<float>(static_cast<const float*>(x), static_cast<float*>(y), frames, HW, C, G,
                                       gamma, beta, eps, scratch, nsm, false, s);
    return e ? TOK_ECUDA : TOK_OK;
}
