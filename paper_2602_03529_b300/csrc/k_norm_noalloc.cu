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
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture. The cache remembers the CUDA context
// it was taken in (its process-unique id), so a call after cudaDeviceReset,
// or in another context of the same device, looks the address up again.
//
// The kernels fully overwrite the part of the scratch they read in the same
// call (every partial triple and every group's statistics are written before
// they are read), so nothing has to be cleared between calls. All calls share
// the one array: two calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it and may return wrong
// results; serialise them on one stream.
#include <cudaTypedefs.h>
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
unsigned long long g_ctx_id[kMaxDevices] = {};  // context the address was looked up in

// Process-unique id of the current CUDA context, or 0 when there is none yet
// (the driver calls are reached through the runtime's entry-point query, as
// the tensor-map encoder is).
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_gn_scratch on the current device: looked up once per
// device and context (the set-up of the first call there).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOK_EDEVICE;
    if (dev < 0 || dev >= kMaxDevices) return TOK_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_context_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gn_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            g_addr[dev] = nullptr;
            return TOK_ECUDA;
        }
        g_addr[dev] = p;
        g_ctx_id[dev] = current_context_id();  // the lookup has made the context current
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
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOK_EDEVICE;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
        cudaGetLastError();
        return TOK_EDEVICE;
    }
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
