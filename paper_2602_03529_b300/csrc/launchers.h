// Host-side launchers of the tokenizer kernels (one translation unit each).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "conv_args.h"

namespace tok {

int launch_conv_tc(const ConvArgs& a, int num_sms, cudaStream_t stream);
// one launch over up to kMaxConvGroup inputs of the same layer (k_conv_tc.cu)
ConvRoute conv_route(const ConvArgs& a);
// A stride-1 3x3x3 BF16 head runs in a form in which spatial taps are MMA rows:
// all nine (dh, dw) taps when 9 * Cout <= 128 and Cin >= 256, else the three dw
// taps when Cout <= 16 (conv_tc_taprows gives 9, 3 or 0); its weights are packed for that
// form (launch_pack_weights_taprows) wherever they are packed, and ConvArgs.w_dwm
// carries the form.
int conv_tc_taprows(int Cout, int Cin, int k, int sh, int sw);
int launch_pack_weights_taprows(const float* w, int Cout, int Cin, int rows_out, int tr, __nv_bfloat16* out,
                                cudaStream_t s);
// The launch writes GroupNorm statistics into a.gn_part (a.gn_cg channels per
// group) only where this holds; conv_tc_gn_slots gives the slots per frame.
bool conv_tc_gn_fusable(const ConvArgs& a);
int conv_tc_gn_slots(const ConvArgs& a);
int launch_conv_tc_group(const ConvArgs* as, int count, int num_sms, cudaStream_t stream, int cta_tiles = 0);
// Fused BF16 stem (k_stem_tc.cu) over up to kMaxConvGroup problems of one layer.
// Returns kStemDeclined, having enqueued nothing, where a problem is outside its
// form (Cout 64 or 128, Kpad 128, H even, W % 8 == 0, 16-byte aligned tensors);
// the caller then runs the im2col gather and the 1x1x1 conv instead. With
// gn_part set, the launch writes the GroupNorm statistics of 32 groups of its
// output: stem_tc_gn_slots per frame.
constexpr int kStemDeclined = -2;
bool stem_tc_accepts(const StemArgs* as, int count);
int launch_stem_tc(const StemArgs* as, int count, int num_sms, cudaStream_t stream, int cta_tiles = 0);
int stem_tc_gn_slots(int H, int W);
int conv_tc_bn(int cout_pad16);
int conv_tc_cout_pad(int Cout);  // packed weight rows of a BF16 conv
int launch_conv_simt(const ConvArgs& a, cudaStream_t stream);

size_t gn_scratch_bytes(long long frames, long long HW, int C, int G, int num_sms, int vec);
// One input of a grouped GroupNorm+SiLU launch (k_norm.cu).
template <typename T>
struct GnItem {
    const T* x;
    T* y;
    long long frames, HW;
    void* scratch;  // gn_scratch_bytes(frames, HW, ...) bytes
    // statistics already reduced by the producing conv: (frames, part_S, G) triples;
    // used when every item of a launch has them, else the statistics pass runs
    const GnTriple* part = nullptr;
    int part_S = 0;
};
// status: a context's device status word (bounded waits record a timeout there), or null
template <typename T>
int launch_gn_silu_group(const GnItem<T>* items, int count, int C, int G, const float* gamma, const float* beta,
                         float eps, bool fast, cudaStream_t stream, int* status = nullptr);
template <typename T>
int launch_gn_silu(const T* x, T* y, long long frames, long long HW, int C, int G, const float* gamma,
                   const float* beta, float eps, void* scratch, int num_sms, bool fast, cudaStream_t stream,
                   int* status = nullptr);
// The apply pass alone, with statistics an earlier launch left in `scratch`.
template <typename T>
int launch_gn_apply_kept(const T* x, T* y, long long frames, long long HW, int C, int G, const float* gamma,
                         const float* beta, void* scratch, bool fast, cudaStream_t stream, int* status);

int launch_fsq(const float* z, long long ntok, const FsqConsts& f, int32_t* idx, float* codes, cudaStream_t s);
int launch_dequant(const int32_t* idx, long long ntok, const FsqConsts& f, float* codes, cudaStream_t s);
int launch_drop(const int32_t* idx, int N, int Tq, int Hq, int Wq, unsigned long long thr, uint64_t seed,
                uint64_t stream_id, uint64_t chunk_id, int32_t zero_index, int32_t* out, uint32_t* keep_bits,
                cudaStream_t s);
int launch_pack(const int32_t* idx, const uint32_t* keep_bits, long long rows, int Wq, int32_t* payload,
                int64_t* offs, cudaStream_t s);
int launch_apply_keep(const int32_t* idx, const uint32_t* keep_bits, long long ntok, int Wq, int32_t zero_index,
                      int32_t* out, cudaStream_t s);
int launch_unpack(const int32_t* payload, const int64_t* offs, const uint32_t* keep_bits, const uint8_t* received,
                  long long rows, int Wq, int32_t zero_index, int32_t* out, cudaStream_t s);

int launch_im2col_pixels(const __nv_bfloat16* x, const __nv_bfloat16* hist, const GatherGeo& g, __nv_bfloat16* A,
                         cudaStream_t s);
int launch_im2col_tokens(const int32_t* idx, const int32_t* hist, const GatherGeo& g, const FsqConsts& f,
                         __nv_bfloat16* A, cudaStream_t s);
template <typename T>
int launch_edge_pad(const T* x, long long frames, int H, int W, int Hp, int Wp, int C, T* y, cudaStream_t s);

template <typename T>
int launch_pack_weights(const float* w, int Cout, int K, int Cout_pad, int Kpad, T* out, cudaStream_t s);

int launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t s);

// GroupNorm statistics only: (mean, rstd) per (frame, group) written at *stats
// (inside scratch); vpt / S report the chunking used.
template <typename T>
int launch_gn_stats(const T* x, long long frames, long long HW, int C, int G, float eps, void* scratch, int num_sms,
                    cudaStream_t s, float2** stats, int* vpt, int* S);

// tensor-core weight gradient (k_wgrad_tc.cu)
bool wgrad_tc_ok(const WgradArgs& a);
int launch_wgrad_tc(const __nv_bfloat16* dy, const __nv_bfloat16* x, const WgradArgs& a, float* part,
                    size_t max_floats, float* dw, float* db, int num_sms, int* status, unsigned long long wait_ns,
                    cudaStream_t s, int k_valid = 0);

// similarity-based token selection (k_select.cu)
size_t similarity_workspace_bytes(long long N, int Tp, long long HW);
int launch_similarity_mask(const int32_t* idx_p, const int32_t* idx_i, long long N, int Tp, int Hq, int Wq,
                           const FsqConsts& f, long long k, int32_t zero_index, int32_t* out, uint32_t* keep_bits,
                           float* sim, void* ws, cudaStream_t s);

// pixel residuals (k_residual.cu)
int launch_residual_mean(bool bf16, const void* x, const float* xh, long long N, int Tf, long long E, int window,
                         float theta, float* r, cudaStream_t s);
size_t residual_sparse_workspace_bytes(long long nseg, long long E);
int launch_residual_sparse(const float* r, long long nseg, long long E, int32_t* pos, float* val, int64_t* seg_off,
                           void* ws, cudaStream_t s);
int launch_residual_apply(float* xh, long long N, int Tf, long long E, int window, const int32_t* pos,
                          const float* val, const int64_t* seg_off, long long cap, cudaStream_t s);

// resolution-control downsampling (k_resize.cu); in_type 0 uint8, 1 bf16, 2 fp32
int launch_downsample(int in_type, const void* x, long long F, int H, int W, int C, int s, bool out_bf16, void* y,
                      cudaStream_t st);

// GoP boundary smoothing (k_gop.cu)
int launch_gop_blend(const float* prev, int Tp, const float* curr, float* out, long long N, int T, long long E, int n,
                     cudaStream_t s);
size_t temporal_loss_workspace_bytes(long long N, int n, long long E);
int launch_temporal_loss(const float* xc, const float* xp, long long N, int Tc, int Tp, long long E, int n,
                         float* loss, float* grad, void* ws, cudaStream_t s);

// backward kernels (k_backward.cu)
size_t wgrad_partial_floats(int Cout, int K, int S);
int wgrad_splits(const WgradArgs& a, int num_sms, size_t max_partial_floats);
template <typename T>
int launch_wgrad(const T* dy, const T* x, WgradArgs a, int S, float* part, float* dw, float* db, cudaStream_t s);
size_t gn_bwd_scratch_bytes(long long frames, int S, int C, int G);
float2* gn_stats_of_scratch(void* scratch, long long frames, long long HW, int C, int G, int vec);  // k_norm.cu
template <typename T>
int launch_gn_silu_bwd(const T* x, const T* dy, const float2* stats, const float* gamma, const float* beta,
                       const T* add, long long frames, long long HW, int C, int G, int vpt, int S, void* scratch,
                       float* dgamma, float* dbeta, T* dx, int* status, unsigned long long wait_ns,
                       cudaStream_t s);
// chunking of the GroupNorm backward (k_backward.cu)
int gn_bwd_vectors_per_thread();
int gn_bwd_chunks_per_frame(long long HW, int C, int vec);
template <typename T>
int launch_ste_bwd(const T* dcodes, int Cd, const float* z, const uint32_t* keep_bits, long long ntok, int Wq,
                   const FsqConsts& f, T* dz, int Co, cudaStream_t s);
template <typename T>
int launch_codes(const int32_t* idx, long long ntok, const FsqConsts& f, T* codes, cudaStream_t s);
template <typename Ti, typename To>
int launch_s2d(const Ti* d, int N, int oT, int oH, int oW, int C, int rt, int rh, int rw, int drop_t, int T, int H,
               int W, int Cpad, To* out, cudaStream_t s);
template <typename T>
int launch_zero_insert(const T* dy, int N, int To, int Ho, int Wo, int C, int Tin, int Hin, int Win, int st, int sh,
                       int sw, T* out, cudaStream_t s);
template <typename T>
int launch_mse(const float* xh, const T* x, long long n, float* dxh, float* loss, float* scratch, cudaStream_t s);
// forward rows, adjoint taps and frame-0 adjoint taps of a BF16 3x3x3 conv in one pass (k_backward.cu)
int launch_pack3(const float* w, int Cout, int Cin, int Cout_pad, int Kpad, int rows_pad, int cpad,
                 __nv_bfloat16* fwd, __nv_bfloat16* wt, __nv_bfloat16* wf0, cudaStream_t s);
// One conv's three BF16 layouts (forward rows, adjoint taps, frame-0 adjoint taps)
// as a job of the batched pack: gx x gy x 9 blocks from block0 on.
struct Pack3Job {
    const float* w;
    __nv_bfloat16 *fwd, *wt, *wf0;
    int Cout, Cin, Cout_pad, Kpad, rows_pad, cpad, gx, gy;
    long long block0;
};
Pack3Job pack3_job(const float* w, int Cout, int Cin, int Cout_pad, int Kpad, int rows_pad, int cpad,
                   __nv_bfloat16* fwd, __nv_bfloat16* wt, __nv_bfloat16* wf0, long long block0);
int launch_pack3_batch(const Pack3Job* d_jobs, int njobs, long long blocks, cudaStream_t s);
template <typename T>
int launch_pack_adjoint(const float* w, int Cout, int Cin, int k, int rows_pad, int cpad, int corr, T* out,
                        cudaStream_t s);
int launch_sgd(float* p, const float* g, long long n, float lr, cudaStream_t s);

int launch_timeout_selftest(int* status, unsigned long long limit_ns, cudaStream_t s);

}  // namespace tok
