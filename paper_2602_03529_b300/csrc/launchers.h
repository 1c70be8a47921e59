// Host-side launchers of the tokenizer kernels (one translation unit each).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "conv_args.h"

namespace tok {

int launch_conv_tc(const ConvArgs& a, int num_sms, cudaStream_t stream);
int conv_tc_bn(int cout_pad16);
int launch_conv_simt(const ConvArgs& a, cudaStream_t stream);

size_t gn_scratch_bytes(long long frames, long long HW, int C, int G, int num_sms, int vec);
template <typename T>
int launch_gn_silu(const T* x, T* y, long long frames, long long HW, int C, int G, const float* gamma,
                   const float* beta, float eps, void* scratch, int num_sms, bool fast, cudaStream_t stream);

int launch_fsq(const float* z, long long ntok, const FsqConsts& f, int32_t* idx, float* codes, cudaStream_t s);
int launch_dequant(const int32_t* idx, long long ntok, const FsqConsts& f, float* codes, cudaStream_t s);
int launch_drop(const int32_t* idx, int N, int Tq, int Hq, int Wq, unsigned long long thr, uint64_t seed,
                uint64_t stream_id, uint64_t chunk_id, int32_t zero_index, int32_t* out, uint32_t* keep_bits,
                cudaStream_t s);
int launch_pack(const int32_t* idx, const uint32_t* keep_bits, long long rows, int Wq, int32_t* payload,
                int64_t* offs, cudaStream_t s);
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

int launch_timeout_selftest(int* status, unsigned long long limit_ns, cudaStream_t s);

}  // namespace tok
