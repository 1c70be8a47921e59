// Resolution control (Sec. 5): integer-factor downsampling of frames before
// encoding (2x or 3x of 1080p in the paper). Each output pixel is the mean of
// the s x s input block it covers (area filter, blocks anchored at the
// top-left corner, floor(H/s) x floor(W/s) outputs).
//
// The result is rounded to its output type, so the mean is computed in
// float32 in a fixed order: float input summed row by row, left to right, each
// addition rounded, then one division by s*s; uint8 input summed exactly as
// integers, divided by s*s and mapped to [-1, 1] as m / 127.5 - 1. The
// explicitly rounded intrinsics keep the compiler from contracting the steps.
// Bandwidth-bound. A block takes one output row (or a chunk of it): it stages
// the s input row segments it covers in shared memory with 16-byte loads (only
// a segment's unaligned head and tail go byte by byte), then each thread forms
// output elements (consecutive threads on consecutive channels and pixels,
// 32-bit index arithmetic) from shared memory and stores them coalesced.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace tok {

namespace {

template <typename T>
__device__ __forceinline__ float in_f(T v) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
        return __bfloat162float(v);
    else
        return (float)v;
}

template <typename T>
__device__ __forceinline__ void out_store(T* p, float v) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
        *p = __float2bfloat16_rn(v);
    else
        *p = v;
}

constexpr int BOX_THREADS = 128;
constexpr int BOX_SMEM = 24 * 1024;  // staged input bytes per buffer
constexpr int BOX_STAGES = 2;        // buffers per block: the next job in flight

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Start copying nb bytes from global memory to shared memory at dst + (src mod
// 16), so that both sides share their alignment: the body in asynchronous
// 16-byte copies, the head up to the first 16-byte boundary and the tail with
// plain byte loads (dst is 16-byte aligned with nb + 16 bytes of room).
__device__ __forceinline__ void stage_bytes(char* dst, const char* src, int nb) {
    const int k = (int)((uintptr_t)src & 15);
    dst += k;
    const int head = min(nb, (16 - k) & 15);
    const int n16 = (nb - head) / 16;
    const int tail0 = head + n16 * 16;
    for (int i = threadIdx.x; i < head; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < n16; i += blockDim.x) cp_async16(dst + head + 16 * i, src + head + 16 * i);
    for (int i = tail0 + threadIdx.x; i < nb; i += blockDim.x) dst[i] = src[i];
}

// uint8 RGB frames, s = 2 or 3: one thread forms PX output pixels (4 for s = 3,
// 8 for s = 2) from 32-bit (128-bit) shared-memory words. Rows are summed first in
// 16-bit lanes (each byte spread by byte_perm, three rows in one add; at most
// 3 * 255 per lane), then the s taps of each output element; the exact integer
// sum indexes the value table. Needs the row segments 4-byte (s = 3) or
// 16-byte (s = 2) aligned in shared memory.
template <int S>
struct RgbGroup {
    static constexpr int PX = S == 3 ? 4 : 8;         // output pixels per thread
    static constexpr int NB = PX * S * 3;             // bytes per input row
    static constexpr int NW = NB / 4;                 // 32-bit words per input row
};

template <int S>
__device__ __forceinline__ void rgb_group_sums(const uint8_t* sm, const int* off, int q, int (&acc)[RgbGroup<S>::PX * 3]) {
    using G = RgbGroup<S>;
    uint32_t lo[G::NW], hi[G::NW];
#pragma unroll
    for (int w = 0; w < G::NW; ++w) lo[w] = hi[w] = 0;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const uint32_t* r = reinterpret_cast<const uint32_t*>(sm + off[a] + q * G::NB);
        uint32_t wv[G::NW];
        if constexpr (S == 2) {
#pragma unroll
            for (int i = 0; i < G::NW / 4; ++i) {
                const uint4 v = reinterpret_cast<const uint4*>(r)[i];
                wv[4 * i] = v.x;
                wv[4 * i + 1] = v.y;
                wv[4 * i + 2] = v.z;
                wv[4 * i + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < G::NW; ++i) wv[i] = r[i];
        }
#pragma unroll
        for (int w = 0; w < G::NW; ++w) {
            lo[w] += __byte_perm(wv[w], 0u, 0x4140);  // bytes 0, 1 -> 16-bit lanes
            hi[w] += __byte_perm(wv[w], 0u, 0x4342);  // bytes 2, 3
        }
    }
#pragma unroll
    for (int j = 0; j < G::PX; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int t = 0;
#pragma unroll
            for (int b = 0; b < S; ++b) {
                const int p = (j * S + b) * 3 + c;  // byte position in the row segment
                const uint32_t word = (p & 2) ? hi[p >> 2] : lo[p >> 2];
                t += (p & 1) ? (int)(word >> 16) : (int)(word & 0xffffu);
            }
            acc[j * 3 + c] = t;
        }
}

template <typename To, int N>
__device__ __forceinline__ void store_group(To* dst, const float (&v)[N], bool vec) {
    if constexpr (std::is_same<To, __nv_bfloat16>::value) {
        uint32_t w[N / 2];
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t*>(&h);
        }
        if (vec) {
            if constexpr ((N / 2) % 4 == 0) {
#pragma unroll
                for (int i = 0; i < N / 8; ++i)
                    reinterpret_cast<uint4*>(dst)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < N / 4; ++i) reinterpret_cast<uint2*>(dst)[i] = make_uint2(w[2 * i], w[2 * i + 1]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) dst[i] = __float2bfloat16_rn(v[i]);
        }
    } else {
        if (vec) {
#pragma unroll
            for (int i = 0; i < N / 4; ++i)
                reinterpret_cast<float4*>(dst)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) dst[i] = v[i];
        }
    }
}

struct BoxGeo {
    int H, W, C, Ho, Wo, s, CW, nchunk, rstride;
    long long jobs;  // F * Ho * nchunk: (output row, chunk of CW output pixels)
};

// Persistent and pipelined: while the block forms the outputs of one job from
// shared memory, the input rows of its next BOX_STAGES - 1 jobs are in flight.
// S > 0: factor fixed at compile time (unrolled taps); S == 0: runtime s (<= 8).
// CC > 0: channel count fixed at compile time (RGB frames); CC == 0: runtime C.
template <int S, int CC, typename Ti, typename To>
__global__ void __launch_bounds__(BOX_THREADS) box_kernel(const Ti* __restrict__ x, BoxGeo g, To* __restrict__ y) {
    extern __shared__ uint4 box_sm[];
    constexpr bool U8 = std::is_same<Ti, uint8_t>::value;
    constexpr int KMAX = S > 0 ? S : 8;
    const int s = S > 0 ? S : g.s;
    const int C = CC > 0 ? CC : g.C;
    const int bufbytes = g.rstride * s;
    char* buf0 = reinterpret_cast<char*>(box_sm);
    float* table = reinterpret_cast<float*>(buf0 + BOX_STAGES * bufbytes);  // uint8: value of every block sum
    const long long row = (long long)g.W * C;

    auto src_of = [&](long long job, int* cw) -> const Ti* {
        const long long orow = job / g.nchunk;
        const int wo0 = (int)(job - orow * g.nchunk) * g.CW;
        *cw = min(g.CW, g.Wo - wo0);
        const long long f = orow / g.Ho;
        const int ho = (int)(orow - f * g.Ho);
        return x + (((f * g.H + (long long)ho * s) * g.W) + (long long)wo0 * s) * C;
    };
    auto issue = [&](long long job, char* buf) {
        int cw;
        const Ti* src0 = src_of(job, &cw);
        const int nb = cw * s * C * (int)sizeof(Ti);
        for (int a = 0; a < s; ++a)
            stage_bytes(buf + a * g.rstride, reinterpret_cast<const char*>(src0 + a * row), nb);
    };

    if constexpr (U8) {
        const int nt = s * s * 255 + 1;
        for (int v = threadIdx.x; v < nt; v += BOX_THREADS)
            table[v] = __fsub_rn(__fdiv_rn(__fdiv_rn((float)v, (float)(s * s)), 127.5f), 1.0f);
    }
    long long job = blockIdx.x;
    int cur = 0;
#pragma unroll
    for (int k = 0; k < BOX_STAGES - 1; ++k) {
        const long long j = job + (long long)k * gridDim.x;
        if (j < g.jobs) issue(j, buf0 + k * bufbytes);
        cp_async_commit();
    }
    for (; job < g.jobs; job += gridDim.x) {
        const long long nxt = job + (long long)(BOX_STAGES - 1) * gridDim.x;
        const int nb_buf = (cur + BOX_STAGES - 1) % BOX_STAGES;
        if (nxt < g.jobs) issue(nxt, buf0 + nb_buf * bufbytes);
        cp_async_commit();
        cp_async_wait<BOX_STAGES - 1>();  // this job's copies have landed (later jobs' may be in flight)
        __syncthreads();
        int cw;
        const Ti* src0 = src_of(job, &cw);
        const long long orow = job / g.nchunk;
        const int wo0 = (int)(job - orow * g.nchunk) * g.CW;
        To* yr = y + (orow * g.Wo + wo0) * C;
        const char* sm = buf0 + cur * bufbytes;
        // element offset of input row a in the buffer: a * rs + (its source address mod 16) / sizeof(Ti)
        const int rs = g.rstride / (int)sizeof(Ti);
        int off[KMAX];
#pragma unroll
        for (int a = 0; a < KMAX; ++a)
            off[a] = a < s ? a * rs + (int)(((uintptr_t)(src0 + a * row) & 15) / sizeof(Ti)) : 0;
        int e0 = 0;  // elements before e0 were formed by the vector groups
        if constexpr (U8 && CC == 3 && (S == 2 || S == 3)) {
            using G = RgbGroup<S>;
            bool rows_ok = true;
#pragma unroll
            for (int a = 0; a < S; ++a) rows_ok = rows_ok && (off[a] % (S == 2 ? 16 : 4)) == 0;
            if (rows_ok) {
                constexpr int VA = (S == 3 && sizeof(To) == 2) ? 8 : 16;  // alignment of the group's vector stores
                const bool vec = ((uintptr_t)yr % VA) == 0;
                const int ng = cw / G::PX;
                for (int q = threadIdx.x; q < ng; q += BOX_THREADS) {
                    int acc[G::PX * 3];
                    rgb_group_sums<S>(reinterpret_cast<const uint8_t*>(sm), off, q, acc);
                    float v[G::PX * 3];
#pragma unroll
                    for (int i = 0; i < G::PX * 3; ++i) v[i] = table[acc[i]];
                    store_group<To, G::PX * 3>(yr + q * G::PX * 3, v, vec);
                }
                e0 = ng * G::PX * 3;
            }
        }
        const int ne = cw * C;
        for (int e = e0 + threadIdx.x; e < ne; e += BOX_THREADS) {
            const int wo = e / C, c = e - wo * C;
            const Ti* p = reinterpret_cast<const Ti*>(sm) + wo * s * C + c;
            float v;
            if constexpr (U8) {
                int acc = 0;  // exact: at most 64 * 255
#pragma unroll
                for (int a = 0; a < KMAX; ++a) {
                    if (a >= s) break;
#pragma unroll
                    for (int b = 0; b < KMAX; ++b) {
                        if (b >= s) break;
                        acc += p[off[a] + b * C];
                    }
                }
                v = table[acc];
            } else {
                float acc = 0.f;  // row by row, left to right, each addition rounded
#pragma unroll
                for (int a = 0; a < KMAX; ++a) {
                    if (a >= s) break;
#pragma unroll
                    for (int b = 0; b < KMAX; ++b) {
                        if (b >= s) break;
                        acc = __fadd_rn(acc, in_f(p[off[a] + b * C]));
                    }
                }
                v = __fdiv_rn(acc, (float)(s * s));
            }
            out_store(yr + e, v);
        }
        __syncthreads();  // the buffer is refilled BOX_STAGES jobs later
        cur = cur + 1 == BOX_STAGES ? 0 : cur + 1;
    }
    cp_async_wait<0>();
}

int box_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
    }
    return n;
}

template <int S, int CC, typename Ti, typename To>
int launch_box_s(const Ti* x, const BoxGeo& g, size_t smem, To* y, cudaStream_t st) {
    auto k = box_kernel<S, CC, Ti, To>;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return (int)cudaGetLastError();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BOX_THREADS, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long grid = std::min<long long>(g.jobs, (long long)box_sms() * per_sm);
    k<<<(unsigned)grid, BOX_THREADS, smem, st>>>(x, g, y);
    return (int)cudaGetLastError();
}

template <typename Ti, typename To>
int launch_box(const Ti* x, long long F, int H, int W, int C, int s, To* y, cudaStream_t st) {
    BoxGeo g;
    g.H = H;
    g.W = W;
    g.C = C;
    g.s = s;
    g.Ho = H / s;
    g.Wo = W / s;
    if (F * g.Ho * g.Wo * C <= 0) return 0;
    // output pixels per job: the whole row if its s input rows fit, else a multiple of 16
    const int per_px = s * s * C * (int)sizeof(Ti);
    int CW = BOX_SMEM / per_px;
    if (CW >= g.Wo)
        CW = g.Wo;
    else
        CW = CW >= 16 ? CW / 16 * 16 : std::max(CW, 1);
    g.CW = CW;
    g.nchunk = (g.Wo + CW - 1) / CW;
    g.rstride = (CW * s * C * (int)sizeof(Ti) + 15) / 16 * 16 + 16;  // + room for the alignment shift
    g.jobs = F * g.Ho * g.nchunk;
    const bool u8 = std::is_same<Ti, uint8_t>::value;
    const size_t smem = (size_t)BOX_STAGES * g.rstride * s + (u8 ? (size_t)(s * s * 255 + 1) * 4 : 0);
    if (smem > 200 * 1024) return (int)cudaErrorInvalidConfiguration;
    if (C == 3 && s == 2) return launch_box_s<2, 3, Ti, To>(x, g, smem, y, st);
    if (C == 3 && s == 3) return launch_box_s<3, 3, Ti, To>(x, g, smem, y, st);
    return launch_box_s<0, 0, Ti, To>(x, g, smem, y, st);
}

template <typename Ti>
int launch_box_out(const Ti* x, long long F, int H, int W, int C, int s, bool out_bf16, void* y, cudaStream_t st) {
    if (out_bf16) return launch_box<Ti, __nv_bfloat16>(x, F, H, W, C, s, static_cast<__nv_bfloat16*>(y), st);
    return launch_box<Ti, float>(x, F, H, W, C, s, static_cast<float*>(y), st);
}

}  // namespace

// in_type: 0 uint8, 1 bf16, 2 fp32; s in 1..8 (the runtime form covers s <= 8)
int launch_downsample(int in_type, const void* x, long long F, int H, int W, int C, int s, bool out_bf16, void* y,
                      cudaStream_t st) {
    switch (in_type) {
        case 0: return launch_box_out(static_cast<const uint8_t*>(x), F, H, W, C, s, out_bf16, y, st);
        case 1: return launch_box_out(static_cast<const __nv_bfloat16*>(x), F, H, W, C, s, out_bf16, y, st);
        default: return launch_box_out(static_cast<const float*>(x), F, H, W, C, s, out_bf16, y, st);
    }
}

}  // namespace tok
