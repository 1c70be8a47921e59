// GroupNorm (statistics per sample, group and frame) fused with SiLU.
//
// Three passes over channels-last activations (x: frames x HW x C):
//   gn_partial  : every block reduces one chunk of one frame to per-group
//                 (count, mean, M2) triples. Each thread keeps sums shifted by
//                 the first value it saw (so E[x^2]-E[x]^2 does not cancel),
//                 then the block merges threads with Chan's pairwise update in
//                 a fixed tree order (deterministic, no atomics).
//   gn_finalize : one warp per (frame, group) merges the chunk triples in a
//                 fixed order into mean and 1/sqrt(var + eps).
//   gn_apply    : SiLU((x - mean) * rstd * gamma + beta), 16-byte vectors; a
//                 block pulls its chunk into shared memory with four bulk
//                 copies (64 KB in flight per block, as many as 3 blocks per
//                 SM), then normalises from there.
// The causal tokenizer may not mix frames, hence statistics per frame.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "conv_args.h"
#include "launchers.h"

namespace tok {

namespace {

constexpr int NT = 256;

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int N = 4;
    __device__ static uint4 raw(const float* p) { return *reinterpret_cast<const uint4*>(p); }
    __device__ static void cvt(uint4 q, float (&v)[4]) {
        v[0] = __uint_as_float(q.x); v[1] = __uint_as_float(q.y); v[2] = __uint_as_float(q.z); v[3] = __uint_as_float(q.w);
    }
    __device__ static void load(const float* p, float (&v)[4]) {
        float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ static uint4 raw(const __nv_bfloat16* p) { return *reinterpret_cast<const uint4*>(p); }
    __device__ static void cvt(uint4 q, float (&v)[8]) {
        uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = unpack_bf16x2(u[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static void load(const __nv_bfloat16* p, float (&v)[8]) {
        uint4 q = *reinterpret_cast<const uint4*>(p);
        uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = unpack_bf16x2(u[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static void store(__nv_bfloat16* p, const float (&v)[8]) {
        uint4 q;
        q.x = pack_bf16x2(v[0], v[1]);
        q.y = pack_bf16x2(v[2], v[3]);
        q.z = pack_bf16x2(v[4], v[5]);
        q.w = pack_bf16x2(v[6], v[7]);
        *reinterpret_cast<uint4*>(p) = q;
    }
};

using Triple = GnTriple;

__device__ __forceinline__ Triple merge(Triple a, Triple b) {
    if (b.n == 0.f) return a;
    if (a.n == 0.f) return b;
    Triple r;
    r.n = a.n + b.n;
    const float d = b.mean - a.mean;
    const float fb = b.n / r.n;
    r.mean = a.mean + d * fb;
    r.m2 = a.m2 + b.m2 + d * d * a.n * fb;
    return r;
}

// One input of a grouped GroupNorm launch (clips or stream chunks of one
// layer). Blocks are numbered problem after problem (blk_end: running totals
// of frames * S), finalize warps likewise over (frame, group) rows.
template <typename T>
struct GnProb {
    const T* x;
    T* y;
    long long frames, vpf;  // frames, 16-byte vectors per frame
    int vpt, S;             // vectors per thread, chunks per frame (apply and statistics passes)
    Triple* part;           // (frames, Sp, G) statistics slots
    int Sp;                 // slots per frame: S, or those of the producing conv
    int pre;                // the producing conv reduced the slots (no statistics pass)
    float2* stats;          // (frames, G): mean, rstd
    long long blk_end, row_end;
};

template <typename T, int MAXP>
struct GnBatch {
    GnProb<T> p[MAXP];
    int count;
};

template <typename T, int MAXP>
__device__ __forceinline__ int gn_block_problem(const GnBatch<T, MAXP>& B, long long b, long long* local) {
    int p = 0;
    if constexpr (MAXP > 1)
        while (p + 1 < B.count && b >= B.p[p].blk_end) ++p;
    *local = p ? b - B.p[p - 1].blk_end : b;
    return p;
}

// NGV = groups covered by one vector of V channels (V / channels-per-group,
// or 1 when a group spans one or more whole vectors).
template <typename T, int NGV, int MAXP>
__global__ void __launch_bounds__(NT) gn_partial_kernel(const __grid_constant__ GnBatch<T, MAXP> B, int C, int G) {
    constexpr int V = Vec<T>::N;
    constexpr int EPG = V / NGV;  // elements of my vector per group slot
    __shared__ Triple red[NT][NGV];
    long long lb;
    const GnProb<T>& P = B.p[gn_block_problem(B, blockIdx.x, &lb)];
    if (P.pre) return;  // statistics from the producing conv
    const long long vec_per_frame = P.vpf;
    const int S = P.S, vpt = P.vpt;
    const int frame = (int)(lb / S), chunk = (int)(lb % S), tid = threadIdx.x;
    Triple* __restrict__ part = P.part;
    const int vpv = C / V;  // vectors per voxel (a power of two dividing NT)
    const T* base = P.x + (long long)frame * vec_per_frame * V;
    float K[NGV], s[NGV], q[NGV];
    float cnt = 0.f;
#pragma unroll
    for (int k = 0; k < NGV; ++k) K[k] = s[k] = q[k] = 0.f;
    const long long v0 = (long long)chunk * NT * vpt;
    for (int i = 0; i < vpt; ++i) {
        const long long vi = v0 + (long long)i * NT + tid;
        if (vi >= vec_per_frame) break;
        float v[V];
        Vec<T>::load(base + vi * V, v);
        if (i == 0) {
#pragma unroll
            for (int k = 0; k < NGV; ++k) K[k] = v[k * EPG];
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const float d = v[j] - K[j / EPG];
            s[j / EPG] += d;
            q[j / EPG] = fmaf(d, d, q[j / EPG]);
        }
        cnt += (float)EPG;
    }
#pragma unroll
    for (int k = 0; k < NGV; ++k) {
        Triple t;
        t.n = cnt;
        t.mean = cnt > 0.f ? K[k] + s[k] / cnt : 0.f;
        t.m2 = cnt > 0.f ? fmaxf(q[k] - s[k] * s[k] / cnt, 0.f) : 0.f;
        red[tid][k] = t;
    }
    __syncthreads();
    // tree over threads holding the same channels (tid, tid + stride, ...)
    for (int stride = NT / 2; stride >= vpv; stride >>= 1) {
        if (tid < stride) {
#pragma unroll
            for (int k = 0; k < NGV; ++k) red[tid][k] = merge(red[tid][k], red[tid + stride][k]);
        }
        __syncthreads();
    }
    // red[p][k] (p < vpv) now covers channels p*V + k*EPG ... ; fold into groups
    const int cg = C / G;
    for (int g = tid; g < G; g += NT) {
        Triple acc = {0.f, 0.f, 0.f};
        if (NGV > 1) {
            const int p = (g * cg) / V, k = ((g * cg) % V) / EPG;
            acc = red[p][k];
        } else {
            const int p0 = (g * cg) / V, np = cg / V;
            for (int p = p0; p < p0 + np; ++p) acc = merge(acc, red[p][0]);
        }
        part[((long long)frame * S + chunk) * G + g] = acc;
    }
}

// One warp per (frame, group): lanes merge chunks lane, lane + 32, ... in
// chunk order, then a fixed shuffle tree merges the lanes (lane i takes lane
// i + o), so the statistics are the same on every run.
template <typename T, int MAXP>
__global__ void gn_finalize_kernel(const __grid_constant__ GnBatch<T, MAXP> B, int G, float eps) {
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    int p = 0;
    if constexpr (MAXP > 1)
        while (p + 1 < B.count && wid >= B.p[p].row_end) ++p;
    if (wid >= B.p[p].row_end) return;
    const GnProb<T>& P = B.p[p];
    const long long row = p ? wid - B.p[p - 1].row_end : wid;
    const long long frame = row / G;
    const int g = (int)(row % G), S = P.Sp;
    Triple acc = {0.f, 0.f, 0.f};
    for (int c = lane; c < S; c += 32) acc = merge(acc, P.part[(frame * S + c) * G + g]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Triple b;
        b.n = __shfl_down_sync(0xffffffffu, acc.n, o);
        b.mean = __shfl_down_sync(0xffffffffu, acc.mean, o);
        b.m2 = __shfl_down_sync(0xffffffffu, acc.m2, o);
        if (lane + o < 32) acc = merge(acc, b);
    }
    if (lane == 0) P.stats[row] = make_float2(acc.mean, rsqrtf(acc.m2 / fmaxf(acc.n, 1.f) + eps));
}

// The chunk of a block (NT * GN_VPT_MAX 16-byte vectors at most) arrives in
// GN_SEGS bulk copies of at most GN_SEG_BYTES, each on its own mbarrier, so that
// normalising the first segment overlaps the arrival of the others.
constexpr int GN_VPT_MAX = 16, GN_SEGS = 4;
constexpr int GN_SEG_BYTES = NT * GN_VPT_MAX * 16 / GN_SEGS;
constexpr int GN_APPLY_SMEM = GN_SEGS * GN_SEG_BYTES;

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

template <typename T, bool FAST, int MAXP>
__global__ void __launch_bounds__(NT) gn_apply_kernel(const __grid_constant__ GnBatch<T, MAXP> B, int C, int G,
                                                      const float* __restrict__ gamma,
                                                      const float* __restrict__ beta, int* status,
                                                      unsigned long long wait_ns) {
    constexpr int V = Vec<T>::N;
    extern __shared__ __align__(128) uint8_t seg[];  // GN_SEGS x GN_SEG_BYTES
    __shared__ uint64_t bar[GN_SEGS];
    long long lb;
    const GnProb<T>& P = B.p[gn_block_problem(B, blockIdx.x, &lb)];
    const long long vec_per_frame = P.vpf;
    const int vpt = P.vpt;
    const int frame = (int)(lb / P.S), chunk = (int)(lb % P.S), tid = threadIdx.x;
    const long long v0 = (long long)chunk * NT * vpt;
    const long long bytes = min((long long)NT * vpt, vec_per_frame - v0) * 16;
    const long long fo = ((long long)frame * vec_per_frame + v0) * V;  // first element of the chunk
    const T* __restrict__ x = P.x + fo;
    T* __restrict__ y = P.y + fo;
    if (tid == 0) {
        for (int sg = 0; sg < GN_SEGS; ++sg) mbar_init(&bar[sg], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int sg = 0; sg < GN_SEGS; ++sg) {
            const long long b = min((long long)GN_SEG_BYTES, bytes - (long long)sg * GN_SEG_BYTES);
            if (b <= 0) break;
            mbar_arrive_expect_tx(&bar[sg], (uint32_t)b);
            bulk_copy_g2s(seg + sg * GN_SEG_BYTES, x + (long long)sg * (GN_SEG_BYTES / 16) * V, (uint32_t)b,
                          &bar[sg]);
        }
    }
    // the thread's channels: vector i of the chunk holds channels (i % vpv) * V ..,
    // and every vector this thread touches has i = tid (mod NT), NT a multiple of vpv
    const int cg = C / G;
    const int vpv = C / V;
    const int c0 = (tid % vpv) * V;
    float sc[V], sh[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int c = c0 + j;
        const float2 st = P.stats[(long long)frame * G + c / cg];
        const float ga = gamma ? gamma[c] : 1.f;
        sc[j] = st.y * ga;
        sh[j] = (beta ? beta[c] : 0.f) - st.x * st.y * ga;
    }
    for (int sg = 0; sg < GN_SEGS; ++sg) {
        const long long b = min((long long)GN_SEG_BYTES, bytes - (long long)sg * GN_SEG_BYTES);
        if (b <= 0) break;
        if (!mbar_wait(&bar[sg], 0, status, wait_ns)) return;
        const uint4* q = reinterpret_cast<const uint4*>(seg + sg * GN_SEG_BYTES);
        const int n = (int)(b / 16), i0 = sg * (GN_SEG_BYTES / 16);
        for (int i = tid; i < n; i += NT) {
            float v[V];
            Vec<T>::cvt(q[i], v);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float h = fmaf(v[j], sc[j], sh[j]);
                v[j] = FAST ? silu_fast(h) : silu_exact(h);
            }
            Vec<T>::store(y + (long long)(i0 + i) * V, v);
        }
    }
}

// A block covers NT x 16 vectors of one frame (64 KB of BF16): the number of
// chunks of a frame grows with the frame's size and never depends on how many
// frames the launch holds, so a frame's statistics are summed in the same
// order whether it is normalised as part of a whole clip or of a streaming
// chunk, and a 4-frame chunk still fills the GPU with blocks.
constexpr int GN_VPT = 16;
static_assert(GN_VPT <= GN_VPT_MAX, "the apply pass stages a whole chunk in shared memory");
void gn_plan(long long frames, long long vec_per_frame, int num_sms, int* vpt, int* S) {
    (void)frames;
    (void)num_sms;
    *vpt = GN_VPT;
    *S = (int)std::max<long long>(1, (vec_per_frame + (long long)NT * GN_VPT - 1) / ((long long)NT * GN_VPT));
}

}  // namespace

// Where a forward launch left the (mean, rstd) of every (frame, group) in its scratch.
float2* gn_stats_of_scratch(void* scratch, long long frames, long long HW, int C, int G, int vec) {
    int vpt, S;
    gn_plan(frames, HW * C / vec, 0, &vpt, &S);
    Triple* own = static_cast<Triple*>(scratch);
    return reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(own + frames * S * G) + 15) & ~uintptr_t(15));
}

size_t gn_scratch_bytes(long long frames, long long HW, int C, int G, int num_sms, int vec) {
    int vpt, S;
    gn_plan(frames, HW * C / vec, num_sms, &vpt, &S);
    return (size_t)frames * S * G * sizeof(Triple) + (size_t)frames * G * sizeof(float2) + 256;
}

namespace {

// Plan a batch: per-problem chunking, scratch carving, block numbering.
// pre: an item's precomputed statistics (GnItem::part), where it has them, are used
// instead of the statistics pass, item by item
template <typename T, int MAXP>
bool gn_batch(const GnItem<T>* items, int count, int C, int G, GnBatch<T, MAXP>* B, long long* blocks,
              long long* rows, bool pre = false) {
    constexpr int V = Vec<T>::N;
    memset(B, 0, sizeof(*B));
    B->count = count;
    long long nb = 0, nr = 0;
    for (int p = 0; p < count; ++p) {
        GnProb<T>& P = B->p[p];
        P.x = items[p].x;
        P.y = items[p].y;
        P.frames = items[p].frames;
        P.vpf = items[p].HW * C / V;
        gn_plan(P.frames, P.vpf, 0, &P.vpt, &P.S);
        Triple* own = static_cast<Triple*>(items[p].scratch);
        P.pre = pre && items[p].part != nullptr && items[p].part_S > 0 ? 1 : 0;
        P.part = P.pre ? const_cast<Triple*>(items[p].part) : own;
        P.Sp = P.pre ? items[p].part_S : P.S;
        P.stats = reinterpret_cast<float2*>(
            (reinterpret_cast<uintptr_t>(own + P.frames * P.S * G) + 15) & ~uintptr_t(15));
        nb += P.frames * P.S;
        nr += P.frames * G;
        P.blk_end = nb;
        P.row_end = nr;
    }
    *blocks = nb;
    *rows = nr;
    return nb > 0;
}

template <typename T, int MAXP>
int gn_stats_batch(const GnBatch<T, MAXP>& B, long long blocks, long long rows, int C, int G, float eps,
                   cudaStream_t stream, bool pre = false) {
    constexpr int V = Vec<T>::N;
    const int cg = C / G;
    const int ngv = cg >= V ? 1 : V / cg;
    // the statistics pass, unless every item has its statistics (its blocks of such
    // items return at once)
    bool all_pre = pre;
    for (int p = 0; p < B.count; ++p) all_pre = all_pre && B.p[p].pre;
    if (!all_pre) switch (ngv) {
        case 1: gn_partial_kernel<T, 1, MAXP><<<(unsigned)blocks, NT, 0, stream>>>(B, C, G); break;
        case 2: gn_partial_kernel<T, 2, MAXP><<<(unsigned)blocks, NT, 0, stream>>>(B, C, G); break;
        case 4: gn_partial_kernel<T, 4, MAXP><<<(unsigned)blocks, NT, 0, stream>>>(B, C, G); break;
        default: return (int)cudaErrorInvalidValue;
    }
    gn_finalize_kernel<T, MAXP><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, stream>>>(B, G, eps);
    return 0;
}

template <typename T, bool FAST, int MAXP>
int gn_apply_launch(const GnBatch<T, MAXP>& B, long long blocks, int C, int G, const float* gamma, const float* beta,
                    int* status, cudaStream_t stream) {
    static std::atomic<unsigned long long> done{0};
    if (smem_attr_once(gn_apply_kernel<T, FAST, MAXP>, GN_APPLY_SMEM, done) != cudaSuccess)
        return (int)cudaGetLastError();
    gn_apply_kernel<T, FAST, MAXP><<<(unsigned)blocks, NT, GN_APPLY_SMEM, stream>>>(B, C, G, gamma, beta, status,
                                                                                   2000000000ull);
    return (int)cudaGetLastError();
}

template <typename T, int MAXP>
int gn_silu_batch(const GnItem<T>* items, int count, int C, int G, const float* gamma, const float* beta, float eps,
                  bool fast, cudaStream_t stream, int* status) {
    GnBatch<T, MAXP> B;
    long long blocks, rows;
    if (!gn_batch(items, count, C, G, &B, &blocks, &rows, true)) return 0;
    if (const int e = gn_stats_batch(B, blocks, rows, C, G, eps, stream, true)) return e;
    return fast ? gn_apply_launch<T, true, MAXP>(B, blocks, C, G, gamma, beta, status, stream)
                : gn_apply_launch<T, false, MAXP>(B, blocks, C, G, gamma, beta, status, stream);
}

}  // namespace

// Every item: x, y (frames, HW, C) channels-last, y may alias x; scratch of at
// least gn_scratch_bytes(...) for that item. Requirements: C % V == 0, (C/V)
// a power of two dividing 256, C/G >= 2, 16-byte aligned tensors. One launch
// per pass over all items (at most kMaxConvGroup).
template <typename T>
int launch_gn_silu_group(const GnItem<T>* items, int count, int C, int G, const float* gamma, const float* beta,
                         float eps, bool fast, cudaStream_t stream, int* status) {
    if (count < 1 || count > kMaxConvGroup) return (int)cudaErrorInvalidValue;
    return count == 1 ? gn_silu_batch<T, 1>(items, 1, C, G, gamma, beta, eps, fast, stream, status)
                      : gn_silu_batch<T, kMaxConvGroup>(items, count, C, G, gamma, beta, eps, fast, stream, status);
}

template <typename T>
int launch_gn_silu(const T* x, T* y, long long frames, long long HW, int C, int G, const float* gamma,
                   const float* beta, float eps, void* scratch, int num_sms, bool fast, cudaStream_t stream,
                   int* status) {
    (void)num_sms;
    GnItem<T> it{x, y, frames, HW, scratch};
    return launch_gn_silu_group<T>(&it, 1, C, G, gamma, beta, eps, fast, stream, status);
}

// The apply pass alone, with the (mean, rstd) an earlier launch over the same
// tensor shape left in `scratch` (the training backward rebuilds a block's
// normalised activations from its kept input and statistics): the same
// chunking and arithmetic as that launch's apply pass, so the result is
// bitwise the same.
template <typename T>
int launch_gn_apply_kept(const T* x, T* y, long long frames, long long HW, int C, int G, const float* gamma,
                         const float* beta, void* scratch, bool fast, cudaStream_t stream, int* status) {
    GnItem<T> it{x, y, frames, HW, scratch};
    GnBatch<T, 1> B;
    long long blocks, rows;
    if (!gn_batch(&it, 1, C, G, &B, &blocks, &rows)) return 0;
    return fast ? gn_apply_launch<T, true, 1>(B, blocks, C, G, gamma, beta, status, stream)
                : gn_apply_launch<T, false, 1>(B, blocks, C, G, gamma, beta, status, stream);
}
template int launch_gn_apply_kept<float>(const float*, float*, long long, long long, int, int, const float*,
                                         const float*, void*, bool, cudaStream_t, int*);
template int launch_gn_apply_kept<__nv_bfloat16>(const __nv_bfloat16*, __nv_bfloat16*, long long, long long, int,
                                                 int, const float*, const float*, void*, bool, cudaStream_t, int*);

template <typename T>
int launch_gn_stats(const T* x, long long frames, long long HW, int C, int G, float eps, void* scratch, int num_sms,
                    cudaStream_t stream, float2** stats_out, int* vpt_out, int* S_out) {
    (void)num_sms;
    GnItem<T> it{x, nullptr, frames, HW, scratch};
    GnBatch<T, 1> B;
    long long blocks, rows;
    if (!gn_batch(&it, 1, C, G, &B, &blocks, &rows)) return 0;
    if (const int e = gn_stats_batch(B, blocks, rows, C, G, eps, stream)) return e;
    *stats_out = B.p[0].stats;
    *vpt_out = B.p[0].vpt;
    *S_out = B.p[0].S;
    return (int)cudaGetLastError();
}
template int launch_gn_stats<float>(const float*, long long, long long, int, int, float, void*, int, cudaStream_t,
                                    float2**, int*, int*);
template int launch_gn_stats<__nv_bfloat16>(const __nv_bfloat16*, long long, long long, int, int, float, void*, int,
                                            cudaStream_t, float2**, int*, int*);

template int launch_gn_silu<float>(const float*, float*, long long, long long, int, int, const float*, const float*,
                                   float, void*, int, bool, cudaStream_t, int*);
template int launch_gn_silu<__nv_bfloat16>(const __nv_bfloat16*, __nv_bfloat16*, long long, long long, int, int,
                                           const float*, const float*, float, void*, int, bool, cudaStream_t, int*);
template int launch_gn_silu_group<float>(const GnItem<float>*, int, int, int, const float*, const float*, float, bool,
                                         cudaStream_t, int*);
template int launch_gn_silu_group<__nv_bfloat16>(const GnItem<__nv_bfloat16>*, int, int, int, const float*,
                                                 const float*, float, bool, cudaStream_t, int*);

}  // namespace tok
