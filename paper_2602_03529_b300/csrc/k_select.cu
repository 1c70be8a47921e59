// Similarity-based token selection (Sec. 6.3, Eq. 3).
//
// For every P-frame token, the cosine S between its code vector and the
// I-frame token's code vector at the same (sample, h, w); per sample and P
// latent frame the k = floor(rate * H'W') tokens with the largest S are
// dropped (zero code index, packet keep bit cleared), ties going to the lower
// linear index: tau is the (1 - rate)-quantile of S.
//
//   sim_key_kernel : S in float32 with explicitly rounded operations (the
//                    decision is taken on these values: dot and squared norms
//                    summed in channel order, their product, one square root,
//                    one division; -0 made +0), and a 64-bit key that orders
//                    tokens by (S descending, index ascending): the
//                    order-preserving bits of S above the complemented index.
//   select_kernel  : one block per frame finds the k-th largest key by an
//                    MSB-first radix select (8 passes of 8-bit digits, shared
//                    memory histograms); keys are unique, so exactly k keys
//                    are >= it.
//   apply_kernel   : warp per 32 tokens of a row: drop iff key >= threshold,
//                    indices out, keep bits by ballot.
// Frames of up to FUSED_MAX_TOKENS tokens (1080p latents and smaller) take one
// fused kernel instead, one block per frame: index -> digits through a table
// built once per call, S kept in shared memory as its 32-bit order-preserving
// image, a 3-pass radix select (11-bit digits, warp-aggregated histogram
// increments: many tokens share a similarity), the cut among tokens equal to
// the k-th largest S placed by a block scan over positions (lower index
// first), then the drop and the keep bits. The three-kernel form serves
// larger frames.
#include "common.cuh"
#include "conv_args.h"

namespace tok {

namespace {

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__device__ __forceinline__ float code_value(int idx, const FsqConsts& f, int c) {
    const int d = (idx / f.basis[c]) % f.levels[c];
    return __fdiv_rn((float)(d - f.half_w[c]), (float)f.half_w[c]);
}

__global__ void sim_key_kernel(const int32_t* __restrict__ idx_p, const int32_t* __restrict__ idx_i, long long N,
                               int Tp, long long HW, FsqConsts f, unsigned long long* __restrict__ keys,
                               float* __restrict__ sim) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * Tp * HW) return;
    const long long j = t % HW;
    const long long n = t / (HW * Tp);
    const int ip = idx_p[t], ii = idx_i[n * HW + j];
    float dot = 0.f, sp = 0.f, si = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (c < f.nlev) {
            const float p = code_value(ip, f, c), q = code_value(ii, f, c);
            dot = __fadd_rn(dot, __fmul_rn(p, q));
            sp = __fadd_rn(sp, __fmul_rn(p, p));
            si = __fadd_rn(si, __fmul_rn(q, q));
        }
    }
    const float den = __fsqrt_rn(__fmul_rn(sp, si));
    float S = den > 0.f ? __fdiv_rn(dot, den) : 0.f;
    S = __fadd_rn(S, 0.f);  // -0 -> +0: equal similarities must have equal keys
    const uint32_t u = __float_as_uint(S);
    const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    keys[t] = ((unsigned long long)ord << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)j);
    if (sim) sim[t] = S;
}

constexpr int SEL_THREADS = 1024;

// thr[frame] = the k-th largest key of the frame's HW keys (1 <= k <= HW).
__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const unsigned long long* __restrict__ keys,
                                                             long long HW, long long k,
                                                             unsigned long long* __restrict__ thr) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ long long s_rem;
    const unsigned long long* fk = keys + (long long)blockIdx.x * HW;
    if (threadIdx.x == 0) {
        s_prefix = 0ull;
        s_mask = 0ull;
        s_rem = k;
    }
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += SEL_THREADS) hist[i] = 0u;
        __syncthreads();
        const unsigned long long prefix = s_prefix, mask = s_mask;
        for (long long i = threadIdx.x; i < HW; i += SEL_THREADS) {
            const unsigned long long key = fk[i];
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long cum = 0, rem = s_rem;
            int d = 255;
            for (; d > 0; --d) {
                if (cum + (long long)hist[d] >= rem) break;
                cum += hist[d];
            }
            s_rem = rem - cum;
            s_prefix = prefix | ((unsigned long long)d << shift);
            s_mask = mask | (255ull << shift);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) thr[blockIdx.x] = s_prefix;
}

__global__ void apply_kernel(const int32_t* __restrict__ idx_p, const unsigned long long* __restrict__ keys,
                             const unsigned long long* __restrict__ thr, long long rows, int Hq, int Wq,
                             int all_keep, int32_t zero_index, int32_t* __restrict__ out,
                             uint32_t* __restrict__ keep_bits) {
    const int nwords = (Wq + 31) / 32;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (gw >= rows * nwords) return;
    const long long row = gw / nwords;
    const int word = (int)(gw % nwords);
    const int w = word * 32 + lane;
    bool keep = false;
    if (w < Wq) {
        const long long o = row * Wq + w;
        keep = all_keep || keys[o] < thr[row / Hq];
        out[o] = keep ? idx_p[o] : zero_index;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    if (keep_bits && lane == 0) keep_bits[row * nwords + word] = m;
}

constexpr int FS_THREADS = 1024;
constexpr long long FUSED_MAX_TOKENS = 53 * 1024;
constexpr int DIGIT_TAB = 64000;  // table entries: indices below prod(levels) <= 2^31 - 1 are decoded directly

// digit table: entry i = digits of index i, 4 bits per channel (levels <= 16)
__global__ void digit_table_kernel(FsqConsts f, int n, uint32_t* __restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t v = 0;
    for (int c = 0; c < f.nlev; ++c) v |= (uint32_t)((i / f.basis[c]) % f.levels[c]) << (4 * c);
    tab[i] = v;
}

__device__ __forceinline__ uint32_t digits_of(int idx, const FsqConsts& f, const uint32_t* tab, int ntab) {
    if (idx >= 0 && idx < ntab) return tab[idx];
    uint32_t v = 0;
    for (int c = 0; c < f.nlev; ++c) v |= (uint32_t)((idx / f.basis[c]) % f.levels[c]) << (4 * c);
    return v;
}

__global__ void __launch_bounds__(FS_THREADS) select_fused_kernel(
    const int32_t* __restrict__ idx_p, const int32_t* __restrict__ idx_i, const uint32_t* __restrict__ tab, int ntab,
    FsqConsts f, int Tp, int Hq, int Wq, long long k, int32_t zero_index, int32_t* __restrict__ out,
    uint32_t* __restrict__ keep_bits, float* __restrict__ sim) {
    extern __shared__ uint32_t ords[];  // HW order-preserving similarity images
    __shared__ float ctab[8][16];
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t wsum[FS_THREADS / 32];
    __shared__ uint32_t s_prefix, s_mask, s_pos;
    __shared__ long long s_rem;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const long long frame = blockIdx.x, n = frame / Tp;
    const long long HW = (long long)Hq * Wq;
    const int32_t* fp = idx_p + frame * HW;
    const int32_t* fi = idx_i + n * HW;
    for (int i = tid; i < 128; i += FS_THREADS) {
        const int c = i / 16, d = i % 16;
        ctab[c][d] = (c < f.nlev && d < f.levels[c]) ? __fdiv_rn((float)(d - f.half_w[c]), (float)f.half_w[c]) : 0.f;
    }
    __syncthreads();
    // phase 1: similarities
    for (long long j = tid; j < HW; j += FS_THREADS) {
        const uint32_t dp = digits_of(fp[j], f, tab, ntab), di = digits_of(fi[j], f, tab, ntab);
        float dot = 0.f, sp = 0.f, si = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c < f.nlev) {
                const float p = ctab[c][(dp >> (4 * c)) & 15u], q = ctab[c][(di >> (4 * c)) & 15u];
                dot = __fadd_rn(dot, __fmul_rn(p, q));
                sp = __fadd_rn(sp, __fmul_rn(p, p));
                si = __fadd_rn(si, __fmul_rn(q, q));
            }
        }
        const float den = __fsqrt_rn(__fmul_rn(sp, si));
        float S = den > 0.f ? __fdiv_rn(dot, den) : 0.f;
        S = __fadd_rn(S, 0.f);
        const uint32_t u = __float_as_uint(S);
        ords[j] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        if (sim) sim[frame * HW + j] = S;
    }
    if (tid == 0) {
        s_prefix = 0u;
        s_mask = 0u;
        s_rem = k;
    }
    __syncthreads();
    const bool all_drop = k >= HW, none = k <= 0;
    if (!all_drop && !none) {
        // phase 2: the k-th largest similarity image (digits of 11, 11 and 10 bits)
        const int shifts[3] = {21, 10, 0};
        const uint32_t dmasks[3] = {0x7FFu, 0x7FFu, 0x3FFu};
        const long long iters = (HW + FS_THREADS - 1) / FS_THREADS;
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = shifts[pass];
            const uint32_t dm = dmasks[pass];
            for (int i = tid; i < 2048; i += FS_THREADS) hist[i] = 0u;
            __syncthreads();
            const uint32_t prefix = s_prefix, mask = s_mask;
            for (long long it = 0; it < iters; ++it) {
                const long long j = it * FS_THREADS + tid;
                const uint32_t o = j < HW ? ords[j] : 0u;
                const bool act = j < HW && (o & mask) == prefix;
                const uint32_t dig = (o >> shift) & dm;
                const uint32_t am = __ballot_sync(0xffffffffu, act);
                if (act) {
                    const uint32_t same = __match_any_sync(am, dig);
                    if (lane == __ffs(same) - 1) atomicAdd(&hist[dig], (uint32_t)__popc(same));
                }
            }
            __syncthreads();
            if (warp == 0) {
                // digit of the rem-th largest: lane l sums bins [2048 - 64(l+1), 2048 - 64 l),
                // a lane scan finds the lane where the count from the top reaches rem, and
                // that lane walks its bins
                const long long rem = s_rem;
                const int hi = 2048 - 64 * lane;
                long long own = 0;
                for (int b = hi - 1; b >= hi - 64; --b) own += hist[b];
                long long incl = own;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const uint32_t hit = __ballot_sync(0xffffffffu, incl >= rem);
                if (lane == __ffs(hit) - 1) {
                    long long cum = incl - own;
                    int d = hi - 1;
                    for (; d > hi - 64; --d) {
                        if (cum + (long long)hist[d] >= rem) break;
                        cum += hist[d];
                    }
                    s_rem = rem - cum;
                    s_prefix = prefix | ((uint32_t)d << shift);
                    s_mask = mask | (dm << shift);
                }
            }
            __syncthreads();
        }
        // phase 3: among the tokens equal to the k-th largest, the s_rem lowest positions drop
        const uint32_t star = s_prefix;
        const long long per = (HW + FS_THREADS - 1) / FS_THREADS;
        const long long j0 = (long long)tid * per, j1 = j0 + per < HW ? j0 + per : HW;
        uint32_t cnt = 0;
        for (long long j = j0; j < j1; ++j) cnt += ords[j] == star ? 1u : 0u;
        // block exclusive scan of cnt
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += v;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = incl - cnt + (warp > 0 ? wsum[warp - 1] : 0u);
        const long long rem = s_rem;
        if ((long long)before < rem && rem <= (long long)(before + cnt)) {
            long long need = rem - before;
            for (long long j = j0; j < j1; ++j)
                if (ords[j] == star && --need == 0) {
                    s_pos = (uint32_t)j;
                    break;
                }
        }
        __syncthreads();
    }
    // phase 4: drop, indices and keep bits (a warp per 32 tokens of a row)
    const uint32_t star = s_prefix, pos = s_pos;
    const int nwords = (Wq + 31) / 32;
    for (long long rw = warp; rw < (long long)Hq * nwords; rw += FS_THREADS / 32) {
        const int h = (int)(rw / nwords), word = (int)(rw % nwords), w = word * 32 + lane;
        bool keep = false;
        if (w < Wq) {
            const long long j = (long long)h * Wq + w;
            const uint32_t o = ords[j];
            const bool drop = all_drop || (!none && (o > star || (o == star && (uint32_t)j <= pos)));
            keep = !drop;
            out[frame * HW + j] = keep ? fp[j] : zero_index;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep_bits && lane == 0) keep_bits[(frame * Hq + h) * nwords + word] = m;
    }
}

}  // namespace

size_t similarity_workspace_bytes(long long N, int Tp, long long HW) {
    return (size_t)(N * Tp * HW) * 8 + (size_t)(N * Tp) * 8 + (size_t)DIGIT_TAB * 4 + 512;
}

int launch_similarity_mask(const int32_t* idx_p, const int32_t* idx_i, long long N, int Tp, int Hq, int Wq,
                           const FsqConsts& f, long long k, int32_t zero_index, int32_t* out, uint32_t* keep_bits,
                           float* sim, void* ws, cudaStream_t s) {
    const long long HW = (long long)Hq * Wq, ntok = N * Tp * HW, frames = N * Tp;
    if (ntok <= 0) return 0;
    unsigned long long* keys = static_cast<unsigned long long*>(ws);
    unsigned long long* thr = keys + ntok;
    bool small_levels = true;
    for (int c = 0; c < f.nlev; ++c) small_levels = small_levels && f.levels[c] <= 16;
    if (HW <= FUSED_MAX_TOKENS && small_levels) {
        uint32_t* tab = reinterpret_cast<uint32_t*>(thr + frames);
        int prod = 1;
        for (int c = 0; c < f.nlev; ++c) prod *= f.levels[c];
        const int ntab = prod < DIGIT_TAB ? prod : DIGIT_TAB;
        digit_table_kernel<<<blocks_for(ntab, 256), 256, 0, s>>>(f, ntab, tab);
        const size_t smem = (size_t)HW * 4;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(select_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(FUSED_MAX_TOKENS * 4));
            attr = true;
        }
        select_fused_kernel<<<(unsigned)frames, FS_THREADS, smem, s>>>(idx_p, idx_i, tab, ntab, f, Tp, Hq, Wq, k,
                                                                       zero_index, out, keep_bits, sim);
        return (int)cudaGetLastError();
    }
    sim_key_kernel<<<blocks_for(ntok, 256), 256, 0, s>>>(idx_p, idx_i, N, Tp, HW, f, keys, sim);
    const int all_keep = k <= 0 ? 1 : 0;
    if (!all_keep) select_kernel<<<(unsigned)frames, SEL_THREADS, 0, s>>>(keys, HW, k < HW ? k : HW, thr);
    const long long rows = frames * Hq;
    apply_kernel<<<blocks_for(rows * ((Wq + 31) / 32) * 32, 256), 256, 0, s>>>(idx_p, keys, thr, rows, Hq, Wq,
                                                                                all_keep, zero_index, out,
                                                                                keep_bits);
    return (int)cudaGetLastError();
}

}  // namespace tok
