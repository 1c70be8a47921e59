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

// ---------------------------------------------------------------- integer form
//
// When every channel's half-width floor(L/2) is a power of two (FSQ [8,8,8,5,5,5]:
// 4, 4, 4, 2, 2, 2), every code value q/hw is a dyadic rational and the float32
// sums of the definition are exact: with Q = max hw^2 and w = Q / hw^2 per
// channel, dot = D / Q, |p|^2 = A / Q, |q|^2 = B / Q for the integers
// D = sum w qp qi, A = sum w qp^2, B = sum w qi^2, and the product of the squared
// norms A B / Q^2 is exact too. So S = D/Q divided (rounded) by the rounded
// square root of A B / Q^2: the same float32 value, bit for bit, as the three
// sums, one square root and one division of the definition. (A table of S over
// (|D|, A B) measured slower than computing it: one L2 lookup per token, 0.186
// against 0.167 ms on 14.7 M tokens.) A token index is split as lo + 2^shift hi; small tables give the
// centered digits q (one signed byte per channel) and w q of each part, and two
// dp4a per dot product sum them.
//
// The k-th largest similarity of a frame is then found from a 2048-bucket
// histogram of S (bucket = floor((S + 1) * 1023.5): monotone in S), built in the
// same pass as the similarities: the bucket holding the k-th largest is either
// one value (often: P tokens equal to their I token all have S = 1), resolved at
// once, or a short list of candidates, radix-selected in shared memory; only a
// bucket of more than SB_CAND tokens with distinct values falls back to the
// radix select over the whole frame.
constexpr int SB_THREADS = 1024, SB_BINS = 2048, SB_CAND = 1024;
constexpr long long SB_MAX_TOKENS = 16384;
constexpr int SB_TAB_MAX = 512;     // entries of each index-part table

struct SelTables {
    const uint4* lo;   // [2^shift]: bytes of x, y = q of channels 0..7 (lo part), bytes of z, w = w q
    const uint4* hi;   // [nhi]: the same for the hi part (disjoint channels, OR-able)
    float invQ, invQ2;
    int shift, nhi, prod;
};

__global__ void sel_tables_kernel(FsqConsts f, int split_c, int shift, int nhi, int Q, uint4* lo, uint4* hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nlo = 1 << shift;
    auto pack = [&](int part, int v) {
        uint32_t q[2] = {0u, 0u}, wq[2] = {0u, 0u};
        for (int c = 0; c < f.nlev; ++c) {
            if ((c < split_c) != (part == 0)) continue;
            const int base = part == 0 ? f.basis[c] : f.basis[c] / nlo;
            const int d = (v / base) % f.levels[c];
            const int qc = d - f.half_w[c], w = Q / (f.half_w[c] * f.half_w[c]);
            q[c / 4] |= (uint32_t)(qc & 0xFF) << (8 * (c % 4));
            wq[c / 4] |= (uint32_t)((w * qc) & 0xFF) << (8 * (c % 4));
        }
        return make_uint4(q[0], q[1], wq[0], wq[1]);
    };
    if (i < nlo) lo[i] = pack(0, i);
    if (i < nhi) hi[i] = pack(1, i);
}

// Code vector (q and w q) of a token index; an index outside [0, prod) is decoded
// as the other forms decode it.
__device__ __forceinline__ uint4 sel_code(int idx, const SelTables& t, const FsqConsts& f) {
    if ((unsigned)idx < (unsigned)t.prod) {
        const uint4 a = t.lo[idx & ((1 << t.shift) - 1)], b = t.hi[idx >> t.shift];
        return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
    }
    const int Q = (int)(1.0f / t.invQ);
    uint32_t q[2] = {0u, 0u}, wq[2] = {0u, 0u};
    for (int c = 0; c < f.nlev; ++c) {
        const int d = (idx / f.basis[c]) % f.levels[c];
        const int qc = d - f.half_w[c], w = Q / (f.half_w[c] * f.half_w[c]);
        q[c / 4] |= (uint32_t)(qc & 0xFF) << (8 * (c % 4));
        wq[c / 4] |= (uint32_t)((w * qc) & 0xFF) << (8 * (c % 4));
    }
    return make_uint4(q[0], q[1], wq[0], wq[1]);
}

__device__ __forceinline__ uint32_t sim_order(float S) {
    const uint32_t u = __float_as_uint(S);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ int sim_bucket(float S) {
    const int b = (int)__fmul_rn(__fadd_rn(S, 1.0f), 1023.5f);
    return min(max(b, 0), SB_BINS - 1);
}

__device__ __forceinline__ float sim_of_order(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// Digit d (from the top) holding the rem-th largest of a histogram of nb bins,
// counted from bin nb - 1 down; warp 0 calls it. Returns (digit, rem within it).
__device__ __forceinline__ void top_digit(const uint32_t* hist, int nb, long long rem, int lane, int* d_out,
                                          long long* rem_out) {
    const int per = nb / 32, hi = nb - per * lane;
    long long own = 0;
    for (int b = hi - 1; b >= hi - per; --b) own += hist[b];
    long long incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t hit = __ballot_sync(0xffffffffu, incl >= rem);
    if (hit && lane == __ffs(hit) - 1) {
        long long cum = incl - own;
        int d = hi - 1;
        for (; d > hi - per; --d) {
            if (cum + (long long)hist[d] >= rem) break;
            cum += hist[d];
        }
        *d_out = d;
        *rem_out = rem - cum;
    }
}

// Block-wide: the rem-th largest of keys key(0 .. n-1) (MSB-first radix over 11, 11
// and 10 bits). Every thread calls it; the result (value, rem among the keys equal
// to it) is in *star / *rem_out after the closing barrier.
template <typename F>
__device__ void radix_kth(F key, int n, long long rem, uint32_t* hist, uint32_t* s_prefix, uint32_t* s_mask,
                          long long* s_rem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        *s_prefix = 0u;
        *s_mask = 0u;
        *s_rem = rem;
    }
    const int shifts[3] = {21, 10, 0};
    const uint32_t dmasks[3] = {0x7FFu, 0x7FFu, 0x3FFu};
    for (int pass = 0; pass < 3; ++pass) {
        for (int i = tid; i < SB_BINS; i += SB_THREADS) hist[i] = 0u;
        __syncthreads();
        const uint32_t prefix = *s_prefix, mask = *s_mask;
        const int shift = shifts[pass];
        const uint32_t dm = dmasks[pass];
        for (int it = 0; it < (n + SB_THREADS - 1) / SB_THREADS; ++it) {
            const int j = it * SB_THREADS + tid;
            const uint32_t o = j < n ? key(j) : 0u;
            const bool act = j < n && (o & mask) == prefix;
            const uint32_t dig = (o >> shift) & dm;
            const uint32_t am = __ballot_sync(0xffffffffu, act);
            if (act) {
                const uint32_t same = __match_any_sync(am, dig);
                if (lane == __ffs(same) - 1) atomicAdd(&hist[dig], (uint32_t)__popc(same));
            }
        }
        __syncthreads();
        if (warp == 0) {
            int d = -1;
            long long r = 0;
            top_digit(hist, pass < 2 ? 2048 : 1024, *s_rem, lane, &d, &r);
            if (d >= 0) {  // the lane that found the digit publishes it
                *s_rem = r;
                *s_prefix = prefix | ((uint32_t)d << shift);
                *s_mask = mask | (dm << shift);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SB_THREADS, 2) select_bucket_kernel(
    const int32_t* __restrict__ idx_p, const int32_t* __restrict__ idx_i, const SelTables tb, FsqConsts f, int Tp,
    int Hq, int Wq, long long k, int32_t zero_index, int32_t* __restrict__ out, uint32_t* __restrict__ keep_bits,
    float* __restrict__ sim) {
    extern __shared__ uint32_t ords[];  // HW order-preserving similarity images
    __shared__ uint32_t hist[SB_BINS];
    __shared__ uint32_t cand[SB_CAND];  // order images of the threshold bucket's tokens
    __shared__ uint32_t wsum[SB_THREADS / 32];
    __shared__ uint32_t s_prefix, s_mask, s_pos, s_min, s_max, s_n;
    __shared__ int s_bin;
    __shared__ long long s_rem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long frame = blockIdx.x, n = frame / Tp;
    const int HW = Hq * Wq;
    const int32_t* fp = idx_p + frame * HW;
    const int32_t* fi = idx_i + n * HW;
    for (int i = tid; i < SB_BINS; i += SB_THREADS) hist[i] = 0u;
    if (tid == 0) {
        s_min = 0xFFFFFFFFu;
        s_max = 0u;
        s_n = 0u;
        s_pos = 0u;
        s_bin = 0;
        s_rem = 0;
    }
    __syncthreads();
    // phase 1: similarities, their order images and the bucket histogram
    const int iters = (HW + SB_THREADS - 1) / SB_THREADS, full = HW / SB_THREADS;
    float* const simf = sim ? sim + frame * HW : nullptr;
    const uint32_t lomask = (1u << tb.shift) - 1u;
    const auto similarity = [&](int ip, int ii) {
        uint4 a, b;
        if ((unsigned)ip < (unsigned)tb.prod && (unsigned)ii < (unsigned)tb.prod) {
            const uint4 a0 = tb.lo[ip & lomask], a1 = tb.hi[ip >> tb.shift];
            const uint4 b0 = tb.lo[ii & lomask], b1 = tb.hi[ii >> tb.shift];
            a = make_uint4(a0.x | a1.x, a0.y | a1.y, a0.z | a1.z, a0.w | a1.w);
            b = make_uint4(b0.x | b1.x, b0.y | b1.y, b0.z | b1.z, b0.w | b1.w);
        } else {
            a = sel_code(ip, tb, f);
            b = sel_code(ii, tb, f);
        }
        const int D = __dp4a((int)a.z, (int)b.x, __dp4a((int)a.w, (int)b.y, 0));
        const int A = __dp4a((int)a.z, (int)a.x, __dp4a((int)a.w, (int)a.y, 0));
        const int B = __dp4a((int)b.z, (int)b.x, __dp4a((int)b.w, (int)b.y, 0));
        // the definition's one rounded square root of the exact norm product and one
        // rounded division of the exact dot product
        const int Pq = A * B, aD = abs(D);
        const float S =
            Pq > 0 ? __fdiv_rn(__fmul_rn((float)aD, tb.invQ), __fsqrt_rn(__fmul_rn((float)Pq, tb.invQ2))) : 0.f;
        return D < 0 ? -S : S;  // rounding is symmetric; D = 0 gives +0
    };
    // the next iteration's two indices are loaded while this one's similarity is formed
    int ip_n = tid < HW ? fp[tid] : 0, ii_n = tid < HW ? fi[tid] : 0;
    for (int it = 0; it < iters; ++it) {
        const int j = it * SB_THREADS + tid;
        const bool act = it < full || j < HW;
        const int ip = ip_n, ii = ii_n;
        if (j + SB_THREADS < HW) {
            ip_n = fp[j + SB_THREADS];
            ii_n = fi[j + SB_THREADS];
        }
        int bkt = 0;
        if (act) {
            const float S = similarity(ip, ii);
            ords[j] = sim_order(S);
            bkt = sim_bucket(S);
            if (simf) simf[j] = S;
        }
        // the S = 1 bucket (P tokens equal to their I token, the redundancy the selection
        // removes) takes one warp-aggregated increment; the others, spread over 2047
        // buckets, plain shared-memory atomics (a warp-wide match for every token cost 3%)
        const uint32_t top = __ballot_sync(0xffffffffu, act && bkt == SB_BINS - 1);
        if (lane == 0 && top) atomicAdd(&hist[SB_BINS - 1], (uint32_t)__popc(top));
        if (act && bkt != SB_BINS - 1) atomicAdd(&hist[bkt], 1u);
    }
    __syncthreads();
    const bool all_drop = k >= HW, none = k <= 0;
    uint32_t star = 0u;
    if (!all_drop && !none) {
        // phase 2: the bucket holding the k-th largest similarity
        if (warp == 0) {
            int d = -1;
            long long r = 0;
            top_digit(hist, SB_BINS, k, lane, &d, &r);
            if (d >= 0) {
                s_bin = d;
                s_rem = r;
            }
        }
        __syncthreads();
        const int bin = s_bin;
        const long long rem_b = s_rem;
        const uint32_t m = hist[bin];
        // phase 3: that bucket's tokens: extent of their images (per thread, then one
        // warp reduction and one shared atomic per warp), and the images themselves
        uint32_t tmin = 0xFFFFFFFFu, tmax = 0u;
        for (int it = 0; it < iters; ++it) {
            const int j = it * SB_THREADS + tid;
            const uint32_t o = j < HW ? ords[j] : 0u;
            const bool in = j < HW && sim_bucket(sim_of_order(o)) == bin;
            if (in) {
                tmin = min(tmin, o);
                tmax = max(tmax, o);
            }
            if (m <= SB_CAND) {
                const uint32_t bm = __ballot_sync(0xffffffffu, in);
                if (bm) {
                    uint32_t base = 0u;
                    if (lane == 0) base = atomicAdd(&s_n, (uint32_t)__popc(bm));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (in) cand[base + __popc(bm & ((1u << lane) - 1u))] = o;
                }
            }
        }
        tmin = __reduce_min_sync(0xffffffffu, tmin);
        tmax = __reduce_max_sync(0xffffffffu, tmax);
        if (lane == 0) {
            atomicMin(&s_min, tmin);
            atomicMax(&s_max, tmax);
        }
        __syncthreads();
        if (s_min == s_max) {
            star = s_min;  // one value: the rem_b lowest positions among its tokens drop
            if (tid == 0) s_rem = rem_b;
            __syncthreads();
        } else if (m <= SB_CAND) {
            radix_kth([&](int i) { return cand[i]; }, (int)m, rem_b, hist, &s_prefix, &s_mask, &s_rem);
            star = s_prefix;
        } else {
            radix_kth([&](int i) { return ords[i]; }, HW, k, hist, &s_prefix, &s_mask, &s_rem);
            star = s_prefix;
        }
        // phase 4: among the tokens equal to the k-th largest, the s_rem lowest positions drop
        const int per = (HW + SB_THREADS - 1) / SB_THREADS;
        const int j0 = tid * per, j1 = min(j0 + per, HW);
        uint32_t cnt = 0;
        for (int j = j0; j < j1; ++j) cnt += ords[j] == star ? 1u : 0u;
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
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t before = incl - cnt + (warp > 0 ? wsum[warp - 1] : 0u);
        const long long rem = s_rem;
        if ((long long)before < rem && rem <= (long long)(before + cnt)) {
            long long need = rem - before;
            for (int j = j0; j < j1; ++j)
                if (ords[j] == star && --need == 0) {
                    s_pos = (uint32_t)j;
                    break;
                }
        }
        __syncthreads();
    }
    // phase 5: drop, indices and keep bits (a warp per 32 tokens of a row)
    const uint32_t pos = s_pos;
    const int nwords = (Wq + 31) / 32;
    const auto drops = [&](int j) {
        const uint32_t o = ords[j];
        return all_drop || (!none && (o > star || (o == star && (uint32_t)j <= pos)));
    };
    if (Wq % 32 == 0) {
        // rows of whole mask words: word rw holds tokens 32 rw .. 32 rw + 31 of the frame;
        // two words per warp in flight
        const int nw = Hq * nwords;
        uint32_t* const kb = keep_bits ? keep_bits + (long long)frame * nw : nullptr;
        int32_t* const fo = out + frame * HW;
        for (int rw = warp; rw < nw; rw += 2 * (SB_THREADS / 32)) {
            const int rw2 = rw + SB_THREADS / 32;
            const int j = rw * 32 + lane, j2 = rw2 * 32 + lane;
            const bool k1 = !drops(j), k2 = rw2 < nw && !drops(j2);
            const int32_t v1 = k1 ? fp[j] : zero_index;
            const int32_t v2 = k2 ? fp[j2] : zero_index;
            fo[j] = v1;
            if (rw2 < nw) fo[j2] = v2;
            const uint32_t m1 = __ballot_sync(0xffffffffu, k1), m2 = __ballot_sync(0xffffffffu, k2);
            if (kb && lane == 0) {
                kb[rw] = m1;
                if (rw2 < nw) kb[rw2] = m2;
            }
        }
        return;
    }
    for (int rw = warp; rw < Hq * nwords; rw += SB_THREADS / 32) {
        const int h = rw / nwords, word = rw - h * nwords, w = word * 32 + lane;
        bool keep = false;
        if (w < Wq) {
            const int j = h * Wq + w;
            const uint32_t o = ords[j];
            const bool drop = all_drop || (!none && (o > star || (o == star && (uint32_t)j <= pos)));
            keep = !drop;
            out[frame * HW + j] = keep ? fp[j] : zero_index;
        }
        const uint32_t msk = __ballot_sync(0xffffffffu, keep);
        if (keep_bits && lane == 0) keep_bits[(frame * Hq + h) * nwords + word] = msk;
    }
}

// Whether the integer form applies (see above), and its table geometry.
struct SelPlan {
    bool ok = false;
    int split_c = 0, shift = 0, nhi = 0, Q = 0, prod = 0;
};

SelPlan sel_plan(const FsqConsts& f, long long HW) {
    SelPlan p;
    if (HW > SB_MAX_TOKENS || HW < 1) return p;
    int Q = 1;
    for (int c = 0; c < f.nlev; ++c) {
        const int h = f.half_w[c];
        if (h < 1 || (h & (h - 1)) || h > 8) return p;
        Q = std::max(Q, h * h);
    }
    const long long prod = (long long)f.basis[f.nlev - 1] * f.levels[f.nlev - 1];
    // |D|, A, B <= nlev Q: the products A B stay exact in float32 below 2^24
    const long long dmax = (long long)f.nlev * Q;
    if (dmax * dmax >= (1LL << 24)) return p;
    for (int c = 1; c < f.nlev; ++c) {
        const int b = f.basis[c];
        if (b & (b - 1)) continue;
        if (b <= SB_TAB_MAX && prod / b <= SB_TAB_MAX && prod % b == 0) {
            p.ok = true;
            p.split_c = c;
            p.shift = __builtin_ctz((unsigned)b);
            p.nhi = (int)(prod / b);
            p.Q = Q;
            p.prod = (int)prod;
            return p;
        }
    }
    return p;
}

}  // namespace

size_t similarity_workspace_bytes(long long N, int Tp, long long HW) {
    // per-token keys and per-frame thresholds (the three-kernel form), the digit
    // table, and the integer form's tables
    return (size_t)(N * Tp * HW) * 8 + (size_t)(N * Tp) * 8 + (size_t)DIGIT_TAB * 4 + 512 +
           (size_t)2 * SB_TAB_MAX * 16 + 512;
}

int launch_similarity_mask(const int32_t* idx_p, const int32_t* idx_i, long long N, int Tp, int Hq, int Wq,
                           const FsqConsts& f, long long k, int32_t zero_index, int32_t* out, uint32_t* keep_bits,
                           float* sim, void* ws, cudaStream_t s) {
    const long long HW = (long long)Hq * Wq, ntok = N * Tp * HW, frames = N * Tp;
    if (ntok <= 0) return 0;
    unsigned long long* keys = static_cast<unsigned long long*>(ws);
    unsigned long long* thr = keys + ntok;
    const SelPlan pl = sel_plan(f, HW);
    if (pl.ok) {
        // the integer form: its tables after the digit table (see the workspace size)
        char* tb = reinterpret_cast<char*>(thr + frames) + (size_t)DIGIT_TAB * 4;
        tb = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(tb) + 255) & ~uintptr_t(255));
        uint4* lo = reinterpret_cast<uint4*>(tb);
        uint4* hi = lo + SB_TAB_MAX;
        const int nt = std::max(1 << pl.shift, pl.nhi);
        sel_tables_kernel<<<blocks_for(nt, 256), 256, 0, s>>>(f, pl.split_c, pl.shift, pl.nhi, pl.Q, lo, hi);
        SelTables t;
        t.lo = lo;
        t.hi = hi;
        t.invQ = 1.0f / (float)pl.Q;
        t.invQ2 = 1.0f / (float)(pl.Q * pl.Q);
        t.shift = pl.shift;
        t.nhi = pl.nhi;
        t.prod = pl.prod;
        static std::atomic<unsigned long long> attr_b{0};
        if (smem_attr_once(select_bucket_kernel, (int)(SB_MAX_TOKENS * 4), attr_b) != cudaSuccess)
            return (int)cudaGetLastError();
        select_bucket_kernel<<<(unsigned)frames, SB_THREADS, (size_t)HW * 4, s>>>(idx_p, idx_i, t, f, Tp, Hq, Wq, k,
                                                                                  zero_index, out, keep_bits, sim);
        return (int)cudaGetLastError();
    }
    bool small_levels = true;
    for (int c = 0; c < f.nlev; ++c) small_levels = small_levels && f.levels[c] <= 16;
    if (HW <= FUSED_MAX_TOKENS && small_levels) {
        uint32_t* tab = reinterpret_cast<uint32_t*>(thr + frames);
        int prod = 1;
        for (int c = 0; c < f.nlev; ++c) prod *= f.levels[c];
        const int ntab = prod < DIGIT_TAB ? prod : DIGIT_TAB;
        digit_table_kernel<<<blocks_for(ntab, 256), 256, 0, s>>>(f, ntab, tab);
        const size_t smem = (size_t)HW * 4;
        static std::atomic<unsigned long long> attr{0};
        if (smem_attr_once(select_fused_kernel, (int)(FUSED_MAX_TOKENS * 4), attr) != cudaSuccess)
            return (int)cudaGetLastError();
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
