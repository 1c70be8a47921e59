// The encoder's stem on the tensor cores with its im2col rows formed on chip:
// the causal 3x3x3 conv from the 3 pixel channels to the first level's Cout
// channels (64 or 128), stride (st, 2, 2) (Sec. 2.4's encoder input; the 8x8x8
// setting of Sec. 4.1 uses st = 2), plus its bias, the BF16 output and the
// GroupNorm statistics of that output, in one persistent kernel.
//
// Tile: 128 consecutive output voxels of one output row, (n, to, ho, wo0 ..
// wo0 + 127): the MMA's M = 128 (TMEM lane = voxel), N = Cout channels, K =
// (dt, dh, dw, ci) = 81 taps x channels, zero-padded to 96 (six K = 16 steps).
// The input a tile reads -- 3 frames x 3 rows x the 257 pixels (771 BF16
// values, x = 3 w + ci) of its window -- arrives by TMA as 12 boxes of 3 rows
// x 200 values; the TMA's zero fill gives the spatial zero padding (the frame
// needs no edge extension: H and W are the padded extent), frames before the
// clip come from the stream history, frame 0 or a zero box.
//
// Warp roles (768 threads, one CTA per SM):
//   warp 0      TMA producer (weights once, then the input boxes per tile,
//               up to four tiles ahead)
//   warp 1      MMA issuer: six tcgen05.mma into one of two TMEM accumulators
//   warp 2      TMEM allocation
//   warp 3      statistics: merges the epilogue warps' sums per tile
//   warps 4-7   im2col: thread v writes row v of the A tile (128B-swizzled,
//               K-major) from the input boxes
//   warps 8-23  epilogue: TMEM -> + bias -> BF16, written out through a
//               per-warp staging area with 16-byte stores (the TMA unit is
//               left to the input boxes), and the statistics of its 32
//               voxels x Cout/4 channels (four epilogue warps per SM
//               sub-partition hide each other's latencies)
// Every wait is bounded; a wait that gives up records TOK_ETIMEOUT and every
// role leaves its loop, drains its own copies and MMAs, and the CTA frees TMEM.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "conv_args.h"
#include "launchers.h"

namespace tok {

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn();
bool encode_w_map(CUtensorMap* m, const void* base, int rows, int Kpad, int BN, int kc);

namespace {

constexpr int SV = 128;                    // output voxels per tile
constexpr int XB = 200;                    // BF16 values per input box row
constexpr int NXB = 4;                     // boxes along x: 800 >= 6 * 127 + 14
constexpr int BOXB = 1280;                 // 3 rows x 200 values (1200 B), 128-byte aligned
constexpr int RAWB = 3 * NXB * BOXB;       // one tile's input boxes
constexpr int NRAW = 4;                    // input stages (tiles of input in flight)
constexpr int NSB = 4;                     // statistics buffers (tiles the merge may lag behind)
constexpr uint32_t RAW_TX = 3 * NXB * 3 * XB * 2;
constexpr int KSTEPS = 6;                  // K = 96
constexpr int NTHREADS = 768;

template <int CO>
struct StemCfg {
    static constexpr int W_ATOM = CO * 128;       // 64 K values of every weight row, SW128
    static constexpr int A_ATOM = SV * 128;       // 64 K values of every voxel row, SW128
    static constexpr int A_STAGE = 2 * A_ATOM;
    static constexpr int RB = CO / 2;             // bytes of an epilogue warp's staged row (Cout/4 bf16)
    static constexpr int OFF_W = 0;
    static constexpr int OFF_A = 2 * W_ATOM;
    static constexpr int OFF_RAW = OFF_A + 2 * A_STAGE;
    static constexpr int OFF_STG = OFF_RAW + NRAW * RAWB;  // 16 warps x 32 rows x RB
    static constexpr int OFF_BIAS = OFF_STG + 16 * 32 * RB;
    // statistics of a tile per buffer: shifts K[4][32], sums (s, q)[4][32], counts n[4]
    static constexpr int OFF_STK = OFF_BIAS + CO * 4;
    static constexpr int OFF_STSQ = OFF_STK + NSB * 4 * 32 * 4;
    static constexpr int OFF_STN = OFF_STSQ + NSB * 4 * 32 * 8;
    static constexpr int OFF_BAR = OFF_STN + NSB * 4 * 4;
    static constexpr int NBAR = 2 * NRAW + 9 + 2 * NSB;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 8 + 1024;  // + TMEM address, + alignment slack
    static constexpr int TMEM_COLS = 2 * CO;
    static constexpr uint32_t IDESC = idesc_bf16_f32(128, CO);
    static_assert(OFF_A % 1024 == 0 && OFF_RAW % 1024 == 0, "swizzle atoms");
    static_assert(SMEM <= 232448 - 64, "shared memory");
};

struct StemProb {
    CUtensorMap tm_x, tm_h;
    long long tile_end;  // tiles of the problems up to this one
    GnTriple* gn_part;
    __nv_bfloat16* out;
    int N, Tin, hist_T, Tout, Hout, Wout, st, t_off, pad_mode, tiles_w, has_hist;
};

template <int MAXP>
struct StemBatch {
    CUtensorMap tm_w;
    StemProb q[MAXP];
    const float* bias;
    int* status;
    unsigned long long wait_ns;
    long long num_tiles;
    int count;
};

struct StemTile {
    int p, n, to, ho, tw;
};

template <int MAXP>
__device__ __forceinline__ StemTile stem_tile(const StemBatch<MAXP>& B, long long u) {
    StemTile t;
    int p = 0;
    if constexpr (MAXP > 1)
        while (p + 1 < B.count && u >= B.q[p].tile_end) ++p;
    // 32-bit arithmetic (a launch holds fewer than 2^31 tiles)
    int lu = (int)(p ? u - B.q[p - 1].tile_end : u);
    const StemProb& q = B.q[p];
    t.p = p;
    int r = lu / q.tiles_w;
    t.tw = lu - r * q.tiles_w;
    lu = r;
    r = lu / q.Hout;
    t.ho = lu - r * q.Hout;
    lu = r;
    r = lu / q.Tout;
    t.to = lu - r * q.Tout;
    t.n = r;
    return t;
}

// The tiles one CTA visits (u = blockIdx.x, + gridDim.x, ...), decoded once and
// then advanced by the stride in mixed radix (tw, ho, to, n) with carries; a
// step into the next problem decodes again.
template <int MAXP>
struct StemCursor {
    long long u;
    StemTile t;
    int s0, s1, s2, s3;  // the stride in the current problem's radices
    __device__ __forceinline__ void stride_digits(const StemBatch<MAXP>& B, int ncl) {
        const StemProb& q = B.q[t.p];
        int r = ncl / q.tiles_w;
        s0 = ncl - r * q.tiles_w;
        int r2 = r / q.Hout;
        s1 = r - r2 * q.Hout;
        s3 = r2 / q.Tout;
        s2 = r2 - s3 * q.Tout;
    }
    __device__ __forceinline__ void start(const StemBatch<MAXP>& B, long long u0, int ncl) {
        u = u0;
        t = stem_tile(B, u0 < B.num_tiles ? u0 : 0);
        stride_digits(B, ncl);
    }
    __device__ __forceinline__ void next(const StemBatch<MAXP>& B, int ncl) {
        u += ncl;
        if (u >= B.num_tiles) return;
        if (MAXP > 1 && u >= B.q[t.p].tile_end) {
            const int p0 = t.p;
            t = stem_tile(B, u);
            if (t.p != p0) stride_digits(B, ncl);
            return;
        }
        const StemProb& q = B.q[t.p];
        int c;
        t.tw += s0;
        c = t.tw >= q.tiles_w;
        t.tw -= c ? q.tiles_w : 0;
        t.ho += s1 + c;
        c = t.ho >= q.Hout;
        t.ho -= c ? q.Hout : 0;
        t.to += s2 + c;
        c = t.to >= q.Tout;
        t.to -= c ? q.Tout : 0;
        t.n += s3 + c;
    }
};

// Frame coordinate of input frame ti of sample n and the map it is read from:
// the clip, the history before it, frame 0 (replicate padding) or -1 (a box
// wholly outside the tensor: zeros).
__device__ __forceinline__ int stem_frame(const StemProb& q, int n, int ti, const CUtensorMap** m) {
    *m = &q.tm_x;
    if (ti >= q.Tin) return -1;
    if (ti >= 0) return n * q.Tin + ti;
    if (q.has_hist) {
        *m = &q.tm_h;
        return n * q.hist_T + q.hist_T + ti;
    }
    return q.pad_mode == 0 ? n * q.Tin : -1;
}

// Every lane waits; the warp goes on only if all of them saw the phase.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* status, unsigned long long ns) {
    const bool ok = mbar_wait(bar, parity, status, ns);
    return __all_sync(0xffffffffu, ok);
}

// 16 bits (half ha of a, half hb of b) -> one word, a's half in the low bits.
__device__ __forceinline__ uint32_t pick2(uint32_t a, int ha, uint32_t b, int hb) {
    return __byte_perm(a, b, (unsigned)((ha ? 0x32 : 0x10) | ((hb ? 0x76 : 0x54) << 8)));
}

__device__ __forceinline__ GnTriple stem_merge(GnTriple a, GnTriple b) {
    if (b.n == 0.f) return a;
    if (a.n == 0.f) return b;
    GnTriple r;
    r.n = a.n + b.n;
    const float d = b.mean - a.mean;
    const float fb = b.n * __frcp_rn(r.n);  // counts: small integers
    r.mean = a.mean + d * fb;
    r.m2 = a.m2 + b.m2 + d * d * a.n * fb;
    return r;
}

__device__ __forceinline__ uint32_t ld_shared_u32(const uint8_t* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// Two FP32 values in one 64-bit register (low: first) and the paired FP32
// arithmetic of sm_100-family SMs (each lane rounded as the scalar operation).
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
    return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t shfl_xor2(uint64_t v, int o) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, o);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), o);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}
// bf16 pair (low: first) -> the two values as FP32
__device__ __forceinline__ uint64_t bf2_to_f2(uint32_t w) {
    return f2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// Per group g of WPG bf16 pairs: (sum, sum of squares) of the values minus the
// group's shift Kg[g], each weighted by M (0 or 1 per lane) when MASK.
template <int NG, int WPG, bool MASK>
__device__ __forceinline__ void group_sums(const uint32_t (&pk)[NG * WPG], const float (&Kg)[NG], uint64_t M,
                                           uint64_t (&sq)[NG]) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const uint64_t KK = f2(Kg[g], Kg[g]);
        uint64_t d = sub2(bf2_to_f2(pk[g * WPG]), KK);
        if (MASK) d = mul2(d, M);
        uint64_t s2 = d, q2 = mul2(d, d);
#pragma unroll
        for (int j = 1; j < WPG; ++j) {
            d = sub2(bf2_to_f2(pk[g * WPG + j]), KK);
            if (MASK) d = mul2(d, M);
            s2 = add2(s2, d);
            q2 = fma2(d, d, q2);
        }
        sq[g] = f2(f2_lo(s2) + f2_hi(s2), f2_lo(q2) + f2_hi(q2));
    }
}

template <int CO, int MAXP>
__global__ void __launch_bounds__(NTHREADS, 1) stem_tc_kernel(const __grid_constant__ StemBatch<MAXP> B) {
    using C = StemCfg<CO>;
    extern __shared__ uint8_t smem_dyn[];
    uint8_t* smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    uint64_t* raw_full = bars;                // [NRAW] TMA bytes of a tile's input boxes
    uint64_t* raw_empty = bars + NRAW;        // [NRAW] 4 im2col warps
    uint64_t* a_full = bars + 2 * NRAW;       // [2] 4 im2col warps
    uint64_t* a_empty = a_full + 2;           // [2] MMA commit
    uint64_t* t_full = a_full + 4;            // [2] MMA commit
    uint64_t* t_empty = a_full + 6;           // [2] 16 epilogue warps
    uint64_t* o_ready = a_full + 8;           // [NSB] 16 epilogue warps: a tile's statistics staged
    uint64_t* o_free = o_ready + NSB;         // [NSB] statistics warp
    uint64_t* w_full = o_free + NSB;          // weights
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + C::NBAR);
    float* sbias = reinterpret_cast<float*>(smem + C::OFF_BIAS);

    int* status = B.status;
    const unsigned long long wait_ns = B.wait_ns;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long cid = blockIdx.x, ncl = gridDim.x;
    // a context already in error skips the launch (decided once per CTA)
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (status && *(volatile int*)status != 0) ? 1 : 0;
    __syncthreads();
    if (s_skip) return;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NRAW; ++i) {
            mbar_init(&raw_full[i], 1);
            mbar_init(&raw_empty[i], 4);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&a_full[i], 4);
            mbar_init(&a_empty[i], 1);
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 16);
        }
        for (int i = 0; i < NSB; ++i) {
            mbar_init(&o_ready[i], 16);
            mbar_init(&o_free[i], 1);
        }
        mbar_init(w_full, 1);
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < CO; i += NTHREADS) sbias[i] = B.bias ? B.bias[i] : 0.f;
    if (warp == 0 && lane < B.count) {
        tma_prefetch_desc(&B.q[lane].tm_x);
        if (B.q[lane].has_hist) tma_prefetch_desc(&B.q[lane].tm_h);
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            mbar_arrive_expect_tx(w_full, 2 * C::W_ATOM);
            tma_load_2d(smem + C::OFF_W, &B.tm_w, w_full, 0, 0);
            tma_load_2d(smem + C::OFF_W + C::W_ATOM, &B.tm_w, w_full, 64, 0);
            int last[NRAW];
#pragma unroll
            for (int i = 0; i < NRAW; ++i) last[i] = -1;
            int it = 0;
            StemCursor<MAXP> cur;
            cur.start(B, cid, (int)ncl);
            for (; cur.u < B.num_tiles; cur.next(B, (int)ncl), ++it) {
                const int s = it % NRAW;
                const uint32_t ph = (uint32_t)((it / NRAW) & 1);
                const StemTile t = cur.t;
                if (!mbar_wait(&raw_empty[s], ph ^ 1, status, wait_ns)) break;
                const StemProb& q = B.q[t.p];
                uint8_t* dst = smem + C::OFF_RAW + s * RAWB;
                mbar_arrive_expect_tx(&raw_full[s], RAW_TX);
                // x = 3 w + ci from the window's first pixel 2 wo0 - 1, rounded down to a
                // 16-byte boundary (8 values): x0 = 6 wo0 - 8
                const int x0 = t.tw * (6 * SV) - 8, h0 = 2 * t.ho - 1;
#pragma unroll
                for (int dt = 0; dt < 3; ++dt) {
                    const CUtensorMap* m;
                    const int f = stem_frame(q, t.n, t.to * q.st + dt + q.t_off, &m);
#pragma unroll
                    for (int b = 0; b < NXB; ++b)
                        tma_load_3d(dst + (dt * NXB + b) * BOXB, m, &raw_full[s], x0 + b * XB, h0, f);
                }
#pragma unroll
                for (int i = 0; i < NRAW; ++i)
                    if (i == s) last[i] = (int)ph;
            }
            // no copy may still be in flight when the CTA exits
#pragma unroll
            for (int i = 0; i < NRAW; ++i)
                if (last[i] >= 0) mbar_wait(&raw_full[i], (uint32_t)last[i], status, wait_ns);
            mbar_wait(w_full, 0, status, wait_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer
            int last0 = -1, last1 = -1;
            if (mbar_wait(w_full, 0, status, wait_ns)) {
                tc_fence_after();
                const uint32_t wa = smem_u32(smem + C::OFF_W);
                int it = 0;
                for (long long u = cid; u < B.num_tiles; u += ncl, ++it) {
                    const int s = it & 1;
                    const uint32_t ph = (uint32_t)((it >> 1) & 1);
                    if (!mbar_wait(&t_empty[s], ph ^ 1, status, wait_ns)) break;
                    if (!mbar_wait(&a_full[s], ph, status, wait_ns)) break;
                    tc_fence_after();
                    const uint32_t aa = smem_u32(smem + C::OFF_A + s * C::A_STAGE);
                    const uint32_t d = tmem_base + (uint32_t)(s * CO);
#pragma unroll
                    for (int k = 0; k < KSTEPS; ++k)
                        tc_mma_bf16(d, sw128_desc(aa + (uint32_t)((k >> 2) * C::A_ATOM + (k & 3) * 32)),
                                    sw128_desc(wa + (uint32_t)((k >> 2) * C::W_ATOM + (k & 3) * 32)), C::IDESC,
                                    k ? 1u : 0u);
                    tc_commit(&a_empty[s]);
                    tc_commit(&t_full[s]);
                    if (s) last1 = (int)ph;
                    else last0 = (int)ph;
                }
            }
            // our own MMAs complete before TMEM can be released
            if (last0 >= 0) mbar_wait(&t_full[0], (uint32_t)last0, status, wait_ns);
            if (last1 >= 0) mbar_wait(&t_full[1], (uint32_t)last1, status, wait_ns);
        }
    } else if (warp == 3) {
        // -------------------------------------------------------- statistics
        // lane g merges group g's shifted sums over the four TMEM lane quarters in a
        // fixed order into the tile's statistics slot
        int it = 0;
        StemCursor<MAXP> cur;
        cur.start(B, cid, (int)ncl);
        for (; cur.u < B.num_tiles; cur.next(B, (int)ncl), ++it) {
            const int s = it % NSB;
            const uint32_t ph = (uint32_t)((it / NSB) & 1);
            const StemTile t = cur.t;
            if (!warp_wait(&o_ready[s], ph, status, wait_ns)) break;
            const StemProb& pq = B.q[t.p];
            if (pq.gn_part) {
                const float* stk = reinterpret_cast<const float*>(smem + C::OFF_STK) + s * 4 * 32;
                const float2* stsq = reinterpret_cast<const float2*>(smem + C::OFF_STSQ) + s * 4 * 32;
                const float* stn = reinterpret_cast<const float*>(smem + C::OFF_STN) + s * 4;
                GnTriple tr[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const float n = stn[qq], K = stk[qq * 32 + lane];
                    const float2 sq = stsq[qq * 32 + lane];
                    const float inv = n > 0.f ? __frcp_rn(n) : 0.f;
                    const float sm = sq.x * inv;
                    tr[qq].n = n;
                    tr[qq].mean = K + sm;
                    tr[qq].m2 = fmaxf(sq.y - sq.x * sm, 0.f);
                }
                const long long S = (long long)pq.Hout * pq.tiles_w;
                pq.gn_part[(((long long)t.n * pq.Tout + t.to) * S + (long long)t.ho * pq.tiles_w + t.tw) * 32 + lane] =
                    stem_merge(stem_merge(tr[0], tr[1]), stem_merge(tr[2], tr[3]));
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&o_free[s]);
        }
    } else if (warp >= 4 && warp < 8) {
        // -------------------------------------------------------- im2col
        // Row v of the A tile is voxel v: K = 9 r + k with r = dt * 3 + dh and k = 3 dw +
        // ci is value x = 6 v + 5 + k of input row r (x from x0). Its ten values x = 6 v +
        // 4 .. 6 v + 13 are five aligned words (no word straddles two boxes: a box row
        // holds an even number of values), read once per row.
        const int v = threadIdx.x - 128;
        uint32_t woff[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int e = 6 * v + 4 + 2 * j, b = e / XB;
            woff[j] = (uint32_t)(b * BOXB + (e - b * XB) * 2);
        }
        const uint32_t arow = (uint32_t)v * 128u, sw = (uint32_t)(v & 7);
        int it = 0;
        for (long long u = cid; u < B.num_tiles; u += ncl, ++it) {
            const int sr = it % NRAW, s = it & 1;
            if (!warp_wait(&raw_full[sr], (uint32_t)((it / NRAW) & 1), status, wait_ns)) break;
            if (!warp_wait(&a_empty[s], (uint32_t)(((it >> 1) & 1) ^ 1), status, wait_ns)) break;
            const uint8_t* rb = smem + C::OFF_RAW + sr * RAWB;
            uint8_t* ab = smem + C::OFF_A + s * C::A_STAGE;
            // output word m = K values (2m, 2m + 1); value k of row r is half k + 1 of the
            // row's ten (word (k + 1) / 2); K >= 81 is zero. Rows are read in order, two
            // live at a time (cur: row `rc`, prev: row rc - 1), and every 16-byte chunk is
            // stored as soon as its four words are formed.
            uint32_t cur[5], prev[5], o4[4];
            int rc = -1;
#pragma unroll
            for (int m = 0; m < 48; ++m) {
                const int k0 = 2 * m, k1 = 2 * m + 1;
                const int rneed = (k1 < 81 ? k1 : 80) / 9;
                if (rneed > rc) {
#pragma unroll
                    for (int j = 0; j < 5; ++j) prev[j] = cur[j];
                    rc = rneed;
#pragma unroll
                    for (int j = 0; j < 5; ++j)
                        cur[j] = ld_shared_u32(rb + ((rc / 3) * NXB * BOXB + (rc % 3) * XB * 2) + woff[j]);
                }
                auto word = [&](int k) -> uint32_t {
                    if (k >= 81) return 0u;
                    const int r = k / 9, wj = (k % 9 + 1) >> 1;
                    return r == rc ? cur[wj] : prev[wj];
                };
                o4[m & 3] = pick2(word(k0), k0 < 81 ? (k0 % 9 + 1) & 1 : 0, word(k1), k1 < 81 ? (k1 % 9 + 1) & 1 : 0);
                if ((m & 3) == 3) {
                    const int c = m >> 2;
                    uint8_t* dst = ab + (c >> 3) * C::A_ATOM + arow + ((((uint32_t)c & 7u) ^ sw) << 4);
                    *reinterpret_cast<uint4*>(dst) = make_uint4(o4[0], o4[1], o4[2], o4[3]);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&a_full[s]);
                mbar_arrive(&raw_empty[sr]);
            }
        }
    } else if (warp >= 8) {
        // -------------------------------------------------------- epilogue
        // warp (q, c4): TMEM lanes 32 q .. 32 q + 31 (voxels), channels c4 * Cout/4 ..;
        // GroupNorm of 32 groups: CG channels each, NG = 8 groups per warp. The
        // statistics are those of the stored BF16 values, as shifted sums per group
        // (the shift: lane 0's first value of the group; voxels past the row's end
        // weigh 0), reduced over the warp's voxels by a butterfly that leaves group
        // (lane >> 2) on lanes 4g .. 4g + 3. The warp stages its 32 rows in its own
        // region and writes them out with 16-byte stores, each row's bytes contiguous.
        constexpr int HC = CO / 4;
        constexpr int CG = CO / 32;
        constexpr int NG = HC / CG;
        constexpr int WPG = CG / 2;        // bf16 pairs per group
        constexpr int RB = C::RB;          // staged bytes per voxel row
        constexpr int CPR = RB / 16;       // 16-byte chunks per staged row
        constexpr int RPI = 32 / CPR;      // staged rows per copy-out instruction
        static_assert(NG == 8 && (CPR == 4 || CPR == 2) && RB == HC * 2, "epilogue shape");
        const int e = warp - 8, q = warp & 3, c4 = e >> 2;
        const int v = q * 32 + lane;
        const float* bias = sbias + c4 * HC;
        uint8_t* stg = smem + C::OFF_STG + e * 32 * RB;
        // chunk j of staged row r sits at chunk j ^ swz(r): the row-per-lane writes and
        // the contiguous reads are both free of bank conflicts
        auto swz = [](int r) { return CPR == 4 ? ((r >> 1) & 3) : ((r >> 2) & 1); };
        const int crow = lane / CPR, cchk = lane % CPR;
        int it = 0;
        StemCursor<MAXP> cur;
        cur.start(B, cid, (int)ncl);
        while (cur.u < B.num_tiles) {
            const int s = it & 1;
            const uint32_t ph = (uint32_t)((it >> 1) & 1);
            const int sb = it % NSB;
            const StemTile t = cur.t;
            if (!warp_wait(&t_full[s], ph, status, wait_ns)) break;
            tc_fence_after();
            const StemProb& pq = B.q[t.p];
            const int wo0 = t.tw * SV;
            const int nvalid = min(SV, pq.Wout - wo0);  // voxels of the tile inside the row
            const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(s * CO + c4 * HC);
            uint32_t r[HC / 16][16];
#pragma unroll
            for (int b = 0; b < HC / 16; ++b) tmem_ld16_issue(ta + (uint32_t)(b * 16), r[b]);
            tmem_ld_wait();
#pragma unroll
            for (int b = 0; b < HC / 16; ++b) tmem_regs_fence(r[b]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[s]);
            // + bias, to BF16 pairs: columns b * 16 + 4 i ..
            uint32_t pk[HC / 2];
#pragma unroll
            for (int b = 0; b < HC / 16; ++b) {
                const float4* b4 = reinterpret_cast<const float4*>(bias + b * 16);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4 bb = b4[i];
                    const uint64_t x0 = add2(f2(__uint_as_float(r[b][4 * i]), __uint_as_float(r[b][4 * i + 1])), f2(bb.x, bb.y));
                    const uint64_t x1 =
                        add2(f2(__uint_as_float(r[b][4 * i + 2]), __uint_as_float(r[b][4 * i + 3])), f2(bb.z, bb.w));
                    pk[b * 8 + 2 * i] = pack_bf16x2(f2_lo(x0), f2_hi(x0));
                    pk[b * 8 + 2 * i + 1] = pack_bf16x2(f2_lo(x1), f2_hi(x1));
                }
            }
            // statistics: (sum, sum of squares) of the shifted values per group, into the
            // buffer the statistics warp has released (every tile passes both barriers)
            cur.next(B, (int)ncl);  // the next tile's coordinates, early
            if (!warp_wait(&o_free[sb], (uint32_t)(((it / NSB) & 1) ^ 1), status, wait_ns)) break;
            const bool gstat = pq.gn_part != nullptr;
            uint64_t sq[NG];
            if (gstat) {
                // the shifts first, all eight broadcasts in flight together
                float Kg[NG];
#pragma unroll
                for (int g = 0; g < NG; ++g) Kg[g] = __shfl_sync(0xffffffffu, __uint_as_float(pk[g * WPG] << 16), 0);
                if (lane == 0) {
                    float4* stk = reinterpret_cast<float4*>(reinterpret_cast<float*>(smem + C::OFF_STK) +
                                                            (sb * 4 + q) * 32 + c4 * NG);
                    stk[0] = make_float4(Kg[0], Kg[1], Kg[2], Kg[3]);
                    stk[1] = make_float4(Kg[4], Kg[5], Kg[6], Kg[7]);
                }
                const float m = v < nvalid ? 1.f : 0.f;
                if (nvalid == SV)  // a whole tile (uniform over the CTA): no weights
                    group_sums<NG, WPG, false>(pk, Kg, 0ull, sq);
                else
                    group_sums<NG, WPG, true>(pk, Kg, f2(m, m), sq);
                // step o: a lane keeps the lower (upper if lane & o) half of its groups and
                // adds its partner's sums of them; then lanes 4g .. 4g + 3 sum group g
#pragma unroll
                for (int o = 16; o >= 4; o >>= 1) {
                    const int half = o / 4;
                    const bool up = (lane & o) != 0;
#pragma unroll
                    for (int i = 0; i < half; ++i) {
                        const uint64_t rr = shfl_xor2(up ? sq[i] : sq[i + half], o);
                        sq[i] = add2(up ? sq[i + half] : sq[i], rr);
                    }
                }
                sq[0] = add2(sq[0], shfl_xor2(sq[0], 2));
                sq[0] = add2(sq[0], shfl_xor2(sq[0], 1));
                uint64_t* stsq = reinterpret_cast<uint64_t*>(smem + C::OFF_STSQ) + (sb * 4 + q) * 32 + c4 * NG;
                if ((lane & 3) == 0) stsq[lane >> 2] = sq[0];
                if (lane == 0 && c4 == 0)
                    reinterpret_cast<float*>(smem + C::OFF_STN)[sb * 4 + q] =
                        (float)(CG * max(0, min(32, nvalid - q * 32)));
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&o_ready[sb]);
            // stage this warp's 32 rows, then write them out: RPI rows per instruction,
            // CPR lanes on each row's contiguous bytes
#pragma unroll
            for (int j = 0; j < CPR; ++j)
                *reinterpret_cast<uint4*>(stg + lane * RB + ((j ^ swz(lane)) << 4)) =
                    make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
            __syncwarp();
            {
                const long long vox0 = (((long long)t.n * pq.Tout + t.to) * pq.Hout + t.ho) * pq.Wout + wo0 + q * 32;
                __nv_bfloat16* op = pq.out + vox0 * CO + c4 * HC + cchk * 8;
#pragma unroll
                for (int i = 0; i < 32 / RPI; ++i) {
                    const int rr = crow + RPI * i;
                    const uint4 val = *reinterpret_cast<const uint4*>(stg + rr * RB + ((cchk ^ swz(rr)) << 4));
                    if (q * 32 + rr < nvalid) *reinterpret_cast<uint4*>(op + (long long)rr * CO) = val;
                }
            }
            __syncwarp();
            ++it;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 2) tmem_dealloc(tmem_base, C::TMEM_COLS);
}

// Pixels as (x = 3 w + ci, h, frame), boxes of 200 values x 3 rows x 1 frame,
// no swizzle; reads outside the tensor are zeros.
bool encode_pixels_map(CUtensorMap* m, const void* base, long long frames, int H, int W) {
    auto enc = get_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)3 * W, (cuuint64_t)H, (cuuint64_t)frames};
    cuuint64_t strides[2] = {(cuuint64_t)6 * W, (cuuint64_t)6 * W * H};
    cuuint32_t box[3] = {(cuuint32_t)XB, 3, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool stem_form_ok(const StemArgs& a) {
    return (a.Cout == 64 || a.Cout == 128) && a.Cout_pad == a.Cout && a.Kpad == 128 && a.N > 0 && a.Tin > 0 &&
           a.Tout > 0 && a.H >= 2 && a.H % 2 == 0 && a.W >= 8 && a.W % 8 == 0 && (a.st == 1 || a.st == 2) &&
           aligned16(a.x) && aligned16(a.out) && aligned16(a.w) && (!a.hist || (aligned16(a.hist) && a.hist_T > 0));
}

template <int CO, int MAXP>
int launch_co(const StemArgs* as, int count, int num_sms, cudaStream_t stream, int cta_tiles) {
    using C = StemCfg<CO>;
    auto kern = stem_tc_kernel<CO, MAXP>;
    StemBatch<MAXP> B;
    memset(&B, 0, sizeof(B));
    if (!encode_w_map(&B.tm_w, as[0].w, as[0].Cout_pad, as[0].Kpad, CO, 64)) return kStemDeclined;
    long long total = 0;
    for (int p = 0; p < count; ++p) {
        const StemArgs& a = as[p];
        StemProb& q = B.q[p];
        q.N = a.N;
        q.Tin = a.Tin;
        q.Tout = a.Tout;
        q.Hout = a.H / 2;
        q.Wout = a.W / 2;
        q.st = a.st;
        q.t_off = a.t_off;
        q.pad_mode = a.pad_mode;
        q.tiles_w = (q.Wout + SV - 1) / SV;
        q.gn_part = a.gn_part;
        if (!encode_pixels_map(&q.tm_x, a.x, (long long)a.N * a.Tin, a.H, a.W)) return kStemDeclined;
        if (a.hist) {
            if (!encode_pixels_map(&q.tm_h, a.hist, (long long)a.N * a.hist_T, a.H, a.W)) return kStemDeclined;
            q.has_hist = 1;
            q.hist_T = a.hist_T;
        } else {
            q.tm_h = q.tm_x;
        }
        q.out = static_cast<__nv_bfloat16*>(a.out);
        total += (long long)a.N * a.Tout * q.Hout * q.tiles_w;
        q.tile_end = total;
    }
    B.bias = as[0].bias;
    B.status = as[0].status;
    B.wait_ns = as[0].wait_ns;
    B.num_tiles = total;
    B.count = count;
    if (total == 0) return 0;
    if (total >= (1LL << 31)) return kStemDeclined;
    static std::atomic<unsigned long long> attr_done{0};
    if (smem_attr_once(kern, C::SMEM, attr_done) != cudaSuccess) return (int)cudaGetLastError();
    // persistent (one CTA per SM), or CTAs of at most cta_tiles tiles each
    long long grid = std::min<long long>(total, num_sms);
    if (cta_tiles > 0) grid = std::max(grid, std::min<long long>((total + cta_tiles - 1) / cta_tiles, 1LL << 30));
    kern<<<(unsigned)grid, NTHREADS, C::SMEM, stream>>>(B);
    return (int)cudaGetLastError();
}

template <int CO>
int launch_cog(const StemArgs* as, int count, int num_sms, cudaStream_t stream, int cta_tiles) {
    return count == 1 ? launch_co<CO, 1>(as, 1, num_sms, stream, cta_tiles)
                      : launch_co<CO, kMaxConvGroup>(as, count, num_sms, stream, cta_tiles);
}

}  // namespace

int stem_tc_gn_slots(int H, int W) { return (H / 2) * ((W / 2 + SV - 1) / SV); }

bool stem_tc_accepts(const StemArgs* as, int count) {
    if (count < 1 || count > kMaxConvGroup) return false;
    for (int p = 0; p < count; ++p)
        if (!stem_form_ok(as[p]) || as[p].Cout != as[0].Cout || as[p].w != as[0].w) return false;
    return true;
}

int launch_stem_tc(const StemArgs* as, int count, int num_sms, cudaStream_t stream, int cta_tiles) {
    if (!stem_tc_accepts(as, count)) return kStemDeclined;
    return as[0].Cout == 64 ? launch_cog<64>(as, count, num_sms, stream, cta_tiles)
                            : launch_cog<128>(as, count, num_sms, stream, cta_tiles);
}

}  // namespace tok
