// BF16 causal 3D convolution on the 5th-generation tensor cores (sm_103a).
//
// Implicit GEMM: M = output voxels, N = output channels, K = taps x Cin.
// Persistent CTAs (one per SM, or CTAs of a bounded number of tiles) walk
// output tiles; a voxel tile is a BH x BW block of one output frame. A K block
// is one tap (dt,dh,dw) x 64 input channels, fetched by one TMA box load of
// the input frame at the tap's offset (boundary padding = TMA out-of-bounds
// zero fill; stride-2 convs read a parity view of the input, see the host
// side) -- or, for stride-1 3x3x3 layers (the halo form), one (dt, dw, 64
// channels) group: a single box of BH + 2 rows serves the three dh taps. The
// time-causal left padding is folded into the loader: a tap that falls
// before frame 0 reads the stream's history tensor (streaming), frame 0
// (replicate) or nothing (zero fill via an out-of-range coordinate).
//
// Warp roles (192 threads):
//   warp 0      TMA producer (one lane): activation and weight boxes into a
//               ring of 128B-swizzled shared-memory stages, or (the wide halo
//               form) into separate rings of activation and weight slots.
//   warp 1      TMEM allocation and MMA issue (one lane): tcgen05.mma.kind::f16
//               (K = 16 each) per stage into one of two FP32 accumulators in
//               TMEM; tcgen05.commit frees the stage (or slot).
//   warps 2..5  epilogue: tcgen05.ld the accumulator (each warp its 32 TMEM
//               lanes), add bias and residual, round to BF16 and store; or
//               scatter through depth-to-space; or FSQ-quantise (rounding
//               thresholds on z); and reduce
//               the GroupNorm statistics of the stored values.
// The epilogue of tile i overlaps the MMAs of tile i+1 (double-buffered TMEM).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "conv_args.h"

namespace tok {

bool encode_act_map(CUtensorMap* m, const void* base, int frames, int H, int W, int C, int BH, int BW, bool strided,
                    int kc = 64);
bool encode_w_map(CUtensorMap* m, const void* base, int rows, int Kpad, int BN, int kc = 64);

struct TcGeo {
    int BH, BW;              // output tile = BH rows x BW cols of one frame
    int tiles_w, tiles_h;
    int n_tiles;             // Cout_pad / BN
    long long num_tiles;     // m tiles x n tiles
    int cpt;                 // KC-channel blocks per tap
    int nkb;                 // K blocks per tile = taps * cpt
    int strided;             // parity view (sh = sw = 2)
    long long m_tiles;       // voxel tiles
    int halo;                // K blocks are (dt, dw, channel block) groups of three dh taps
    int bwo;                 // output columns per tile: BW, or BW - 2 in the dw-rows form (DWM)
    int nvox;                // swapped forms: voxels per tile = BH * BW = the MMA's N (16 | nvox, <= 256)
    int bho;                 // output rows per tile: BH, or BH - 2 when all nine taps are MMA rows
};

// A grouped launch: up to MAXP inputs of one layer (clips or stream chunks of
// different sizes), one weight tensor. Tiles are numbered problem after
// problem (tile_end holds the running totals) and a tile never spans two
// problems; the persistent CTAs stride over all of them. unit_end holds the
// running totals of tiles per problem.
template <int MAXP>
struct TcBatch {
    CUtensorMap tm_w;
    CUtensorMap tm_w0;  // weights of the output-frame-0 tiles (a.w0), else a copy of tm_w
    int w_rows;  // rows of each weight box: BN, or the 16/32 real rows of a narrow halo layer
    CUtensorMap tm_x[MAXP];
    CUtensorMap tm_h[MAXP];
    ConvArgs a[MAXP];
    TcGeo g[MAXP];
    long long unit_end[MAXP];
    long long num_units;
    int count;
    int na;        // split rings: activation slots in flight (2..4)
    int act_slot;  // split rings: bytes per activation slot (a multiple of 1 KB)
};

namespace {

// Two operand arrangements of the same implicit GEMM:
//  SWAP = false: MMA M = 128 voxels, N = BN output channels (A = activations).
//  SWAP = true : MMA M = 128 output channels, N = 256 voxels (A = weights), for
//                layers with exactly 128 output channels: an M128 x N256 MMA
//                reads 12 KB of operands from shared memory per 128 tensor
//                cycles where M128 x N128 reads 8 KB per 64, so the wide form
//                keeps the tensor pipe fed. TMEM then holds D^T (lanes =
//                channels, columns = voxels) and the epilogue transposes
//                through a small per-warp staging buffer.
//  HALO        : stride-1 3x3x3 layers load, per (dt, dw, 64-channel block),
//                one box of BH + 2 input rows that serves the three dh taps:
//                tap dh reads the box from row dh * BW on, a whole number of
//                1 KB swizzle atoms for BW = 16, 32, 64, so the operand
//                descriptor simply starts there. Three weight boxes (one per
//                dh) go into the same stage. The activation bytes per K block
//                drop from ROWS to (ROWS + 2 BW) / 3 voxel rows.
//                BW = 16, 32 or 64. Halo layers run swapped; a narrow layer (at
//                most 32 channels) loads only its 16 or 32 weight rows per tap
//                into weight slots whose other rows stay zero.
constexpr int HALO_BW_MAX = 64;
// Input channels per K block of the wide halo form: 64 (128-byte rows) or 32
// (64-byte rows, four 48 KB stages of the unified ring). What bounds the form,
// measured on the level-0 layer of the 720p step (17 x 360 x 640, 128 -> 128
// channels, 3.47 TFLOP, before the clocks drop under the power cap): the whole
// kernel 1.95-2.05 ms; with the epilogue's work left out 1.91-1.94 ms; with the
// TMA fills left out (MMAs over whatever the slots hold) 1.71 ms, and 1.67 ms
// with neither, i.e. 2070 TFLOP/s. The fills (84 KB per K block for 256 voxels)
// and the MMAs' operand reads (12 KB per 128-cycle M128 x N256 x K16 MMA) share
// the SM's shared-memory bandwidth, where ncu counts the tensor core's reads at
// 59.5 % and the fills at 36.4 % of it. Deeper pipelines do not change that
// (32-channel blocks: no gain; the split rings below: 2 %); fewer fill bytes per
// FLOP would, and for a layer of 128 output channels that takes accumulators of
// more than 256 voxels, which leave no second TMEM buffer for the epilogue.
constexpr int kHaloKC = 64;
constexpr bool kHaloSplit = true;  // 64-channel K blocks in the split rings (see Cfg)
constexpr int DWM_BH = 8, DWM_BW = 32;  // taps-in-rows forms: rows (dw rows: output rows) x columns of a tile's box

//                HALO = number of 64-channel blocks per stage (0: no halo).
//                TR: taps in the MMA rows. 3: the dw rows (a 10 x 32 box, weight slots of
//                64 rows); 9: the (dh, dw) rows (an 8 x 32 box, one 128-row weight slot).
//                KC: input channels per K block (64: rows of 128 B, 128-byte swizzle;
//                32: rows of 64 B, 64-byte swizzle, stages half as large and twice
//                as many in flight).
//                SPLIT: separate rings for the wide halo form (KC = 64): NW weight
//                slots of one dh tap each (16 KB), and activation slots sized at
//                launch for the largest box of the launch (2..4 of them in the
//                rest of the 227 KB). One stage of the unified ring (box + three
//                weight boxes, up to 96 KB) allows two stages in flight; the split
//                rings keep two K blocks of weights and three boxes in flight and
//                let the first dh tap's MMAs start before the other two weight
//                boxes land (measured 2 % faster on the level-0 layer).
template <int BN, bool SWAP, int HALO = 0, int TR = 0, int KC = 64, bool SPLIT = false>
struct Cfg {
    static_assert(!SPLIT || (HALO == 1 && TR == 0 && KC == 64 && SWAP), "split rings: the wide halo form");
    static_assert(KC == 64 || (KC == 32 && TR == 0), "32-channel K blocks: plain and halo forms");
    static constexpr int ROWB = KC * 2;            // bytes of one voxel's (or weight row's) K block
    static constexpr int ROWS = SWAP ? 256 : 128;  // voxels per tile
    static constexpr int HALO_BW = HALO_BW_MAX;
    // one channel block's input box
    static constexpr int SUB_ACT = TR == 3   ? (DWM_BH + 2) * DWM_BW * ROWB
                                   : TR == 9 ? DWM_BH * DWM_BW * ROWB
                                             : (ROWS + (HALO ? 2 * HALO_BW : 0)) * ROWB;
    static constexpr int ACT_BYTES = (HALO ? HALO : 1) * SUB_ACT;  // KC bf16 channels per row
    static constexpr int W_TAP_BYTES = (TR == 3 ? 64 : BN) * ROWB;
    static constexpr int W_BYTES = (TR == 9 ? HALO : HALO ? 3 * HALO : 1) * W_TAP_BYTES;
    static constexpr int STAGE = ACT_BYTES + W_BYTES;
    static constexpr int STAGES = (200 * 1024 / STAGE) > 8 ? 8 : (200 * 1024 / STAGE);
    static constexpr int ACC_COLS = SWAP ? ROWS : BN;  // TMEM columns per accumulator
    static constexpr int TMEM_COLS = (2 * ACC_COLS <= 32) ? 32 : (2 * ACC_COLS <= 64) ? 64 : (2 * ACC_COLS <= 128) ? 128 : (2 * ACC_COLS <= 256) ? 256 : 512;
    static constexpr int BAR_BYTES = 256;
    static constexpr int EPI_STRIDE = 36;  // floats per staged voxel row (16B-aligned, bank-spread)
    // (nine taps in rows: a staged box row of 128 accumulator rows and one output row of 16 channels)
    // (unswapped: per epilogue warp 32 voxel rows of 64 bf16 channels)
    static constexpr int EPI_BYTES = TR == 9 ? (128 + 16) * 33 * 4 : SWAP ? 4 * 16 * EPI_STRIDE * 4 : 4 * 32 * 128;
    static constexpr int NW = 6;                  // split rings: weight slots
    static constexpr int W_SLOT = BN * ROWB;      // split rings: one dh tap's weight box
    // a CTA's shared memory (227 KB) holds the kernel's static variables too: 64 bytes
    // are left for them; aligning the (16-byte aligned) dynamic base to 1 KB costs at
    // most 1008 bytes
    static constexpr int SMEM_LIMIT = 232448 - 64;
    static constexpr int SLACK = SPLIT ? 1008 : 1024;
    static constexpr int SPLIT_ACT_BYTES = SMEM_LIMIT - NW * W_SLOT - SLACK - BAR_BYTES - EPI_BYTES;
    static constexpr int BAR_OFF = SPLIT ? NW * W_SLOT + SPLIT_ACT_BYTES : STAGES * STAGE;
    static constexpr int SMEM = BAR_OFF + SLACK + BAR_BYTES + EPI_BYTES;
    static_assert(SMEM <= SMEM_LIMIT, "shared memory");
    // (the swapped halo forms build theirs per tile: N = the tile's voxels, and M = 64
    // for heads of at most 16 rows, whose output channel r stays in TMEM lane r)
    static constexpr uint32_t IDESC = SWAP ? idesc_bf16_f32(BN, ROWS) : idesc_bf16_f32(128, BN);
};

struct TileCoord {
    int n, to, th, tw, nt;
};

// Operand descriptor of a K block of KC channels (128- or 64-byte swizzle).
template <int KC>
__device__ __forceinline__ uint64_t kdesc(uint32_t addr) {
    if constexpr (KC == 64)
        return sw128_desc(addr);
    else
        return sw64_desc(addr);
}

// Voxel tiles are numbered with the output frame fastest: the CTAs working at
// the same time cover a few spatial blocks across all frames, so an input
// frame is fetched into L2 once and read there by the three output frames
// whose temporal taps need it, instead of again after a whole frame of tiles.
__device__ __forceinline__ TileCoord decode_tile(const ConvArgs& a, const TcGeo& g, long long tile) {
    TileCoord c;
    c.nt = (int)(tile % g.n_tiles);
    long long m = tile / g.n_tiles;
    c.to = (int)(m % a.Tout);
    m /= a.Tout;
    c.tw = (int)(m % g.tiles_w);
    m /= g.tiles_w;
    c.th = (int)(m % g.tiles_h);
    c.n = (int)(m / g.tiles_h);
    return c;
}

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16* dst, const float (&v)[16]) {
    uint4 o0, o1;
    o0.x = pack_bf16x2(v[0], v[1]);
    o0.y = pack_bf16x2(v[2], v[3]);
    o0.z = pack_bf16x2(v[4], v[5]);
    o0.w = pack_bf16x2(v[6], v[7]);
    o1.x = pack_bf16x2(v[8], v[9]);
    o1.y = pack_bf16x2(v[10], v[11]);
    o1.z = pack_bf16x2(v[12], v[13]);
    o1.w = pack_bf16x2(v[14], v[15]);
    reinterpret_cast<uint4*>(dst)[0] = o0;
    reinterpret_cast<uint4*>(dst)[1] = o1;
}

__device__ __forceinline__ void add_bf16x16(const __nv_bfloat16* src, float (&v)[16]) {
    uint4 r0 = reinterpret_cast<const uint4*>(src)[0];
    uint4 r1 = reinterpret_cast<const uint4*>(src)[1];
    uint32_t u[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 f = unpack_bf16x2(u[i]);
        v[2 * i] += f.x;
        v[2 * i + 1] += f.y;
    }
}

__device__ __forceinline__ GnTriple gn_merge(GnTriple a, GnTriple b) {
    if (b.n == 0.f) return a;
    if (a.n == 0.f) return b;
    GnTriple r;
    r.n = a.n + b.n;
    const float d = b.mean - a.mean;
    const float fb = b.n / r.n;
    r.mean = a.mean + d * fb;
    r.m2 = a.m2 + b.m2 + d * d * a.n * fb;
    return r;
}

__device__ __forceinline__ GnTriple gn_shfl_down(GnTriple t, int o) {
    GnTriple b;
    b.n = __shfl_down_sync(0xffffffffu, t.n, o);
    b.mean = __shfl_down_sync(0xffffffffu, t.mean, o);
    b.m2 = __shfl_down_sync(0xffffffffu, t.m2, o);
    return b;
}

// Frame coordinate of input frame ti of sample n in the map *src it is read from:
// frames past the last read zeros (adjoint convs read ahead), frames before the
// first read the stream's history, frame 0 (replicate padding) or zeros.
template <int MAXP>
__device__ __forceinline__ int tap_frame(const TcBatch<MAXP>& B, int p, int n, int ti, const CUtensorMap** src) {
    const ConvArgs& a = B.a[p];
    *src = &B.tm_x[p];
    if (ti >= a.Tin) return -1;  // whole box out of range -> zeros
    if (ti >= 0) return n * a.Tin + ti;
    if (a.hist) {
        *src = &B.tm_h[p];
        return n * a.hist_T + a.hist_T + ti;
    }
    return a.pad_mode == 0 ? n * a.Tin : -1;
}

// Problem of a global unit index and the unit's index within that problem.
template <int MAXP>
__device__ __forceinline__ int problem_of(const TcBatch<MAXP>& B, long long unit, long long* local) {
    int p = 0;
    if constexpr (MAXP > 1)
        while (p + 1 < B.count && unit >= B.unit_end[p]) ++p;
    *local = p ? unit - B.unit_end[p - 1] : unit;
    return p;
}

// One CTA per tile; persistent CTAs stride over the tiles of all problems.
// DWM (narrow heads of at most 16 channels, swapped halo form): the three dw
// taps are MMA rows (row dw * 16 + co, 48 of 64), so a K block is (dt, 64
// channels) with the three dh taps inside and an input box 32 columns wide
// serves 30 output columns; the epilogue adds the dw rows with their column
// shift: out[co][x] = D[co][x] + D[16 + co][x + 1] + D[32 + co][x + 2].
//
// Nine taps in rows (narrow heads with 9 * Cout <= 128): the weights are rows
// (dh * 3 + dw) * Cout + co over K = (dt, ci), so one M = 128 MMA computes all
// nine spatial taps and a K block is (dt, 64 channels) with one 8 x 32 input
// box (6 x 30 outputs); the epilogue adds the tap rows with their row and
// column shifts, out[co][y][x] = sum over dh, dw of D[(dh, dw, co)][y + dh][x + dw].
template <int BN, bool SWAP, int MAXP, int HALO, int TR = 0, int KC = 64, bool SPLIT = false>
__global__ void __launch_bounds__(192, 1) conv_tc_kernel(const __grid_constant__ TcBatch<MAXP> B) {
    using C = Cfg<BN, SWAP, HALO, TR, KC, SPLIT>;
    constexpr bool DWM = TR == 3, T9 = TR == 9;
    constexpr int NDH = T9 ? 1 : 3;  // weight boxes (dh taps) per channel block of a K block
    static_assert(TR == 0 || ((TR == 3 || TR == 9) && SWAP && HALO == 1), "taps in rows: swapped halo form");
    int* const status = B.a[0].status;
    const unsigned long long wait_ns = B.a[0].wait_ns;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
    // full/empty: the stages of the unified ring, or the activation slots of the split
    // rings (wfull/wempty: their weight slots)
    constexpr int NFE = SPLIT ? 4 : C::STAGES, NWB = SPLIT ? C::NW : 0;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
    uint64_t* empty = full + NFE;
    uint64_t* wfull = empty + NFE;
    uint64_t* wempty = wfull + NWB;
    uint64_t* tfull = wempty + NWB;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
    float* epi = reinterpret_cast<float*>(smem + C::BAR_OFF + C::BAR_BYTES);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long cid = blockIdx.x, ncl = gridDim.x;
    // A context already in error skips the launch (decided once per CTA).
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (status && *(volatile int*)status != 0) ? 1 : 0;
    __syncthreads();
    if (s_skip) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NFE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < NWB; ++s) {
            mbar_init(&wfull[s], 1);
            mbar_init(&wempty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 4);
        }
        fence_mbar_init();
    }
    if constexpr (HALO > 0 && !SPLIT) {
        // narrow layer: the weight boxes fill only the first w_rows rows of each
        // 128-row weight slot; the others are zero for the whole launch
        if (B.w_rows < BN) {
            for (int st = 0; st < C::STAGES; ++st) {
                uint4* wz = reinterpret_cast<uint4*>(smem + st * C::STAGE + C::ACT_BYTES);
                for (int i = threadIdx.x; i < C::W_BYTES / 16; i += blockDim.x) wz[i] = make_uint4(0u, 0u, 0u, 0u);
            }
            fence_proxy_async_smem();
        }
    }
    if (warp == 0 && lane < B.count) {
        tma_prefetch_desc(&B.tm_x[lane]);
        if (B.a[lane].hist) tma_prefetch_desc(&B.tm_h[lane]);
        if (lane == 0) tma_prefetch_desc(&B.tm_w);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (SPLIT && lane == 0) {
            // ------------------------------------------------ TMA producer, split rings
            // per K block (dt, dw, 64 channels): the box into the next activation slot,
            // then the three dh taps' weight boxes into the next three weight slots
            int sa = 0, sw = 0;
            uint32_t pa = 0, pw = 0;
            int last_a[4] = {-1, -1, -1, -1}, last_w[C::NW];
#pragma unroll
            for (int i = 0; i < C::NW; ++i) last_w[i] = -1;
            const int na = B.na;
            const uint32_t w_bytes = (uint32_t)(B.w_rows * C::ROWB);
            bool ok = true;
            for (long long u = cid; u < B.num_units && ok; u += ncl) {
                long long lu;
                const int p = problem_of(B, u, &lu);
                const ConvArgs& a = B.a[p];
                const TcGeo& g = B.g[p];
                const TileCoord tc = decode_tile(a, g, lu);
                const uint32_t act_bytes = (uint32_t)((g.BH + 2) * g.BW * C::ROWB);
                const CUtensorMap* wmap = (tc.to == 0) ? &B.tm_w0 : &B.tm_w;
                for (int kb = 0; kb < g.nkb && ok; ++kb) {
                    const int tap = kb / g.cpt, cb = kb - tap * g.cpt;
                    const int dw = tap % 3, dt = tap / 3;
                    const CUtensorMap* src;
                    const int tcoord = tap_frame(B, p, tc.n, tc.to * a.st + dt + a.t_off, &src);
                    if (!mbar_wait(&empty[sa], pa ^ 1, status, wait_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[sa], act_bytes);
                    tma_load_4d(smem + C::NW * C::W_SLOT + sa * B.act_slot, src, &full[sa], cb * KC,
                                tc.tw * g.BW + dw - 1, tc.th * g.BH - 1, tcoord);
                    last_a[sa] = (int)pa;
                    if (++sa == na) {
                        sa = 0;
                        pa ^= 1;
                    }
                    for (int d = 0; d < 3; ++d) {
                        if (!mbar_wait(&wempty[sw], pw ^ 1, status, wait_ns)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&wfull[sw], w_bytes);
                        tma_load_2d(smem + sw * C::W_SLOT, wmap, &wfull[sw], ((dt * 3 + d) * 3 + dw) * a.Cin + cb * KC,
                                    tc.nt * BN);
                        last_w[sw] = (int)pw;
                        if (++sw == C::NW) {
                            sw = 0;
                            pw ^= 1;
                        }
                    }
                }
            }
            // no copy may still be in flight when the CTA exits
            for (int i = 0; i < na; ++i)
                if (last_a[i] >= 0) mbar_wait(&full[i], (uint32_t)last_a[i], status, wait_ns);
            for (int i = 0; i < C::NW; ++i)
                if (last_w[i] >= 0) mbar_wait(&wfull[i], (uint32_t)last_w[i], status, wait_ns);
        } else if (lane == 0) {
            // ------------------------------------------------ TMA producer
            int s = 0;
            uint32_t ph = 0;
            int last_ph[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) last_ph[i] = -1;
            bool ok = true;
            for (long long u = cid; u < B.num_units && ok; u += ncl) {
                long long lu;
                const int p = problem_of(B, u, &lu);
                const ConvArgs& a = B.a[p];
                const TcGeo& g = B.g[p];
                const int ph_ = (a.kh - 1) / 2, pw_ = (a.kw - 1) / 2;
                const TileCoord tc = decode_tile(a, g, lu);
                for (int kb = 0; kb < g.nkb; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1, status, wait_ns)) {
                        ok = false;
                        break;
                    }
                    // plain: kb = (tap, cb); halo: kb = (dt, dw, block group) with the three dh taps
                    // and HALO channel blocks inside
                    const int cpg = HALO ? g.cpt / HALO : g.cpt;
                    const int tap = kb / cpg, cb = kb - tap * cpg;
                    const int dw = TR ? 0 : (HALO ? tap % 3 : tap % a.kw);
                    const int dh = HALO ? 0 : (tap / a.kw) % a.kh;
                    const int dt = TR ? tap : (HALO ? tap / 3 : tap / (a.kw * a.kh));
                    const CUtensorMap* src;
                    const int tcoord = tap_frame(B, p, tc.n, tc.to * a.st + dt + a.t_off, &src);
                    uint8_t* sa = smem + s * C::STAGE;
                    uint8_t* sb = sa + C::ACT_BYTES;
                    const CUtensorMap* wmap = (tc.to == 0) ? &B.tm_w0 : &B.tm_w;
                    if constexpr (HALO > 0) {
                        // rows th*BH - 1 .. th*BH + BH of the input frame (zeros outside), per block
                        // (nine taps in rows: a box of BH rows, th*bho - 1 .. th*bho + bho)
                        mbar_arrive_expect_tx(&full[s], (uint32_t)(HALO * ((T9 ? g.BH : g.BH + 2) * g.BW * C::ROWB +
                                                                           NDH * B.w_rows * C::ROWB)));
#pragma unroll
                        for (int c = 0; c < HALO; ++c) {
                            const int ci = (cb * HALO + c) * KC;
                            // taps in rows: columns tw*bwo - 1 .. tw*bwo + bwo of the input (all three dw)
                            tma_load_4d(sa + c * C::SUB_ACT, src, &full[s], ci,
                                        TR ? tc.tw * g.bwo - 1 : tc.tw * g.BW + dw - 1, tc.th * g.bho - 1, tcoord);
#pragma unroll
                            for (int d = 0; d < NDH; ++d) {
                                const int kw0 = T9    ? dt * a.Cin + ci
                                                : DWM ? (dt * 3 + d) * a.Cin + ci
                                                      : ((dt * 3 + d) * 3 + dw) * a.Cin + ci;
                                tma_load_2d(sb + (c * NDH + d) * C::W_TAP_BYTES, wmap, &full[s], kw0, tc.nt * BN);
                            }
                        }
                        last_ph[s] = (int)ph;
                        if (++s == C::STAGES) {
                            s = 0;
                            ph ^= 1;
                        }
                        continue;
                    }
                    mbar_arrive_expect_tx(&full[s], C::STAGE);
                    if (!g.strided) {
                        tma_load_4d(sa, src, &full[s], cb * KC, tc.tw * g.BW + dw - pw_, tc.th * g.BH + dh - ph_,
                                    tcoord);
                    } else {
                        const int pwp = (dw == 1) ? 0 : 1, php = (dh == 1) ? 0 : 1;
                        tma_load_5d(sa, src, &full[s], pwp * a.Cin + cb * KC, tc.tw * g.BW + (dw == 0 ? -1 : 0), php,
                                    tc.th * g.BH + (dh == 0 ? -1 : 0), tcoord);
                    }
                    tma_load_2d(sb, wmap, &full[s], tap * a.Cin + cb * KC, tc.nt * BN);
                    last_ph[s] = (int)ph;
                    if (++s == C::STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
            }
            // make sure no copy is still in flight before the CTA may exit
            for (int i = 0; i < C::STAGES; ++i)
                if (last_ph[i] >= 0) mbar_wait(&full[i], (uint32_t)last_ph[i], status, wait_ns);
        }
    } else if (warp == 1) {
        if (SPLIT && lane == 0) {
            // ------------------------------------------------ MMA issuer, split rings
            // per K block: wait for the box, then per dh tap for its weight slot, four
            // MMAs (K = 16 each) reading the box from row dh * BW on, and release that
            // weight slot; the box is released after the third tap
            int sa = 0, sw = 0;
            uint32_t pa = 0, pw = 0;
            const int na = B.na;
            int last_acc_ph[2] = {-1, -1};
            bool ok = true;
            int it = 0;
            for (long long u = cid; u < B.num_units && ok; u += ncl, ++it) {
                long long lu;
                const TcGeo& gu = B.g[problem_of(B, u, &lu)];
                const uint32_t row_step = (uint32_t)gu.BW * C::ROWB;
                const uint32_t idesc = idesc_bf16_f32(BN, gu.nvox);
                const int acc = it & 1;
                const uint32_t aph = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(&tempty[acc], aph ^ 1, status, wait_ns)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * C::ACC_COLS);
                for (int kb = 0; kb < gu.nkb && ok; ++kb) {
                    if (!mbar_wait(&full[sa], pa, status, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t xa = smem_u32(smem + C::NW * C::W_SLOT + sa * B.act_slot);
                    for (int dh = 0; dh < 3; ++dh) {
                        if (!mbar_wait(&wfull[sw], pw, status, wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t wa = smem_u32(smem + sw * C::W_SLOT);
#pragma unroll
                        for (int k = 0; k < KC / 16; ++k)
                            tc_mma_bf16(d, kdesc<KC>(wa + k * 32), kdesc<KC>(xa + (uint32_t)dh * row_step + k * 32), idesc,
                                        (kb | dh | k) != 0 ? 1u : 0u);
                        tc_commit(&wempty[sw]);
                        if (++sw == C::NW) {
                            sw = 0;
                            pw ^= 1;
                        }
                    }
                    if (!ok) break;
                    tc_commit(&empty[sa]);
                    if (++sa == na) {
                        sa = 0;
                        pa ^= 1;
                    }
                }
                tc_commit(&tfull[acc]);
                last_acc_ph[acc] = (int)aph;
            }
            // wait for our own MMAs before TMEM can be released
            for (int i = 0; i < 2; ++i)
                if (last_acc_ph[i] >= 0) mbar_wait(&tfull[i], (uint32_t)last_acc_ph[i], status, wait_ns);
        } else if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            int s = 0;
            uint32_t ph = 0;
            int last_acc_ph[2] = {-1, -1};
            bool ok = true;
            int it = 0;
            for (long long u = cid; u < B.num_units && ok; u += ncl, ++it) {
                long long lu;
                const TcGeo& gu = B.g[problem_of(B, u, &lu)];
                const int nkb = gu.nkb;
                const uint32_t row_step = (uint32_t)gu.BW * C::ROWB;  // one input row of the halo box
                const int acc = it & 1;
                const uint32_t aph = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(&tempty[acc], aph ^ 1, status, wait_ns)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * C::ACC_COLS);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&full[s], ph, status, wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t s_act = smem_u32(smem + s * C::STAGE);
                    const uint32_t s_w = s_act + C::ACT_BYTES;
                    if constexpr (HALO > 0) {
                        const uint32_t idesc =
                            SWAP ? idesc_bf16_f32((DWM || B.w_rows <= 16) ? 64 : BN, gu.nvox) : C::IDESC;
#pragma unroll
                        for (int c = 0; c < HALO; ++c)
#pragma unroll
                            for (int dh = 0; dh < NDH; ++dh) {
                                const uint32_t xa = s_act + (uint32_t)(c * C::SUB_ACT) + (uint32_t)dh * row_step;
                                const uint32_t wa = s_w + (uint32_t)((c * NDH + dh) * C::W_TAP_BYTES);
                                const uint32_t op_a = SWAP ? wa : xa, op_b = SWAP ? xa : wa;
#pragma unroll
                                for (int k = 0; k < KC / 16; ++k)
                                    tc_mma_bf16(d, kdesc<KC>(op_a + k * 32), kdesc<KC>(op_b + k * 32), idesc,
                                                (kb | c | dh | k) != 0 ? 1u : 0u);
                            }
                    } else {
                        const uint32_t op_a = SWAP ? s_w : s_act, op_b = SWAP ? s_act : s_w;
#pragma unroll
                        for (int k = 0; k < KC / 16; ++k)
                            tc_mma_bf16(d, kdesc<KC>(op_a + k * 32), kdesc<KC>(op_b + k * 32), C::IDESC,
                                        (kb | k) != 0 ? 1u : 0u);
                    }
                    tc_commit(&empty[s]);
                    if (++s == C::STAGES) {
                        s = 0;
                        ph ^= 1;
                    }
                }
                tc_commit(&tfull[acc]);
                last_acc_ph[acc] = (int)aph;
            }
            // wait for our own MMAs before TMEM can be released
            for (int i = 0; i < 2; ++i)
                if (last_acc_ph[i] >= 0) mbar_wait(&tfull[i], (uint32_t)last_acc_ph[i], status, wait_ns);
        }
    } else {
        // ---------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quarter accessible to this warp
        const int r = q * 32 + lane;
        int it = 0;
        for (long long u = cid; u < B.num_units; u += ncl, ++it) {
            const int acc = it & 1;
            const uint32_t aph = (uint32_t)((it >> 1) & 1);
            int okw = 1;
            if (lane == 0) okw = mbar_wait(&tfull[acc], aph, status, wait_ns) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) break;
            tc_fence_after();
            long long lu;
            const int p = problem_of(B, u, &lu);
            const ConvArgs& a = B.a[p];
            const TcGeo& g = B.g[p];
            const TileCoord tc = decode_tile(a, g, lu);
            if constexpr (SWAP) {
                // lane = output channel co, TMEM column = voxel of the 256-voxel tile
                const int co = tc.nt * BN + r;
                const float bias = (a.bias && co < a.Cout) ? a.bias[co] : 0.f;
                float* stg = epi + q * 16 * C::EPI_STRIDE;
                const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * C::ACC_COLS);
                const int j = lane >> 1, half = lane & 1;  // read-back role: voxel j, 16 channels
                if constexpr (T9) {
                    // Row r = (dh * 3 + dw) * Cout + co of the M = 128 accumulator is TMEM lane
                    // r. Box row b (32 columns) at a time is staged in shared memory; thread t
                    // keeps channel co = t & 15 at columns x = t / 16 + 8 i and three running
                    // sums, for output rows b, b - 1 and b - 2, which take tap row dh of box
                    // row b into output row b - dh; output row b - 2 is complete after box row b.
                    float* buf = epi;              // [128 rows][33]
                    float* orow = epi + 128 * 33;  // [16 channels][33]: a finished output row (FSQ)
                    const int t = q * 32 + lane;
                    const int co = t & 15, xg = t >> 4;
                    const int Co = a.Cout, rows_used = 9 * Co;
                    const int Hout = a.Hout, Wout = a.Wout, oT = a.oT, oH = a.oH, oW = a.oW, oC = a.oC;
                    const int bwo = g.bwo, wo0 = tc.tw * bwo;
                    const bool fsq = a.mode == OUT_FSQ, f32 = a.out_fp32 != 0;
                    int ch = co, cc = 0, bb = 0, rw = 1, rh = 1, ot = tc.to;
                    if (a.mode == OUT_D2S) {
                        const int sub = co / oC;
                        ch = co - sub * oC;
                        rw = a.rw;
                        rh = a.rh;
                        cc = sub % rw;
                        bb = (sub / rw) % rh;
                        ot = tc.to * a.rt + sub / (rw * rh) - a.drop_t;
                    }
                    const bool c_ok = co < Co && ot >= 0 && ot < oT;
                    const float bias_c = (a.bias && co < Co) ? a.bias[co] : 0.f;
                    const __nv_bfloat16* const resid = static_cast<const __nv_bfloat16*>(a.residual);
                    void* const out = a.out;
                    float s0[4], s1[4], s2[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) s0[i] = s1[i] = s2[i] = 0.f;
                    for (int b = 0; b < g.BH; ++b) {
                        {
                            float v[16];
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                tmem_ld16(tbase + (uint32_t)(b * 32 + h2 * 16), v);
                                if (t < rows_used) {
#pragma unroll
                                    for (int i2 = 0; i2 < 16; ++i2) buf[t * 33 + h2 * 16 + i2] = v[i2];
                                }
                            }
                        }
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                        if (co < Co) {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int x = xg + 8 * i;
                                if (x < bwo) {
                                    float p[3];
#pragma unroll
                                    for (int dh = 0; dh < 3; ++dh) {
                                        const float* r0 = buf + ((dh * 3) * Co + co) * 33 + x;
                                        p[dh] = r0[0] + r0[Co * 33 + 1] + r0[2 * Co * 33 + 2];
                                    }
                                    s0[i] += p[0];
                                    s1[i] += p[1];
                                    s2[i] += p[2];
                                }
                            }
                        }
                        const int yo = b - 2, ho = tc.th * g.bho + yo;
                        if (yo >= 0 && yo < g.bho && ho < Hout) {
                            if (fsq) {
                                if (co < Co) {
#pragma unroll
                                    for (int i = 0; i < 4; ++i)
                                        if (xg + 8 * i < bwo) orow[co * 33 + xg + 8 * i] = s2[i] + bias_c;
                                }
                                asm volatile("bar.sync 1, 128;" ::: "memory");
                                const int x = t >> 2;
                                if ((t & 3) == 0 && x < bwo && wo0 + x < Wout) {
                                    const long long vox =
                                        (((long long)tc.n * a.Tout + tc.to) * Hout + ho) * Wout + wo0 + x;
                                    float* z = static_cast<float*>(out) + vox * a.fsq.nlev;
                                    int idx = 0;
#pragma unroll
                                    for (int c = 0; c < 8; ++c) {
                                        if (c < a.fsq.nlev) {
                                            const float zz = orow[c * 33 + x];
                                            z[c] = zz;
                                            idx += fsq_digit<15>(*a.fsq_thr, c, zz) * a.fsq.basis[c];
                                        }
                                    }
                                    if (a.idx) a.idx[vox] = idx;
                                }
                            } else if (c_ok) {
                                const int oh = ho * rh + bb;
                                if (oh < oH) {
                                    const long long rowoff = (((long long)tc.n * oT + ot) * oH + oh) * oW;
#pragma unroll
                                    for (int i = 0; i < 4; ++i) {
                                        const int x = xg + 8 * i, wo = wo0 + x, ow = wo * rw + cc;
                                        if (x >= bwo || wo >= Wout || ow >= oW) continue;
                                        float o = s2[i] + bias_c;
                                        const long long off = (rowoff + ow) * oC + ch;
                                        if (resid) o += __bfloat162float(resid[off]);
                                        if (f32)
                                            static_cast<float*>(out)[off] = gop_blend_out(a, off, o);
                                        else
                                            static_cast<__nv_bfloat16*>(out)[off] = __float2bfloat16_rn(o);
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            s2[i] = s1[i];
                            s1[i] = s0[i];
                            s0[i] = 0.f;
                        }
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[acc]);
                    continue;
                }
                if constexpr (DWM) {
                    // An M = 64 accumulator keeps rows 16q .. 16q + 15 in lanes 0 .. 15 of
                    // TMEM quarter q, so quarter dw (< 3) holds the rows of tap dw. One output
                    // row (32 box columns) at a time is staged in shared memory; then each of
                    // the 128 epilogue threads adds the dw rows for one channel co = t & 15 at
                    // columns x = t / 16 + 8 i (FSQ: one voxel per four threads).
                    float* buf = epi;  // [48 rows][33]
                    const int t = q * 32 + lane;
                    const int co = t & 15, xg = t >> 4;
                    const int Hout = a.Hout, Wout = a.Wout, oT = a.oT, oH = a.oH, oW = a.oW, oC = a.oC;
                    const int bwo = g.bwo, wo0 = tc.tw * bwo;
                    const bool fsq = a.mode == OUT_FSQ, f32 = a.out_fp32 != 0;
                    // this thread's channel: depth-to-space sub-position and stored channel
                    int ch = co, cc = 0, bb = 0, rw = 1, rh = 1, ot = tc.to;
                    if (a.mode == OUT_D2S) {
                        const int sub = co / oC;
                        ch = co - sub * oC;
                        rw = a.rw;
                        rh = a.rh;
                        cc = sub % rw;
                        bb = (sub / rw) % rh;
                        ot = tc.to * a.rt + sub / (rw * rh) - a.drop_t;
                    }
                    const bool c_ok = co < a.Cout && ot >= 0 && ot < oT;
                    const float bias_c = (a.bias && co < a.Cout) ? a.bias[co] : 0.f;
                    const __nv_bfloat16* const resid = static_cast<const __nv_bfloat16*>(a.residual);
                    void* const out = a.out;
                    for (int y = 0; y < g.BH; ++y) {
                        if (q < 3) {
                            float v[16];
#pragma unroll
                            for (int h2 = 0; h2 < 2; ++h2) {
                                tmem_ld16(tbase + (uint32_t)(y * 32 + h2 * 16), v);
                                if (lane < 16) {
#pragma unroll
                                    for (int i2 = 0; i2 < 16; ++i2) buf[(q * 16 + lane) * 33 + h2 * 16 + i2] = v[i2];
                                }
                            }
                        }
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                        const int ho = tc.th * g.BH + y;
                        if (ho < Hout) {
                            if (fsq) {
                                const int x = t >> 2;
                                if ((t & 3) == 0 && x < bwo && wo0 + x < Wout) {
                                    const long long vox =
                                        (((long long)tc.n * a.Tout + tc.to) * Hout + ho) * Wout + wo0 + x;
                                    float* z = static_cast<float*>(out) + vox * a.fsq.nlev;
                                    int idx = 0;
#pragma unroll
                                    for (int c = 0; c < 8; ++c) {
                                        if (c < a.fsq.nlev) {
                                            const float zz = buf[c * 33 + x] + buf[(16 + c) * 33 + x + 1] +
                                                             buf[(32 + c) * 33 + x + 2] + (a.bias ? a.bias[c] : 0.f);
                                            z[c] = zz;
                                            idx += fsq_digit<15>(*a.fsq_thr, c, zz) * a.fsq.basis[c];
                                        }
                                    }
                                    if (a.idx) a.idx[vox] = idx;
                                }
                            } else if (c_ok) {
                                const int oh = ho * rh + bb;
                                if (oh < oH) {
                                    const long long rowoff = (((long long)tc.n * oT + ot) * oH + oh) * oW;
                                    for (int x = xg; x < bwo; x += 8) {
                                        const int wo = wo0 + x, ow = wo * rw + cc;
                                        if (wo >= Wout || ow >= oW) break;
                                        float o = buf[co * 33 + x] + buf[(16 + co) * 33 + x + 1] +
                                                  buf[(32 + co) * 33 + x + 2] + bias_c;
                                        const long long off = (rowoff + ow) * oC + ch;
                                        if (resid) o += __bfloat162float(resid[off]);
                                        if (f32)
                                            static_cast<float*>(out)[off] = gop_blend_out(a, off, o);
                                        else
                                            static_cast<__nv_bfloat16*>(out)[off] = __float2bfloat16_rn(o);
                                    }
                                }
                            }
                        }
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[acc]);
                    continue;
                }
                if (a.Cout <= 32) {
                    // narrow layer (pixel head, latent head): only TMEM lanes 0..Cout-1 hold
                    // channels, all in the warp of quarter 0; the others have nothing to store
                    if (q == 0) {
                        // layer and tile constants in registers, the lane's channel decomposed once
                        const int Hout = a.Hout, Wout = a.Wout, BW = g.BW, BH = g.BH, mode = a.mode;
                        const int oT = a.oT, oH = a.oH, oW = a.oW, oC = a.oC;
                        const bool f32 = a.out_fp32 != 0, lane_ok = co < a.Cout;
                        void* const out = a.out;
                        const __nv_bfloat16* const resid = static_cast<const __nv_bfloat16*>(a.residual);
                        int cc = 0, bb = 0, ot = tc.to, ch = co, rw = 1;
                        if (mode == OUT_D2S) {
                            const int sub = co / oC;
                            ch = co - sub * oC;
                            rw = a.rw;
                            cc = sub % a.rw;
                            bb = (sub / a.rw) % a.rh;
                            ot = tc.to * a.rt + sub / (a.rw * a.rh) - a.drop_t;
                        }
                        const int rh = mode == OUT_D2S ? a.rh : 1;
                        const bool t_ok = ot >= 0 && ot < oT;
                        const long long fbase = ((long long)tc.n * oT + ot) * oH;
#pragma unroll 1
                        for (int c16 = 0; c16 < g.nvox / 16; ++c16) {
                            float v[16];
                            tmem_ld16(tbase + (uint32_t)(c16 * 16), v);
                            const int vv0 = c16 * 16;
                            if (mode == OUT_FSQ) {
                                // gather each voxel's nlev channels through the staging buffer
#pragma unroll
                                for (int i2 = 0; i2 < 16; ++i2) stg[i2 * C::EPI_STRIDE + lane] = v[i2] + bias;
                                __syncwarp();
                                if (lane < 16) {
                                    const int vv = vv0 + lane;
                                    const int ho = tc.th * BH + vv / BW, wo = tc.tw * BW + vv % BW;
                                    if (ho < Hout && wo < Wout) {
                                        const long long vox =
                                            (((long long)tc.n * a.Tout + tc.to) * Hout + ho) * Wout + wo;
                                        float* z = static_cast<float*>(out) + vox * a.fsq.nlev;
                                        int idx = 0;
#pragma unroll
                                        for (int c = 0; c < 8; ++c) {
                                            if (c < a.fsq.nlev) {
                                                const float x = stg[lane * C::EPI_STRIDE + c];
                                                z[c] = x;
                                                idx += fsq_digit<15>(*a.fsq_thr, c, x) * a.fsq.basis[c];
                                            }
                                        }
                                        if (a.idx) a.idx[vox] = idx;
                                    }
                                }
                                __syncwarp();
                                continue;
                            }
                            if (!lane_ok || !t_ok) continue;
                            if ((BW & 15) == 0) {
                                // the 16 voxels lie in one tile row: one row base, stride rw * oC
                                const int ho = tc.th * BH + vv0 / BW, wo0 = tc.tw * BW + vv0 % BW;
                                const int oh = ho * rh + bb;
                                if (ho >= Hout || oh >= oH) continue;
                                const long long rowoff = (fbase + oh) * oW;
                                const int nv = min(16, Wout - wo0);
#pragma unroll
                                for (int i2 = 0; i2 < 16; ++i2) {
                                    const int ow = (wo0 + i2) * rw + cc;
                                    if (i2 >= nv || ow >= oW) continue;
                                    const long long off = (rowoff + ow) * oC + ch;
                                    float x = v[i2] + bias;
                                    if (resid) x += __bfloat162float(resid[off]);
                                    if (f32)
                                        static_cast<float*>(out)[off] = gop_blend_out(a, off, x);
                                    else
                                        static_cast<__nv_bfloat16*>(out)[off] = __float2bfloat16_rn(x);
                                }
                                continue;
                            }
#pragma unroll
                            for (int i2 = 0; i2 < 16; ++i2) {
                                const int vv = vv0 + i2;
                                const int ho = tc.th * BH + vv / BW, wo = tc.tw * BW + vv % BW;
                                const int oh = ho * rh + bb, ow = wo * rw + cc;
                                if (ho >= Hout || wo >= Wout || oh >= oH || ow >= oW) continue;
                                const long long off = ((fbase + oh) * oW + ow) * oC + ch;
                                float x = v[i2] + bias;
                                if (resid) x += __bfloat162float(resid[off]);
                                if (f32)
                                    static_cast<float*>(out)[off] = gop_blend_out(a, off, x);
                                else
                                    static_cast<__nv_bfloat16*>(out)[off] = __float2bfloat16_rn(x);
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[acc]);
                    continue;
                }
                // GroupNorm statistics of the stored values: this thread's 16 channels as four
                // quads of 4 (shifted sums, the shift being the quad's first stored value)
                const bool gstat = a.gn_part != nullptr;
                float gK[4] = {0.f, 0.f, 0.f, 0.f}, gs[4] = {0.f, 0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
                float gcnt = 0.f;
                // per tile: this lane's 16 channels (c0 ..) and, for a depth-to-space output,
                // their sub-position (t, b, c) of the output block (oC % 16 == 0); BW is a
                // power of two, so voxel vv of the tile is (vv >> bwl, vv & (BW - 1))
                const int c0 = tc.nt * BN + q * 32 + half * 16;
                const int bwl = __ffs(g.BW) - 1;
                const int Hout = a.Hout, Wout = a.Wout, oT = a.oT, oH = a.oH, oW = a.oW, oC = a.oC;
                int ot = tc.to, ch0 = c0, rh = 1, rw = 1, bb = 0, cc = 0;
                if (a.mode == OUT_D2S) {
                    const int sub = c0 / oC;
                    ch0 = c0 - sub * oC;
                    rw = a.rw;
                    rh = a.rh;
                    cc = sub % rw;
                    bb = (sub / rw) % rh;
                    ot = tc.to * a.rt + sub / (rw * rh) - a.drop_t;
                }
                const bool lane_ok = c0 < a.Cout && ot >= 0 && ot < oT;
                const long long fbase = ((long long)tc.n * oT + ot) * oH;  // first output row of the frame
                const int ho0 = tc.th * g.BH, wo0 = tc.tw * g.BW;
#pragma unroll 1
                for (int c16 = 0; c16 < g.nvox / 16; ++c16) {
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)(c16 * 16), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) stg[i * C::EPI_STRIDE + lane] = v[i] + bias;
                    __syncwarp();
                    const int vv = c16 * 16 + j;
                    const int ho = ho0 + (vv >> bwl), wo = wo0 + (vv & (g.BW - 1));
                    if (ho < Hout && wo < Wout && c0 < a.Cout) {
                        float o[16];
                        const float4* src = reinterpret_cast<const float4*>(stg + j * C::EPI_STRIDE + half * 16);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 f = src[i];
                            o[4 * i] = f.x;
                            o[4 * i + 1] = f.y;
                            o[4 * i + 2] = f.z;
                            o[4 * i + 3] = f.w;
                        }
                        // plain: voxel (to, ho, wo); depth-to-space: sub-position (ot, bb, cc)
                        const int oh = ho * rh + bb, ow = wo * rw + cc;
                        if (lane_ok && oh < oH && ow < oW) {
                            const long long off = ((fbase + oh) * oW + ow) * oC + ch0;
                            if (a.residual) add_bf16x16(static_cast<const __nv_bfloat16*>(a.residual) + off, o);
                            uint32_t w8[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) w8[i] = pack_bf16x2(o[2 * i], o[2 * i + 1]);
                            uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.out) + off);
                            dst[0] = make_uint4(w8[0], w8[1], w8[2], w8[3]);
                            dst[1] = make_uint4(w8[4], w8[5], w8[6], w8[7]);
                            if (gstat) {
                                float r[16];
#pragma unroll
                                for (int i = 0; i < 8; ++i) {
                                    const float2 f = unpack_bf16x2(w8[i]);
                                    r[2 * i] = f.x;
                                    r[2 * i + 1] = f.y;
                                }
                                if (gcnt == 0.f) {
#pragma unroll
                                    for (int k = 0; k < 4; ++k) gK[k] = r[4 * k];
                                }
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    const float d = r[i] - gK[i / 4];
                                    gs[i / 4] += d;
                                    gq[i / 4] = fmaf(d, d, gq[i / 4]);
                                }
                                gcnt += 4.f;
                            }
                        }
                    }
                    __syncwarp();
                }
                if (gstat) {
                    // quads -> triples, merged over the 16 lanes holding the same channels
                    // (lane i takes lane i + o: a fixed order), then into groups of gn_cg channels
                    GnTriple t[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        t[k].n = gcnt;
                        t[k].mean = gcnt > 0.f ? gK[k] + gs[k] / gcnt : 0.f;
                        t[k].m2 = gcnt > 0.f ? fmaxf(gq[k] - gs[k] * gs[k] / gcnt, 0.f) : 0.f;
                    }
#pragma unroll
                    for (int o = 16; o >= 2; o >>= 1)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const GnTriple b = gn_shfl_down(t[k], o);
                            if (lane + o < 32) t[k] = gn_merge(t[k], b);
                        }
                    const int cg = a.gn_cg;
                    if (cg >= 8) {
                        t[0] = gn_merge(t[0], t[1]);
                        t[1] = gn_merge(t[2], t[3]);
                    }
                    if (cg == 16) t[0] = gn_merge(t[0], t[1]);
                    const int gc0 = tc.nt * BN + q * 32 + lane * 16;  // lanes 0, 1: the two halves
                    if (lane < 2 && gc0 < a.Cout) {
                        int gch = gc0, fr = tc.to, slot = tc.th * g.tiles_w + tc.tw, S = g.tiles_h * g.tiles_w;
                        if (a.mode == OUT_D2S) {
                            const int sub = gc0 / a.oC;
                            gch = gc0 - sub * a.oC;
                            fr = tc.to * a.rt + sub / (a.rw * a.rh) - a.drop_t;
                            slot = (slot * a.rh + (sub / a.rw) % a.rh) * a.rw + sub % a.rw;
                            S *= a.rh * a.rw;
                        }
                        if (fr >= 0 && fr < a.oT) {
                            const int G = a.oC / cg;
                            GnTriple* dst = a.gn_part + (((long long)tc.n * a.oT + fr) * S + slot) * G + gch / cg;
                            const int ng = 16 / cg;
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k < ng) dst[k] = t[k];
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[acc]);
                continue;
            }
            const int ho = tc.th * g.BH + r / g.BW;
            const int wo = tc.tw * g.BW + r % g.BW;
            const bool valid = ho < a.Hout && wo < a.Wout;
            const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * C::ACC_COLS);
            const long long vox = (((long long)tc.n * a.Tout + tc.to) * a.Hout + ho) * a.Wout + wo;
            // one voxel per thread. Plain bf16 output of whole 64-channel groups: four TMEM
            // loads and the group's bias in flight at once, then the warp's staging rows
            // (64 channels = 128 B of each of its 32 voxels) written as whole 128-byte
            // lines (a direct store would touch 32 lines per instruction, one per voxel).
            // The other channels (a ragged last group, fp32 or depth-to-space or FSQ
            // output) 16 per step, the TMEM load of the next step in flight.
            const bool bias4 = a.bias && (reinterpret_cast<uintptr_t>(a.bias) & 15) == 0;
            const int ngrp = (BN >= 64 && a.mode == OUT_PLAIN && !a.out_fp32 && (a.oC & 7) == 0)
                                 ? max(0, min(BN, a.Cout - tc.nt * BN)) / 64
                                 : 0;  // whole 64-channel groups taken staged
            const long long fbase = ((long long)tc.n * a.oT + tc.to) * a.oH;
            {
                uint8_t* const srow = reinterpret_cast<uint8_t*>(epi) + q * 4096;  // 16-byte slots XOR row & 7
                const int bwl = __ffs(g.BW) - 1, sw = lane & 7;
                const __nv_bfloat16* const resid = static_cast<const __nv_bfloat16*>(a.residual);
                __nv_bfloat16* const outp = static_cast<__nv_bfloat16*>(a.out);
#pragma unroll 1
                for (int g4 = 0; g4 < ngrp; ++g4) {
                    const int g0 = tc.nt * BN + g4 * 64;
                    uint32_t rr[4][16];
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmem_ld16_issue(tbase + (uint32_t)(g4 * 64 + k * 16), rr[k]);
                    float bv[64];
                    if (bias4) {
                        const float4* b4 = reinterpret_cast<const float4*>(a.bias + g0);
#pragma unroll
                        for (int m = 0; m < 16; ++m) {
                            const float4 b = __ldg(b4 + m);
                            bv[4 * m] = b.x;
                            bv[4 * m + 1] = b.y;
                            bv[4 * m + 2] = b.z;
                            bv[4 * m + 3] = b.w;
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < 64; ++m) bv[m] = a.bias ? a.bias[g0 + m] : 0.f;
                    }
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmem_regs_fence(rr[k]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float v[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(rr[k][j]) + bv[16 * k + j];
                        if (resid && valid) add_bf16x16(resid + ((fbase + ho) * a.oW + wo) * a.oC + g0 + 16 * k, v);
                        uint4 o0, o1;
                        o0.x = pack_bf16x2(v[0], v[1]);
                        o0.y = pack_bf16x2(v[2], v[3]);
                        o0.z = pack_bf16x2(v[4], v[5]);
                        o0.w = pack_bf16x2(v[6], v[7]);
                        o1.x = pack_bf16x2(v[8], v[9]);
                        o1.y = pack_bf16x2(v[10], v[11]);
                        o1.z = pack_bf16x2(v[12], v[13]);
                        o1.w = pack_bf16x2(v[14], v[15]);
                        *reinterpret_cast<uint4*>(srow + lane * 128 + (((2 * k) ^ sw) << 4)) = o0;
                        *reinterpret_cast<uint4*>(srow + lane * 128 + (((2 * k + 1) ^ sw) << 4)) = o1;
                    }
                    __syncwarp();
                    // 8 lanes per voxel row, 4 rows per store
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int vl = i * 4 + (lane >> 3);
                        const uint4 d = *reinterpret_cast<const uint4*>(srow + vl * 128 + ((sw ^ (vl & 7)) << 4));
                        const int r2 = q * 32 + vl;
                        const int ho2 = tc.th * g.BH + (r2 >> bwl), wo2 = tc.tw * g.BW + (r2 & (g.BW - 1));
                        if (ho2 < a.Hout && wo2 < a.Wout)
                            *reinterpret_cast<uint4*>(outp + ((fbase + ho2) * a.oW + wo2) * a.oC + g0 + sw * 8) = d;
                    }
                    __syncwarp();
                }
            }
            const auto emit = [&](const uint32_t(&r)[16], int c16) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
                const int co0 = tc.nt * BN + c16 * 16;
                if (!valid || co0 >= a.Cout) return;
                if (bias4 && co0 + 16 <= a.Cout) {
                    const float4* b4 = reinterpret_cast<const float4*>(a.bias + co0);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float4 b = __ldg(b4 + k);
                        v[4 * k] += b.x;
                        v[4 * k + 1] += b.y;
                        v[4 * k + 2] += b.z;
                        v[4 * k + 3] += b.w;
                    }
                } else if (a.bias) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += (co0 + j < a.Cout) ? a.bias[co0 + j] : 0.f;
                }
                if (a.mode == OUT_PLAIN) {
                    const long long off = ((((long long)tc.n * a.oT + tc.to) * a.oH + ho) * a.oW + wo) * a.oC + co0;
                    if (co0 + 16 <= a.Cout && (a.oC & 7) == 0 && !a.out_fp32) {
                        if (a.residual) add_bf16x16(static_cast<const __nv_bfloat16*>(a.residual) + off, v);
                        store_bf16x16(static_cast<__nv_bfloat16*>(a.out) + off, v);
                    } else {
                        // a partial group of 16 channels (narrow or ragged layers), or fp32 output
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (co0 + j >= a.Cout) break;
                            float x = v[j];
                            if (a.residual) x += __bfloat162float(static_cast<const __nv_bfloat16*>(a.residual)[off + j]);
                            if (a.out_fp32)
                                static_cast<float*>(a.out)[off + j] = x;
                            else
                                static_cast<__nv_bfloat16*>(a.out)[off + j] = __float2bfloat16_rn(x);
                        }
                    }
                } else if (a.mode == OUT_D2S) {
                    if ((a.oC & 15) == 0) {
                        const int sub = co0 / a.oC, ch0 = co0 - sub * a.oC;
                        const int c = sub % a.rw, b = (sub / a.rw) % a.rh, t = sub / (a.rw * a.rh);
                        const int ot = tc.to * a.rt + t - a.drop_t, oh = ho * a.rh + b, ow = wo * a.rw + c;
                        if (ot >= 0 && ot < a.oT && oh < a.oH && ow < a.oW) {
                            const long long off =
                                ((((long long)tc.n * a.oT + ot) * a.oH + oh) * a.oW + ow) * a.oC + ch0;
                            if (a.out_fp32) {
                                float* o = static_cast<float*>(a.out) + off;
#pragma unroll
                                for (int j = 0; j < 16; ++j) o[j] = gop_blend_out(a, off + j, v[j]);
                            } else {
                                store_bf16x16(static_cast<__nv_bfloat16*>(a.out) + off, v);
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int co = co0 + j;
                            if (co >= a.Cout) break;
                            const int sub = co / a.oC, ch = co - sub * a.oC;
                            const int c = sub % a.rw, b = (sub / a.rw) % a.rh, t = sub / (a.rw * a.rh);
                            const int ot = tc.to * a.rt + t - a.drop_t, oh = ho * a.rh + b, ow = wo * a.rw + c;
                            if (ot < 0 || ot >= a.oT || oh >= a.oH || ow >= a.oW) continue;
                            const long long off =
                                ((((long long)tc.n * a.oT + ot) * a.oH + oh) * a.oW + ow) * a.oC + ch;
                            if (a.out_fp32)
                                static_cast<float*>(a.out)[off] = gop_blend_out(a, off, v[j]);
                            else
                                static_cast<__nv_bfloat16*>(a.out)[off] = __float2bfloat16_rn(v[j]);
                        }
                    }
                } else {  // OUT_FSQ: the latent z (fp32) and its token index
                    float* z = static_cast<float*>(a.out) + vox * a.fsq.nlev;
                    int idx = 0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (j < a.fsq.nlev) {
                            z[j] = v[j];
                            idx += fsq_digit<15>(*a.fsq_thr, j, v[j]) * a.fsq.basis[j];
                        }
                    }
                    if (a.idx) a.idx[vox] = idx;
                }
            };
            uint32_t r0[16], r1[16];
            if (ngrp * 4 < BN / 16) tmem_ld16_issue(tbase + (uint32_t)(ngrp * 64), r0);
#pragma unroll 1
            for (int c16 = ngrp * 4; c16 < BN / 16; c16 += 2) {
                tmem_ld_wait();
                tmem_regs_fence(r0);
                if (c16 + 1 < BN / 16) tmem_ld16_issue(tbase + (uint32_t)((c16 + 1) * 16), r1);
                emit(r0, c16);
                if (c16 + 1 < BN / 16) {
                    tmem_ld_wait();
                    tmem_regs_fence(r1);
                    if (c16 + 2 < BN / 16) tmem_ld16_issue(tbase + (uint32_t)((c16 + 2) * 16), r0);
                    emit(r1, c16 + 1);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, C::TMEM_COLS);
}

template <int BN, bool SWAP, int MAXP, int HALO = 0, int TR = 0, int KC = 64, bool SPLIT = false>
int launch_bn(const ConvArgs* as, const TcGeo* gs, int count, int num_sms, int cta_tiles, cudaStream_t stream) {
    using C = Cfg<BN, SWAP, HALO, TR, KC, SPLIT>;
    auto kern = conv_tc_kernel<BN, SWAP, MAXP, HALO, TR, KC, SPLIT>;
    TcBatch<MAXP> B;
    memset(&B, 0, sizeof(B));
    // a narrow halo layer loads its real weight rows only
    // (taps in rows: 48 weight rows dw * 16 + co over K = (dt, dh, ci), or 128 rows
    // (dh * 3 + dw) * Cout + co over K = (dt, ci))
    B.w_rows = TR == 3   ? 48
               : TR == 9 ? 128
               : (HALO > 0 && SWAP && as[0].Cout <= 32) ? (as[0].Cout + 15) / 16 * 16
                                                        : BN;
    const int wk = TR == 3 ? 9 * as[0].Cin : TR == 9 ? 3 * as[0].Cin : as[0].Kpad;
    if (!encode_w_map(&B.tm_w, as[0].w, as[0].Cout_pad, wk, B.w_rows, KC)) return -1;
    if (as[0].w0) {
        if (!encode_w_map(&B.tm_w0, as[0].w0, as[0].Cout_pad, wk, B.w_rows, KC)) return -1;
    } else {
        B.tm_w0 = B.tm_w;
    }
    long long total = 0;
    for (int p = 0; p < count; ++p) {
        const ConvArgs& a = as[p];
        TcGeo g = gs[p];
        const bool strided = g.strided != 0;
        // the halo box: one input row above and below (nine taps in rows: BH rows in all)
        const int box_h = HALO ? (TR == 9 ? g.BH : g.BH + 2) : g.BH;
        if (!encode_act_map(&B.tm_x[p], a.x, a.N * a.Tin, a.Hin, a.Win, a.Cin, box_h, g.BW, strided, KC)) return -1;
        if (a.hist) {
            if (!encode_act_map(&B.tm_h[p], a.hist, a.N * a.hist_T, a.Hin, a.Win, a.Cin, box_h, g.BW, strided, KC))
                return -1;
        } else {
            B.tm_h[p] = B.tm_x[p];
        }
        // weight tiles that hold output channels (narrow layers have padded weight rows)
        g.n_tiles = std::min(a.Cout_pad, (a.Cout + BN - 1) / BN * BN) / BN;
        g.m_tiles = (long long)a.N * a.Tout * g.tiles_h * g.tiles_w;
        g.num_tiles = g.m_tiles * g.n_tiles;
        total += g.num_tiles;
        B.a[p] = a;
        B.g[p] = g;
        B.unit_end[p] = total;
    }
    B.count = count;
    B.num_units = total;
    if (total == 0) return 0;
    if constexpr (SPLIT) {
        // activation slots: the launch's largest box, 1 KB aligned (swizzle atoms)
        int box = 0;
        for (int p = 0; p < count; ++p) box = std::max(box, (B.g[p].BH + 2) * B.g[p].BW * C::ROWB);
        B.act_slot = (box + 1023) / 1024 * 1024;
        B.na = std::min(4, C::SPLIT_ACT_BYTES / B.act_slot);
        if (B.na < 2 || B.w_rows != BN) return -1;
    }
    static std::atomic<unsigned long long> attr_done{0};
    if (smem_attr_once(kern, C::SMEM, attr_done) != cudaSuccess) return -1;
    // persistent (one CTA per SM), or CTAs of at most cta_tiles tiles each
    long long grid = std::min<long long>(total, num_sms);
    if (cta_tiles > 0) grid = std::max(grid, std::min<long long>((total + cta_tiles - 1) / cta_tiles, 1LL << 30));
    kern<<<(unsigned)grid, 192, C::SMEM, stream>>>(B);
    return (int)cudaGetLastError();
}

template <int BN, bool SWAP, int NCB, int TR = 0, int KC = 64, bool SPLIT = false>  // NCB: KC-channel blocks per halo stage
int launch_bn_halo(const ConvArgs* as, const TcGeo* gs, int count, int num_sms, int cta_tiles, cudaStream_t stream) {
    return count == 1 ? launch_bn<BN, SWAP, 1, NCB, TR, KC, SPLIT>(as, gs, 1, num_sms, cta_tiles, stream)
                      : launch_bn<BN, SWAP, kMaxConvGroup, NCB, TR, KC, SPLIT>(as, gs, count, num_sms, cta_tiles, stream);
}

template <int BN, bool SWAP>
int launch_bn_any(const ConvArgs* as, const TcGeo* gs, int count, int num_sms, int cta_tiles, cudaStream_t stream) {
    return count == 1 ? launch_bn<BN, SWAP, 1>(as, gs, 1, num_sms, cta_tiles, stream)
                      : launch_bn<BN, SWAP, kMaxConvGroup>(as, gs, count, num_sms, cta_tiles, stream);
}

}  // namespace

// ------------------------------------------------------------------ host side
// (tensor-map encoders are shared with the tensor-core wgrad kernel)

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Activation map: plain (C, W, H, N*T) or parity view (2C, W/2, 2, H/2, N*T); boxes of
// kc channels (64: 128-byte swizzle, 32: 64-byte swizzle).
bool encode_act_map(CUtensorMap* m, const void* base, int frames, int H, int W, int C, int BH, int BW,
                    bool strided, int kc) {
    auto enc = get_encode_fn();
    if (!enc) return false;
    const uint64_t es = 2;
    const CUtensorMapSwizzle sw = kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    CUresult r;
    if (!strided) {
        cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)frames};
        cuuint64_t strides[3] = {C * es, (uint64_t)W * C * es, (uint64_t)H * W * C * es};
        cuuint32_t box[4] = {(cuuint32_t)kc, (cuuint32_t)BW, (cuuint32_t)BH, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[5] = {(cuuint64_t)(2 * C), (cuuint64_t)(W / 2), 2, (cuuint64_t)(H / 2),
                              (cuuint64_t)frames};
        cuuint64_t strides[4] = {2 * C * es, (uint64_t)W * C * es, 2ull * W * C * es, (uint64_t)H * W * C * es};
        cuuint32_t box[5] = {(cuuint32_t)kc, (cuuint32_t)BW, 1, (cuuint32_t)BH, 1};
        cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

bool encode_w_map(CUtensorMap* m, const void* base, int rows, int Kpad, int BN, int kc) {
    auto enc = get_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)kc, (cuuint32_t)BN};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Choose the output tile shape (BH x BW = 128) that covers Hout x Wout with
// the fewest tiles; ties go to the wider tile (longer contiguous rows).
void choose_tile(int Hout, int Wout, int rows, int* BH, int* BW) {
    long long best = -1;
    for (int bw : {256, 128, 64, 32, 16, 8}) {
        if (bw > rows || rows / bw > 256) continue;
        int bh = rows / bw;
        long long t = (long long)((Wout + bw - 1) / bw) * ((Hout + bh - 1) / bh);
        if (best < 0 || t < best) {
            best = t;
            *BW = bw;
            *BH = bh;
        }
    }
}

// Halo tiles: BW in {16, 32, 64} (the dh offset is a whole number of swizzle
// atoms and the box fits the stage); fewest tiles, then fewest halo rows.
void choose_tile_halo(int Hout, int Wout, int rows, int* BH, int* BW) {
    long long best = -1, best_rows = 0;
    for (int bw : {16, 32, 64}) {
        const int bh = rows / bw;
        const long long t = (long long)((Wout + bw - 1) / bw) * ((Hout + bh - 1) / bh);
        const long long hr = t * (bh + 2) * bw;
        if (best < 0 || t < best || (t == best && hr < best_rows)) {
            best = t;
            best_rows = hr;
            *BW = bw;
            *BH = bh;
        }
    }
}

int conv_tc_bn(int Cout_pad) {
    if (Cout_pad >= 256) return 256;
    if (Cout_pad >= 128) return 128;
    if (Cout_pad >= 64) return 64;
    if (Cout_pad >= 32) return 32;
    return 16;
}

// Padded output channels of a BF16 conv's packed weights: layers of at most
// 32 channels are padded to 128 and run in the swapped (weights as A) form.
int conv_tc_cout_pad(int Cout) {
    const int c16 = (Cout + 15) / 16 * 16;
    if (c16 <= 32) return 128;
    const int bn = conv_tc_bn(c16);
    return (c16 + bn - 1) / bn * bn;
}

// The kernel form a layer runs in. Stride-1 3x3x3 layers share each input box
// among the three dh taps (halo form); a narrow halo layer (at most 32
// channels) runs unswapped with 16 or 32 weight rows. Wide layers of 128k
// channels with bf16 output (plain, or depth-to-space whose 16-channel groups
// stay within one sub-position) and other 128-channel plain layers run
// swapped; narrow layers without halo run swapped with padded weights.
ConvRoute conv_route(const ConvArgs& a0) {
    ConvRoute r;
    r.taps3 = a0.kh == 3 && a0.kw == 3 && a0.sh == 1 && a0.sw == 1;
    r.narrow = a0.Cout <= 32;
    const bool wide = a0.Cout % 128 == 0 && a0.Cout_pad % 128 == 0 && !a0.out_fp32 &&
                      (a0.mode == OUT_PLAIN || (a0.mode == OUT_D2S && a0.oC % 16 == 0));
    r.swap = (a0.Cout_pad == 128 && ((a0.mode == OUT_PLAIN && !a0.out_fp32 && a0.Cout == 128) || r.narrow)) ||
             (r.taps3 && wide);
    r.halo = r.taps3 && r.swap;
    return r;
}

// Nine taps in rows cut the MMAs per output 2.25-fold against three, but its
// epilogue (nine shifted adds per output through shared memory) costs a fixed
// ~75 SM cycles per output: it wins when the K loop is long. Measured on the
// 720p clip: latent head (512 input channels) 0.098 -> 0.069 ms, pixel head
// (128 input channels) 0.86 -> 1.30 ms; hence 256 input channels or more.
int conv_tc_taprows(int Cout, int Cin, int k, int sh, int sw) {
    if (k != 3 || sh != 1 || sw != 1 || Cout < 1) return 0;
    if (9 * Cout <= 128 && Cin >= 256) return 9;
    return Cout <= 16 ? 3 : 0;
}

// GroupNorm statistics come from the swapped wide epilogue (plain or
// depth-to-space, bf16), for groups of 4, 8 or 16 channels, of 3x3x3 layers:
// a layer with a short K loop (1x1x1, the stem over its im2col matrix) is
// bound by its epilogue, where the extra work costs more than the statistics
// pass it would save (720p stem: conv 0.63 -> 0.98 ms against 0.23 ms saved).
bool conv_tc_gn_fusable(const ConvArgs& a) {
    const ConvRoute r = conv_route(a);
    return r.swap && !r.narrow && a.kh == 3 && (a.mode == OUT_PLAIN || a.mode == OUT_D2S) && !a.out_fp32 &&
           (a.gn_cg == 4 || a.gn_cg == 8 || a.gn_cg == 16);
}

// Statistics slots per output frame: the spatial tiles of the launch (times
// the rh x rw sub-positions of a depth-to-space output).
// Wide swapped halo layers may also take a tile of 192..240 voxels that fits
// the frame better (e.g. 15 x 16 for a 90 x 160 frame, where 8 x 32 computes
// 96 rows): per frame, tiles x (N + 48) (the 48 stands for a tile's fixed cost)
// must drop by 3% or more against the best 256-voxel tile. The choice depends
// on the frame size only, so a stream chunk and a whole clip tile alike.
void choose_tile_halo_fit(int Hout, int Wout, int* BH, int* BW) {
    choose_tile_halo(Hout, Wout, 256, BH, BW);
    const auto cost = [&](int bh, int bw) {
        return (long long)((Hout + bh - 1) / bh) * ((Wout + bw - 1) / bw) * (bh * bw + 48);
    };
    const long long base = cost(*BH, *BW);
    long long best = base;
    int bbh = *BH, bbw = *BW;
    for (int bw : {16, 32, 64})
        for (int bh = (192 + bw - 1) / bw; bh * bw < 256; ++bh) {
            if ((bh * bw) % 16) continue;
            const long long c = cost(bh, bw);
            if (c < best) {
                best = c;
                bbh = bh;
                bbw = bw;
            }
        }
    if (best * 100 <= base * 97) {
        *BH = bbh;
        *BW = bbw;
    }
}

static int device_sms() {
    static const int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                         cudaSuccess || v < 1)
            v = 148;
        return v;
    }();
    return n;
}

// Wave-aware refinement of the wide halo tile. The persistent grid deals the
// units (tile, 128-channel block) to one CTA per SM in turn, so the busiest
// CTA runs ceil(units / SMs) of them, each costing about (voxels + 48). A
// layer with few units (the 512-channel level of a 720p clip: 1200 units of
// 15 x 16 is 8.1 waves, paid as 9) can gain by another tile size: 7 x 32 gives
// 1300 units, still 9 waves, of 224 instead of 240 voxels. Tiles of 128 to
// 256 voxels, width 16, 32 or 64; taken only when at least 3% cheaper. Only
// for layers that do not reduce GroupNorm statistics: those are summed per
// tile, and a tile that depends on the frame count would make a stream of
// chunks round them differently from the whole clip (the conv outputs
// themselves do not depend on the tile), unless the caller allows it.
static void choose_tile_halo_waves(const ConvArgs& a, int* BH, int* BW) {
    choose_tile_halo_fit(a.Hout, a.Wout, BH, BW);
    const long long blocks = (long long)a.N * a.Tout * (a.Cout_pad / 128);
    const long long sms = device_sms();
    const auto cost = [&](int bh, int bw) {
        const long long units = (long long)((a.Hout + bh - 1) / bh) * ((a.Wout + bw - 1) / bw) * blocks;
        return (units + sms - 1) / sms * (bh * bw + 48);
    };
    const long long base = cost(*BH, *BW);
    long long best = base;
    int bbh = *BH, bbw = *BW;
    for (int bw : {16, 32, 64})
        for (int bh = 128 / bw; bh * bw <= 256; ++bh) {
            if ((bh * bw) % 16) continue;
            const long long c = cost(bh, bw);
            if (c < best || (c == best && bh * bw > bbh * bbw)) {
                best = c;
                bbh = bh;
                bbw = bw;
            }
        }
    if (best * 100 <= base * 97) {
        *BH = bbh;
        *BW = bbw;
    }
}

// The output tile of a layer in its route (shared by the launch and the
// GroupNorm statistics slot count).
void conv_tc_tile(const ConvArgs& a, const ConvRoute& r, int* BH, int* BW) {
    if (r.halo && !r.narrow && a.gn_cg && !a.gn_any_tile)
        choose_tile_halo_fit(a.Hout, a.Wout, BH, BW);
    else if (r.halo && !r.narrow)
        choose_tile_halo_waves(a, BH, BW);
    else if (r.halo)
        choose_tile_halo(a.Hout, a.Wout, 256, BH, BW);
    else
        choose_tile(a.Hout, a.Wout, r.swap ? 256 : 128, BH, BW);
}

int conv_tc_gn_slots(const ConvArgs& a) {
    const ConvRoute r = conv_route(a);
    int BH = 1, BW = 1;
    conv_tc_tile(a, r, &BH, &BW);
    const int tiles = ((a.Hout + BH - 1) / BH) * ((a.Wout + BW - 1) / BW);
    return a.mode == OUT_D2S ? tiles * a.rh * a.rw : tiles;
}

// Requirements (checked by the caller's plan): Cin % 64 == 0, Cout_pad a
// multiple of the chosen BN, Kpad = taps * Cin, strided convs have
// sh == sw == 2 with even Hin and Win, bf16 tensors 16-byte aligned.
// A group shares the layer: weights, Cin, Cout, kernel, strides and epilogue
// mode; inputs, outputs, sizes and histories are per problem. cta_tiles = 0
// launches one persistent CTA per SM; n > 0 gives every CTA at most n tiles,
// so that a kernel on a higher-priority CUDA stream gets SMs within one short
// CTA lifetime instead of after the whole layer.
int launch_conv_tc_group(const ConvArgs* as, int count, int num_sms, cudaStream_t stream, int cta_tiles) {
    if (count < 1 || count > kMaxConvGroup) return -1;
    const ConvArgs& a0 = as[0];
    for (int p = 1; p < count; ++p)
        if (as[p].w != a0.w || as[p].w0 != a0.w0 || as[p].Cin != a0.Cin || as[p].Cout_pad != a0.Cout_pad || as[p].Kpad != a0.Kpad ||
            as[p].kt != a0.kt || as[p].kh != a0.kh || as[p].kw != a0.kw || as[p].sh != a0.sh || as[p].mode != a0.mode ||
            as[p].out_fp32 != a0.out_fp32)
            return -1;
    // the wide (swapped) form: exactly 128 output channels with plain bf16 output,
    // or a narrow layer (at most 32 channels, weights padded to 128 rows)
    const ConvRoute rt = conv_route(a0);
    const bool swap = rt.swap, halo = rt.halo;
    const int tr = a0.w_dwm;
    const bool dwm = tr != 0;
    // weights packed with taps in the rows only run in that form
    if (dwm && !(halo && a0.kt == 3 && conv_tc_taprows(a0.Cout, a0.Cin, a0.kh, a0.sh, a0.sw) == tr && !a0.w0 &&
                 a0.Cin % 64 == 0))
        return -1;
    for (int p = 0; p < count; ++p)
        if (as[p].gn_part && (!conv_tc_gn_fusable(as[p]) || as[p].gn_cg != a0.gn_cg)) return -1;
    // wide stride-1 3x3x3 layers: K blocks of kHaloKC channels
    const bool wide_halo = halo && !rt.narrow && tr == 0 && a0.Cin % kHaloKC == 0;
    TcGeo gs[kMaxConvGroup];
    for (int p = 0; p < count; ++p) {
        TcGeo& g = gs[p];
        const ConvArgs& a = as[p];
        if (dwm) {
            g.BH = DWM_BH;  // dw rows: output rows; nine taps: box rows (BH - 2 output rows)
            g.BW = DWM_BW;  // box columns; DWM_BW - 2 output columns per tile
        } else {
            conv_tc_tile(a, rt, &g.BH, &g.BW);
        }
        g.bwo = dwm ? g.BW - 2 : g.BW;
        g.bho = tr == 9 ? g.BH - 2 : g.BH;
        if (swap && (g.BW & (g.BW - 1))) return -1;  // the swapped epilogue splits voxels by shifts
        g.nvox = g.BH * g.BW;
        g.tiles_w = (a.Wout + g.bwo - 1) / g.bwo;
        g.tiles_h = (a.Hout + g.bho - 1) / g.bho;
        g.cpt = a.Cin / (wide_halo ? kHaloKC : 64);
        g.nkb = dwm ? a.kt * g.cpt : halo ? a.kt * a.kw * g.cpt : a.kt * a.kh * a.kw * g.cpt;
        g.strided = (a.sh == 2) ? 1 : 0;
        g.halo = halo ? 1 : 0;
        g.n_tiles = 0;
        g.num_tiles = 0;
    }
    if (tr == 9) return launch_bn_halo<128, true, 1, 9>(as, gs, count, num_sms, cta_tiles, stream);
    if (tr == 3) return launch_bn_halo<128, true, 1, 3>(as, gs, count, num_sms, cta_tiles, stream);
    if (halo && wide_halo) {
        if constexpr (kHaloKC != 64)
            return launch_bn_halo<128, true, 1, 0, kHaloKC>(as, gs, count, num_sms, cta_tiles, stream);
        else
            return launch_bn_halo<128, true, 1, 0, 64, kHaloSplit>(as, gs, count, num_sms, cta_tiles, stream);
    }
    if (halo) return launch_bn_halo<128, true, 1>(as, gs, count, num_sms, cta_tiles, stream);
    if (swap) return launch_bn_any<128, true>(as, gs, count, num_sms, cta_tiles, stream);
    switch (conv_tc_bn(a0.Cout_pad)) {
        case 256: return launch_bn_any<256, false>(as, gs, count, num_sms, cta_tiles, stream);
        case 128: return launch_bn_any<128, false>(as, gs, count, num_sms, cta_tiles, stream);
        case 64: return launch_bn_any<64, false>(as, gs, count, num_sms, cta_tiles, stream);
        case 32: return launch_bn_any<32, false>(as, gs, count, num_sms, cta_tiles, stream);
        default: return launch_bn_any<16, false>(as, gs, count, num_sms, cta_tiles, stream);
    }
}

int launch_conv_tc(const ConvArgs& a, int num_sms, cudaStream_t stream) {
    return launch_conv_tc_group(&a, 1, num_sms, stream, 0);
}

}  // namespace tok
