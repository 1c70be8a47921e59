// Weight gradient of a causal conv on the tensor cores (BF16 -> FP32).
//
//   dW[co][tap][ci] = sum_v dY[v][co] * X[v + off(tap)][ci]
//
// GEMM with M = output channels (128 per tile), N = input channels (BN = 128
// or 256 per tile), K = voxels, one tap per CTA, split-K over voxel tiles
// (deterministic: every split writes its own FP32 partial, a fixed-order
// reduction follows). A K step is one tile of 64 output voxels (BH x BW of one
// frame): TMA loads the dY box {64 channels x 64 voxels} and the tap-shifted X
// box with the same voxel order. Such a box lands in shared memory as 64
// rows (voxels = K) of 128 bytes (64 channels = M or N) with 128B swizzle,
// which is the MN-major canonical layout of tcgen05: rows of 64 MN-contiguous
// elements, 8-row groups 1024 B apart along K (stride byte offset), and
// 64-element MN blocks one box apart (leading byte offset). Out-of-frame taps
// read zeros (TMA out-of-bounds fill); taps before frame 0 read frame 0
// (replicate) or nothing (zero padding); voxels past the frame edge of a
// ragged tile read zero dY and so contribute nothing.
//
// Stride-2 convs (h and w) read X through the parity view
// (2C, W/2, 2, H/2, frames) that the forward conv uses: input column
// 2w + dw - 1 is parity (dw + 1) % 2 at half-column w - (dw == 0), so a tap
// is again one box per 64 channels. Output channels past Cout (a narrow
// layer such as the 12-channel pixel head) and input channels past Cin (an
// im2col matrix of 192 columns) are neither loaded nor stored: row m of the
// product depends on row m of A only, column n on column n of B only.
//
// Halo form (stride-1 3x3x3 layers, BN = 128): a CTA accumulates the three dh
// taps of one (dt, dw) in three TMEM accumulators. Per K step it loads the dY
// box and one X box of BH + 2 rows (BW = 8 or 16); tap dh reads the X box from
// voxel row dh * BW on, a whole number of 8-row (1 KB) groups, so its operand
// descriptor starts there and the two 64-channel halves of X lie one halo box
// apart (the leading byte offset). X bytes per MMA drop about 2.4-fold.
//
// The bias gradient stays a separate column-sum pass over dY (~5 TB/s): taking
// it inside this kernel, in the CTAs of one tap slot, lengthened the launch's
// single wave more than the pass costs (extra M = 128, N = 16 MMAs against a
// tile of ones: +15-23%; the epilogue warps summing each dY stage before its
// release: +18-25%).
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "conv_args.h"

namespace tok {

bool encode_act_map(CUtensorMap* m, const void* base, int frames, int H, int W, int C, int BH, int BW, bool strided,
                    int kc);

namespace {

constexpr int KV = 64;  // voxels per K step

struct WtcGeo {
    int BH, BW, tiles_h, tiles_w;
    long long vtiles;   // voxel tiles (K steps) in total
    int m_tiles, n_tiles, taps, S;  // taps: CTA tap slots (dt, dw groups in the halo form)
    int strided;        // X read through the parity view (stride 2 in h and w)
};

constexpr int HALO_ROWS_MAX = (KV / 16 + 2) * 16;  // X box rows of the widest halo tile (BW = 16)

__device__ __forceinline__ uint64_t mn_sw128_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int BN, bool HT = false>
struct WCfg {
    static constexpr int A_BYTES = 2 * KV * 128;          // 128 output channels = two 64-channel boxes
    static constexpr int B_BOX = (HT ? HALO_ROWS_MAX : KV) * 128;
    static constexpr int B_BYTES = (BN / 64) * B_BOX;     // BN input channels
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = (200 * 1024 / STAGE) > 8 ? 8 : (200 * 1024 / STAGE);
    static constexpr int TMEM_COLS = HT ? 512 : BN;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
    static constexpr uint32_t IDESC = idesc_bf16_mn(128, BN);
};

template <int BN, bool HT>
__global__ void __launch_bounds__(192, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tm_dy, const __grid_constant__ CUtensorMap tm_x,
                    const WgradArgs a, const WtcGeo g, float* __restrict__ part, int* status,
                    unsigned long long wait_ns) {
    using C = WCfg<BN, HT>;
    static_assert(!HT || BN == 128, "three accumulators of 128 columns");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tdone = empty + C::STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tdone + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    // tile: (split, tap, n tile, m tile) with m fastest
    long long t = blockIdx.x;
    const int mt = (int)(t % g.m_tiles);
    t /= g.m_tiles;
    const int nt = (int)(t % g.n_tiles);
    t /= g.n_tiles;
    const int tap = (int)(t % g.taps);
    const int split = (int)(t / g.taps);
    const long long v_begin = (long long)split * g.vtiles / g.S, v_end = (long long)(split + 1) * g.vtiles / g.S;
    // halo form: `tap` is the (dt, dw) slot; dh = 0, 1, 2 are the three accumulators
    // (dw rows: `tap` is dt, the X box unshifted, the dw taps in the rows of dY)
    const int dw = a.dwrows ? 1 : HT ? tap % 3 : tap % a.kw;
    const int dh = HT ? 0 : (tap / a.kw) % a.kh;
    const int dt = a.dwrows ? tap : HT ? tap / 3 : tap / (a.kw * a.kh);
    const int a_boxes = (mt * 128 + 64 < a.Cout) ? 2 : 1;
    const int b_boxes = min(BN / 64, (a.Cin - nt * BN) / 64);
    const int xrows = HT ? (g.BH + 2) * g.BW : KV;  // rows of one X box
    const uint32_t tx_bytes = (uint32_t)(a_boxes * KV + b_boxes * xrows) * 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tdone, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        int s = 0;
        uint32_t ph = 0;
        int last_ph[8];
        for (int i = 0; i < 8; ++i) last_ph[i] = -1;
        // voxel tile vt = ((n * Tout + to) * tiles_h + th) * tiles_w + tw, decoded once and then stepped
        int tw, th, to, n;
        {
            long long m = v_begin;
            tw = (int)(m % g.tiles_w); m /= g.tiles_w;
            th = (int)(m % g.tiles_h); m /= g.tiles_h;
            to = (int)(m % a.Tout);
            n = (int)(m / a.Tout);
        }
        for (long long vt = v_begin; vt < v_end; ++vt) {
            if (vt != v_begin && ++tw == g.tiles_w) {
                tw = 0;
                if (++th == g.tiles_h) {
                    th = 0;
                    if (++to == a.Tout) {
                        to = 0;
                        ++n;
                    }
                }
            }
            if (!mbar_wait(&empty[s], ph ^ 1, status, wait_ns)) break;
            int ti = to * a.st + dt + a.t_off;
            int tcoord;
            if (ti >= a.Tin) tcoord = -1;
            else if (ti >= 0) tcoord = n * a.Tin + ti;
            else if (a.pad_mode == 0) tcoord = n * a.Tin;
            else tcoord = -1;
            uint8_t* sa = smem + s * C::STAGE;
            uint8_t* sb = sa + C::A_BYTES;
            mbar_arrive_expect_tx(&full[s], tx_bytes);
            const int ycoord = n * a.Tout + to;
            for (int j = 0; j < a_boxes; ++j)
                tma_load_4d(sa + j * KV * 128, &tm_dy, &full[s], mt * 128 + j * 64, tw * g.BW, th * g.BH, ycoord);
            if (HT) {
                // rows th*BH - 1 .. th*BH + BH of the input frame (zeros outside)
                for (int j = 0; j < b_boxes; ++j)
                    tma_load_4d(sb + j * C::B_BOX, &tm_x, &full[s], nt * BN + j * 64, tw * g.BW + dw - 1,
                                th * g.BH - 1, tcoord);
            } else if (!g.strided) {
                for (int j = 0; j < b_boxes; ++j)
                    tma_load_4d(sb + j * KV * 128, &tm_x, &full[s], nt * BN + j * 64,
                                tw * g.BW + dw - (a.kw - 1) / 2, th * g.BH + dh - (a.kh - 1) / 2, tcoord);
            } else {
                const int pw = (dw == 1) ? 0 : 1, ph = (dh == 1) ? 0 : 1;
                for (int j = 0; j < b_boxes; ++j)
                    tma_load_5d(sb + j * KV * 128, &tm_x, &full[s], pw * a.Cin + nt * BN + j * 64,
                                tw * g.BW - (dw == 0 ? 1 : 0), ph, th * g.BH - (dh == 0 ? 1 : 0), tcoord);
            }
            last_ph[s] = (int)ph;
            if (++s == C::STAGES) {
                s = 0;
                ph ^= 1;
            }
        }
        for (int i = 0; i < C::STAGES; ++i)
            if (last_ph[i] >= 0) mbar_wait(&full[i], (uint32_t)last_ph[i], status, wait_ns);
    } else if (warp == 1 && lane == 0) {
        int s = 0;
        uint32_t ph = 0;
        bool any = false;
        for (long long vt = v_begin; vt < v_end; ++vt) {
            if (!mbar_wait(&full[s], ph, status, wait_ns)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * C::STAGE);
            const uint32_t sb = sa + C::A_BYTES;
            if constexpr (HT) {
                const uint32_t shift = (uint32_t)g.BW * 128u;  // one input row of the halo box
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tc_mma_bf16(tmem_base + (uint32_t)(d * BN), mn_sw128_desc(sa + k * 2048, KV * 128, 1024),
                                    mn_sw128_desc(sb + d * shift + k * 2048, C::B_BOX, 1024), C::IDESC,
                                    (any || k) ? 1u : 0u);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc_mma_bf16(tmem_base, mn_sw128_desc(sa + k * 2048, KV * 128, 1024),
                                mn_sw128_desc(sb + k * 2048, KV * 128, 1024), C::IDESC, (any || k) ? 1u : 0u);
            }
            any = true;
            tc_commit(&empty[s]);
            if (++s == C::STAGES) {
                s = 0;
                ph ^= 1;
            }
        }
        tc_commit(tdone);
        if (!any) {
            // empty split (more splits than voxel tiles): nothing was accumulated
        }
        mbar_wait(tdone, 0, status, wait_ns);
    } else if (warp >= 2) {
        const int q = warp & 3;
        int okw = 1;
        if (lane == 0) okw = mbar_wait(tdone, 0, status, wait_ns) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (okw) {
            tc_fence_after();
            // The MMAs are done, so the stage ring is free: each warp stages its 32
            // output-channel rows there (row stride BN + 4 floats: the 16-byte writes
            // of 8 consecutive lanes fall in distinct banks), then writes every row as
            // one coalesced run of BN floats.
            constexpr int RS = BN + 4;
            float* buf = reinterpret_cast<float*>(smem) + q * 32 * RS;
            const bool empty_range = v_end <= v_begin;
            const int n_valid = min(BN, a.Cin - nt * BN);  // input channels of this tile (a multiple of 16)
#pragma unroll 1
            for (int d = 0; d < (HT ? 3 : 1); ++d) {
                const int tp = HT ? (dt * 3 + d) * 3 + dw : tap;  // the conv tap of accumulator d
#pragma unroll 1
                for (int c64 = 0; c64 < BN / 64; ++c64) {
                    uint32_t r[4][16];
                    const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * BN + c64 * 64);
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmem_ld16_issue(ta + (uint32_t)(k * 16), r[k]);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 4; ++k) tmem_regs_fence(r[k]);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            *reinterpret_cast<float4*>(buf + lane * RS + c64 * 64 + k * 16 + 4 * i) =
                                empty_range ? make_float4(0.f, 0.f, 0.f, 0.f)
                                            : make_float4(__uint_as_float(r[k][4 * i]), __uint_as_float(r[k][4 * i + 1]),
                                                          __uint_as_float(r[k][4 * i + 2]),
                                                          __uint_as_float(r[k][4 * i + 3]));
                }
                __syncwarp();
                for (int rr = 0; rr < 32; ++rr) {
                    const int r = mt * 128 + q * 32 + rr;  // accumulator row
                    if (r >= a.Cout) break;
                    // output channel and tap of the row (dw rows: r = dw * 16 + co)
                    int co = r, tpr = tp;
                    if (a.dwrows) {
                        co = r % 16;
                        tpr = (dt * 3 + d) * 3 + r / 16;
                        if (co >= a.cout_real) continue;
                    }
                    float* P = part + ((long long)split * (a.dwrows ? a.cout_real : a.Cout) + co) * a.K +
                               (long long)tpr * a.Cin + nt * BN;
#pragma unroll
                    for (int c = 4 * lane; c < BN; c += 128)
                        if (c < n_valid)
                            *reinterpret_cast<float4*>(P + c) = *reinterpret_cast<const float4*>(buf + rr * RS + c);
                }
                __syncwarp();
            }
            tc_fence_before();
        }
    }
    (void)ok;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, C::TMEM_COLS);
}

// Column sums of dY (V rows of Cdy channels, the first Cout summed) into
// per-chunk partials out[chunk][Cout]. A block covers CGT groups of 8
// channels (16-byte loads) and 256 / CGT voxel lanes; lanes are combined in
// a fixed order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) colsum_kernel(const __nv_bfloat16* __restrict__ dy, long long V, int Cdy,
                                                     int Cout, long long vchunk, float* __restrict__ out) {
    __shared__ float red[256 * 8];
    const int CG = (Cout + 7) / 8, CGT = min(CG, 32), lanes = 256 / CGT;
    const int tx = threadIdx.x % CGT, ty = threadIdx.x / CGT;
    const int cg = blockIdx.x * CGT + tx;
    const int chunk = blockIdx.y;
    const long long v0 = chunk * vchunk, v1 = min(V, v0 + vchunk);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (ty < lanes && cg < CG) {
        for (long long v = v0 + ty; v < v1; v += lanes) {
            const uint4 q = *reinterpret_cast<const uint4*>(dy + v * Cdy + cg * 8);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(h[i]);
                acc[2 * i] += f.x;
                acc[2 * i + 1] += f.y;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) red[threadIdx.x * 8 + i] = acc[i];
    __syncthreads();
    if (ty == 0 && cg < CG) {
        float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int l = 0; l < lanes; ++l)
#pragma unroll
            for (int i = 0; i < 8; ++i) t[i] += red[(l * CGT + tx) * 8 + i];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (cg * 8 + i < Cout) out[(long long)chunk * Cout + cg * 8 + i] = t[i];
    }
}

// db[co] = sum over chunks of part[chunk][co]; one warp per column, fixed order.
__global__ void colsum_reduce_kernel(const float* __restrict__ part, int chunks, int Cout, float* __restrict__ db) {
    const int co = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (co >= Cout) return;
    float s = 0.f;
    for (int i = lane; i < chunks; i += 32) s += part[(long long)i * Cout + co];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[co] = s;
}

// dY of a narrow layer as three w-shifted copies: out[v][dw * 16 + co] = dY at
// (v with w - (dw - 1)) channel co, zero outside the frame, past Cout and in
// channels 48..63 (out row pitch 64). A thread writes one 16-byte group of 8
// channels (Cdy a multiple of 8, dY rows 16-byte aligned).
__global__ void dy_dwrows_kernel(const __nv_bfloat16* __restrict__ dy, long long V, int W, int Cdy, int Cout,
                                 __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= V * 8) return;
    const long long v = t >> 3;
    const int grp = (int)(t & 7), dwv = grp >> 1, co0 = (grp & 1) * 8;
    const int w = (int)(v % W), ws = w - (dwv - 1);
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (dwv < 3 && co0 < Cout && ws >= 0 && ws < W) {
        q = *reinterpret_cast<const uint4*>(dy + (v - (dwv - 1)) * Cdy + co0);
        // channels past Cout read as zero
        uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (co0 + 2 * i >= Cout) u[i] = 0u;
            else if (co0 + 2 * i + 1 >= Cout) u[i] &= 0xFFFFu;
        }
        q = make_uint4(u[0], u[1], u[2], u[3]);
    }
    reinterpret_cast<uint4*>(out)[t] = q;
}

__global__ void partial_reduce_kernel(const float* __restrict__ part, int S, long long n, float* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float s = 0.f;
    for (int i = 0; i < S; ++i) s += part[(long long)i * n + t];
    out[t] = s;
}

// Same, keeping the first kv of every K columns (an im2col layer whose K is padded).
__global__ void partial_reduce_crop_kernel(const float* __restrict__ part, int S, int rows, int K, int kv,
                                           float* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)rows * kv) return;
    const long long r = t / kv, k = t % kv, n = (long long)rows * K;
    float s = 0.f;
    for (int i = 0; i < S; ++i) s += part[(long long)i * n + r * K + k];
    out[t] = s;
}

void choose_vtile(int Hout, int Wout, int* BH, int* BW) {
    long long best = -1;
    for (int bw : {64, 32, 16, 8}) {
        const int bh = KV / bw;
        const long long tiles = (long long)((Wout + bw - 1) / bw) * ((Hout + bh - 1) / bh);
        if (best < 0 || tiles < best) {
            best = tiles;
            *BW = bw;
            *BH = bh;
        }
    }
}

// Halo tiles: BW = 8 or 16 (BH = 8 or 4), fewest tiles, then fewest X rows.
void choose_vtile_halo(int Hout, int Wout, int* BH, int* BW) {
    long long best = -1, best_rows = 0;
    for (int bw : {8, 16}) {
        const int bh = KV / bw;
        const long long tiles = (long long)((Wout + bw - 1) / bw) * ((Hout + bh - 1) / bh);
        const long long rows = tiles * (bh + 2) * bw;
        if (best < 0 || tiles < best || (tiles == best && rows < best_rows)) {
            best = tiles;
            best_rows = rows;
            *BW = bw;
            *BH = bh;
        }
    }
}

template <int BN, bool HT>
int launch_bn(const __nv_bfloat16* dy, const __nv_bfloat16* x, const WgradArgs& a, WtcGeo g, float* part,
              int* status, unsigned long long wait_ns, cudaStream_t s) {
    using C = WCfg<BN, HT>;
    CUtensorMap mdy, mx;
    if (!encode_act_map(&mdy, dy, a.N * a.Tout, a.Hout, a.Wout, a.Cdy, g.BH, g.BW, false, 64)) return -1;
    if (!encode_act_map(&mx, x, a.N * a.Tin, a.Hin, a.Win, a.Cin, HT ? g.BH + 2 : g.BH, g.BW, g.strided != 0, 64))
        return -1;
    static std::atomic<unsigned long long> attr{0};
    if (smem_attr_once(wgrad_tc_kernel<BN, HT>, C::SMEM, attr) != cudaSuccess) return (int)cudaGetLastError();
    const long long grid = (long long)g.m_tiles * g.n_tiles * g.taps * g.S;
    wgrad_tc_kernel<BN, HT><<<(unsigned)grid, 192, C::SMEM, s>>>(mdy, mx, a, g, part, status, wait_ns);
    return (int)cudaGetLastError();
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// Eligible: BF16; Cin a multiple of 64; dY channel stride a multiple of 64
// holding all Cout channels; stride 1 or 2 in time; stride 1 in h and w, or 2
// with a 3x3 spatial kernel over an even input frame.
bool wgrad_tc_ok(const WgradArgs& a) {
    const bool hw_ok = (a.sh == 1 && a.sw == 1) ||
                       (a.sh == 2 && a.sw == 2 && a.kh == 3 && a.kw == 3 && a.Hin % 2 == 0 && a.Win % 2 == 0 &&
                        a.Hout == a.Hin / 2 && a.Wout == a.Win / 2);
    return (a.st == 1 || a.st == 2) && hw_ok && a.Cin % 64 == 0 && a.Cin > 0 && a.Cout > 0 && a.Cdy % 64 == 0 &&
           a.Cdy >= a.Cout;
}

// dw (Cout x K, or Cout x k_valid when 0 < k_valid < K) and db (Cout) in
// FP32; `part` holds the split partials (at most max_floats floats).
int launch_wgrad_tc(const __nv_bfloat16* dy, const __nv_bfloat16* x, const WgradArgs& a, float* part,
                    size_t max_floats, float* dw, float* db, int num_sms, int* status, unsigned long long wait_ns,
                    cudaStream_t s, int k_valid) {
    WtcGeo g;
    g.strided = (a.sh == 2) ? 1 : 0;
    // stride-1 3x3 spatial taps: the halo form with 128 input channels per tile
    const bool ht = a.sh == 1 && a.sw == 1 && a.kh == 3 && a.kw == 3;
    if (ht)
        choose_vtile_halo(a.Hout, a.Wout, &g.BH, &g.BW);
    else
        choose_vtile(a.Hout, a.Wout, &g.BH, &g.BW);
    g.tiles_w = (a.Wout + g.BW - 1) / g.BW;
    g.tiles_h = (a.Hout + g.BH - 1) / g.BH;
    g.vtiles = (long long)a.N * a.Tout * g.tiles_h * g.tiles_w;
    const int BN = (!ht && a.Cin % 256 == 0) ? 256 : 128;
    // a narrow stride-1 3x3x3 layer runs with its dw taps as rows of a shifted copy of
    // dY (one CTA slot per dt instead of per (dt, dw)); the copy sits at the end of the
    // partials buffer
    WgradArgs ar = a;
    ar.dwrows = 0;
    ar.cout_real = a.Cout;
    const __nv_bfloat16* dyk = dy;
    const size_t dy3_floats = ((size_t)a.V * 64 * 2 + 255) / 256 * 64;  // bf16 copy, in floats, 256-byte granules
    if (ht && a.kt == 3 && a.st == 1 && a.Cout <= 16 && k_valid <= 0 && dy3_floats < max_floats / 2) {
        __nv_bfloat16* dy3 = reinterpret_cast<__nv_bfloat16*>(part + (max_floats - dy3_floats) / 64 * 64);
        dy_dwrows_kernel<<<blocks_for(a.V * 8, 256), 256, 0, s>>>(dy, a.V, a.Wout, a.Cdy, a.Cout, dy3);
        max_floats = (max_floats - dy3_floats) / 64 * 64;
        ar.dwrows = 1;
        ar.Cout = 48;
        ar.Cdy = 64;
        dyk = dy3;
    }
    g.m_tiles = (ar.Cout + 127) / 128;
    g.n_tiles = (a.Cin + BN - 1) / BN;
    g.taps = ar.dwrows ? a.kt : ht ? a.kt * a.kw : a.kt * a.kh * a.kw;
    const long long out_tiles = (long long)g.m_tiles * g.n_tiles * g.taps;
    // split count: at least 4 voxel tiles per split, partials within max_floats;
    // time ~ waves x (voxel tiles per split + a CTA's fixed cost), the fixed cost
    // (TMEM allocation, pipeline fill, draining three accumulators to the FP32
    // partials) measured at about 30 voxel tiles' worth of MMAs on B300
    constexpr double kCtaFixed = 30.0;
    const long long s_max = std::max(1LL, std::min(g.vtiles / 4, (long long)(max_floats / ((size_t)a.Cout * a.K))));
    const long long s_cap = std::min(s_max, std::max(1LL, (4LL * num_sms + out_tiles - 1) / out_tiles));
    long long S = 1;
    double best = -1.0;
    for (long long sc = 1; sc <= s_cap; ++sc) {
        const long long ctas = out_tiles * sc, waves = (ctas + num_sms - 1) / num_sms;
        const double t = (double)waves * ((double)g.vtiles / (double)sc + kCtaFixed);
        if (best < 0.0 || t < best) {
            best = t;
            S = sc;
        }
    }
    if ((size_t)S * a.Cout * a.K > max_floats) return -1;
    g.S = (int)S;
    int e = ht ? launch_bn<128, true>(dyk, x, ar, g, part, status, wait_ns, s)
               : (BN == 256) ? launch_bn<256, false>(dyk, x, ar, g, part, status, wait_ns, s)
                             : launch_bn<128, false>(dyk, x, ar, g, part, status, wait_ns, s);
    if (e) return e;
    const long long n = (long long)a.Cout * a.K;
    if (k_valid > 0 && k_valid < a.K)
        partial_reduce_crop_kernel<<<blocks_for((long long)a.Cout * k_valid, 256), 256, 0, s>>>(part, g.S, a.Cout,
                                                                                               a.K, k_valid, dw);
    else
        partial_reduce_kernel<<<blocks_for(n, 256), 256, 0, s>>>(part, g.S, n, dw);
    if (db) {
        // column sums of dY, reusing the (now consumed) partial buffer
        const int cgt = std::min((a.Cout + 7) / 8, 32);
        const int gx = ((a.Cout + 7) / 8 + cgt - 1) / cgt;
        const int chunks = (int)std::max<long long>(1, std::min<long long>(4LL * num_sms / gx, a.V / 256));
        const long long vchunk = (a.V + chunks - 1) / chunks;
        colsum_kernel<<<dim3(gx, chunks), 256, 0, s>>>(dy, a.V, a.Cdy, a.Cout, vchunk, part);
        colsum_reduce_kernel<<<(a.Cout + 7) / 8, 256, 0, s>>>(part, chunks, a.Cout, db);
    }
    return (int)cudaGetLastError();
}

}  // namespace tok
