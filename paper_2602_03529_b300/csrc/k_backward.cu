// Backward kernels of the tokenizer's training step (joint encoder/decoder
// training through the masked decode, Sec. 7 / Appendix A.2; MSE objective,
// straight-through FSQ):
//   wgrad        dW[co][tap][ci] = sum_v dY[v][co] * X_tap(v)[ci] and
//                db[co] = sum_v dY[v][co]: split-K over voxels into FP32
//                partials, then a fixed-order reduction (deterministic).
//   GN+SiLU bwd  three passes: per (frame, chunk) partial sums of
//                g = dy*SiLU'(h)*gamma and g*xhat (and per-channel dgamma,
//                dbeta), fixed-order finalize, then
//                dx = rstd * (g - mean(g) - xhat * mean(g*xhat)) (+ a skip term).
//   STE bwd      dz_i = dcode_i * h_i (1 - tanh^2(z_i + s_i)) / floor(L_i/2) at
//                kept tokens, 0 at dropped ones.
//   s2d          adjoint of depth-to-space (zeros for the trimmed frames).
//   zero insert  adjoint of a stride-2 conv as a stride-1 one over dY spread
//                onto the input grid.
//   MSE          loss = mean((xhat - x)^2) and d loss / d xhat.
//   weight packs flipped / transposed weights for the adjoint convs.
//   SGD          p -= lr * g.
// All are bandwidth-bound except wgrad (CUDA-core FP32 FMA).
#include "common.cuh"
#include "conv_args.h"
#include "launchers.h"

#include <algorithm>
#include <type_traits>

namespace tok {

namespace {

template <typename T>
__device__ __forceinline__ float ldf(const T* p) {
    if constexpr (sizeof(T) == 2)
        return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
    else
        return *p;
}

template <typename T>
__device__ __forceinline__ void stf(T* p, float v) {
    if constexpr (sizeof(T) == 2)
        *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
    else
        *p = v;
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ wgrad

constexpr int WB = 64;  // co tile and k tile
constexpr int WV = 16;  // voxels per step

template <typename T>
__global__ void __launch_bounds__(256) wgrad_kernel(const T* __restrict__ dy, const T* __restrict__ x, WgradArgs a,
                                                    float* __restrict__ part, float* __restrict__ dbpart) {
    __shared__ __align__(16) float dyS[WV][WB];
    __shared__ __align__(16) float xS[WV][WB];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int co0 = blockIdx.x * WB, k0 = blockIdx.y * WB, split = blockIdx.z;
    const long long v_begin = (long long)split * a.vchunk;
    const long long v_end = min(a.V, v_begin + a.vchunk);
    float acc[4][4] = {};
    float dbacc[4] = {};
    const bool do_db = blockIdx.y == 0 && tx == 0;
    // loader role: voxel lv (0..15), 4 consecutive columns lc
    const int lv = tid / 16, lc = (tid % 16) * 4;
    for (long long v0 = v_begin; v0 < v_end; v0 += WV) {
        const long long v = v0 + lv;
        float dyv[4] = {0.f, 0.f, 0.f, 0.f}, xv[4] = {0.f, 0.f, 0.f, 0.f};
        if (v < v_end) {
            const T* dp = dy + v * a.Cdy;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (co0 + lc + e < a.Cout) dyv[e] = ldf(dp + co0 + lc + e);
            long long m = v;
            const int wo = (int)(m % a.Wout); m /= a.Wout;
            const int ho = (int)(m % a.Hout); m /= a.Hout;
            const int to = (int)(m % a.Tout);
            const int n = (int)(m / a.Tout);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = k0 + lc + e;
                if (k >= a.K) continue;
                const int tap = k / a.Cin, ci = k - tap * a.Cin;
                const int dw = tap % a.kw, dh = (tap / a.kw) % a.kh, dt = tap / (a.kw * a.kh);
                const int hi = ho * a.sh + dh - (a.kh - 1) / 2, wi = wo * a.sw + dw - (a.kw - 1) / 2;
                if (hi < 0 || hi >= a.Hin || wi < 0 || wi >= a.Win) continue;
                int ti = to * a.st + dt + a.t_off;
                if (ti < 0) {
                    if (a.pad_mode != 0) continue;
                    ti = 0;
                }
                if (ti >= a.Tin) continue;
                xv[e] = ldf(x + ((((long long)n * a.Tin + ti) * a.Hin + hi) * a.Win + wi) * a.Cin + ci);
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            dyS[lv][lc + e] = dyv[e];
            xS[lv][lc + e] = xv[e];
        }
        __syncthreads();
#pragma unroll
        for (int vv = 0; vv < WV; ++vv) {
            const float4 d4 = *reinterpret_cast<const float4*>(&dyS[vv][ty * 4]);
            const float4 x4 = *reinterpret_cast<const float4*>(&xS[vv][tx * 4]);
            const float dv[4] = {d4.x, d4.y, d4.z, d4.w}, xw[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], xw[j], acc[i][j]);
            if (do_db) {
#pragma unroll
                for (int i = 0; i < 4; ++i) dbacc[i] += dv[i];
            }
        }
    }
    float* P = part + (long long)split * a.Cout * a.K;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + ty * 4 + i;
        if (co >= a.Cout) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + tx * 4 + j;
            if (k < a.K) P[(long long)co * a.K + k] = acc[i][j];
        }
        if (do_db) dbpart[(long long)split * a.Cout + co] = dbacc[i];
    }
}

__global__ void wgrad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ dbpart, int S, int Cout,
                                    int K, float* __restrict__ dw, float* __restrict__ db) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)Cout * K;
    if (t < n) {
        float s = 0.f;
        for (int i = 0; i < S; ++i) s += part[(long long)i * n + t];
        dw[t] = s;
    }
    if (db && t < Cout) {
        float s = 0.f;
        for (int i = 0; i < S; ++i) s += dbpart[(long long)i * Cout + t];
        db[t] = s;
    }
}

// ------------------------------------------------------------ GN+SiLU bwd

constexpr int NT = 256;

template <typename T>
struct V8;
template <>
struct V8<float> {
    static constexpr int N = 4;
};
template <>
struct V8<__nv_bfloat16> {
    static constexpr int N = 8;
};

template <typename T>
__device__ __forceinline__ void ldv(const T* p, float (&v)[V8<T>::N]) {
    if constexpr (sizeof(T) == 2) {
        const uint4 q = *reinterpret_cast<const uint4*>(p);
        const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = unpack_bf16x2(u[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    } else {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    }
}

// Raw 16-byte vectors, loaded ahead of use and unpacked when consumed.
template <typename T>
struct Raw {
    using type = typename std::conditional<sizeof(T) == 2, uint4, float4>::type;
};
template <typename T>
__device__ __forceinline__ typename Raw<T>::type ldraw(const T* p) {
    return *reinterpret_cast<const typename Raw<T>::type*>(p);
}
template <typename T>
__device__ __forceinline__ void unpack(const typename Raw<T>::type& q, float (&v)[V8<T>::N]) {
    if constexpr (sizeof(T) == 2) {
        const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = unpack_bf16x2(u[i]);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    } else {
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    }
}
constexpr int GN_BWD_VPT = 8;  // GN backward: 16-byte vectors per thread of a chunk

template <typename T>
__device__ __forceinline__ void stv(T* p, const float (&v)[V8<T>::N]) {
    if constexpr (sizeof(T) == 2) {
        uint4 q;
        q.x = pack_bf16x2(v[0], v[1]);
        q.y = pack_bf16x2(v[2], v[3]);
        q.z = pack_bf16x2(v[4], v[5]);
        q.w = pack_bf16x2(v[6], v[7]);
        *reinterpret_cast<uint4*>(p) = q;
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// GN + SiLU backward, with h = xhat * gamma + beta and y = SiLU(h):
//   dh   = dy * s * (1 + h * (1 - s)),  s = sigmoid(h)
//   g    = dh * gamma
//   dx   = rstd * (g - mean_group(g) - xhat * mean_group(g * xhat))
//   dgamma = sum dh * xhat,  dbeta = sum dh   (over frames and voxels)
//
// The group means need a whole frame, so dx takes two sweeps of x and dy: a
// reduction per (frame, chunk), the group means per frame, then dx per
// (frame, chunk). (One cooperative launch over L2-sized batches of frames, which
// reads x and dy from HBM once, measured slower: with one chunk per block and
// phase, each sweep is a chain of dependent loads.)
//
// sigmoid: BF16 path 1/2 + tanh(h/2)/2 (one tanh.approx; its error is below
// the bf16 rounding of dx), FP32 path 1 / (1 + exp(-h)).
template <typename T>
__device__ __forceinline__ float gn_bwd_sigmoid(float h) {
    if constexpr (sizeof(T) == 2)
        return fmaf(0.5f, tanh_approx(0.5f * h), 0.5f);
    else
        return 1.f / (1.f + expf(-h));
}

template <typename T>
struct GnBwdArgs {
    const T* x;
    const T* dy;
    const float2* stats;  // (mean, rstd) per (frame, group), from the forward
    const float* gamma;   // null: 1
    const float* beta;    // null: 0
    const T* add;         // null, or a gradient added to dx
    T* dx;
    long long frames, vpf;  // vectors of V channels per frame
    int C, G, S, vpt;       // S chunks of NT * vpt vectors per frame
    float2* pg;             // [frames][S][G]: (sum g, sum g * xhat) per chunk
    float2* pc;             // [frames][S][C]: (sum dh * xhat, sum dh) per chunk
    float2* gstat;          // [frames][G]: (mean g, mean g * xhat)
    int* status;
    unsigned long long wait_ns;
};

// A chunk's vectors of x, dy (and add) arrive in GN_BWD_SEGS bulk copies per
// tensor into shared memory (one mbarrier per segment for all tensors), so that
// each thread works from shared memory while later segments land; 32 KB of
// every tensor per chunk keeps three blocks per SM.
constexpr int GN_BWD_SEGS = 4;
constexpr int GN_BWD_SEG = NT * GN_BWD_VPT * 16 / GN_BWD_SEGS;  // bytes per segment and tensor

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Issue the copies of one chunk (thread 0); returns the chunk's bytes per tensor.
template <typename T>
__device__ __forceinline__ long long gn_bwd_stage(const GnBwdArgs<T>& a, long long frame, int chunk, uint8_t* sm,
                                                  uint64_t* bar, int ntensors) {
    constexpr int V = V8<T>::N;
    const long long v0 = (long long)chunk * NT * a.vpt;
    const long long bytes = min((long long)NT * a.vpt, a.vpf - v0) * 16;
    const long long e0 = (frame * a.vpf + v0) * V;  // first element of the chunk
    if (threadIdx.x == 0) {
        for (int sg = 0; sg < GN_BWD_SEGS; ++sg) mbar_init(&bar[sg], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const T* src[3] = {a.x + e0, a.dy + e0, a.add ? a.add + e0 : nullptr};
        for (int sg = 0; sg < GN_BWD_SEGS; ++sg) {
            const long long b = min((long long)GN_BWD_SEG, bytes - (long long)sg * GN_BWD_SEG);
            if (b <= 0) break;
            mbar_arrive_expect_tx(&bar[sg], (uint32_t)(b * ntensors));
            for (int t = 0; t < ntensors; ++t)
                bulk_g2s(sm + (t * GN_BWD_SEGS + sg) * GN_BWD_SEG, src[t] + (long long)sg * (GN_BWD_SEG / 16) * V,
                         (uint32_t)b, &bar[sg]);
        }
    }
    return bytes;
}

// Reduction of one (frame, chunk): per channel (sum dh*xhat, sum dh) combined
// over the block in a fixed tree order; the group sums follow as gamma-weighted
// channel sums (sum g = sum_c gamma_c sum dh, sum g*xhat = sum_c gamma_c sum dh*xhat).
template <typename T>
__device__ __forceinline__ void gn_bwd_reduce_unit(const GnBwdArgs<T>& a, long long frame, int chunk, uint8_t* sm,
                                                   uint64_t* bar, float2 (&redc)[V8<T>::N][NT]) {
    constexpr int V = V8<T>::N;
    const int tid = threadIdx.x;
    const int vpv = a.C / V, cg = a.C / a.G;
    const int c0 = (tid % vpv) * V;  // vector i of the chunk holds channels (i % vpv) * V .., i = tid (mod NT)
    const long long bytes = gn_bwd_stage(a, frame, chunk, sm, bar, 2);
    // xhat = x * rs + xb, h = x * hs + hb (per channel)
    float rs[V], xb[V], hs[V], hb[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const float2 st = a.stats[frame * a.G + (c0 + j) / cg];
        const float ga = a.gamma ? a.gamma[c0 + j] : 1.f, be = a.beta ? a.beta[c0 + j] : 0.f;
        rs[j] = st.y;
        xb[j] = -st.x * st.y;
        hs[j] = st.y * ga;
        hb[j] = fmaf(xb[j], ga, be);
    }
    float sdx[V] = {}, sd[V] = {};
    bool ok = true;
    for (int sg = 0; sg < GN_BWD_SEGS && ok; ++sg) {
        const long long b = min((long long)GN_BWD_SEG, bytes - (long long)sg * GN_BWD_SEG);
        if (b <= 0) break;
        if (!mbar_wait(&bar[sg], 0, a.status, a.wait_ns)) {
            ok = false;
            break;
        }
        const uint4* qx = reinterpret_cast<const uint4*>(sm + sg * GN_BWD_SEG);
        const uint4* qg = reinterpret_cast<const uint4*>(sm + (GN_BWD_SEGS + sg) * GN_BWD_SEG);
        const int n = (int)(b / 16);
        for (int i = tid; i < n; i += NT) {
            float xv[V], gv[V];
            unpack<T>(*reinterpret_cast<const typename Raw<T>::type*>(qx + i), xv);
            unpack<T>(*reinterpret_cast<const typename Raw<T>::type*>(qg + i), gv);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float xh = fmaf(xv[j], rs[j], xb[j]);
                const float h = fmaf(xv[j], hs[j], hb[j]);
                const float sg1 = gn_bwd_sigmoid<T>(h);
                const float dh = gv[j] * sg1 * fmaf(h, 1.f - sg1, 1.f);
                sdx[j] = fmaf(dh, xh, sdx[j]);
                sd[j] += dh;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) redc[j][tid] = make_float2(sdx[j], sd[j]);
    __syncthreads();
    for (int stride = NT / 2; stride >= vpv; stride >>= 1) {
        if (tid < stride) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                redc[j][tid].x += redc[j][tid + stride].x;
                redc[j][tid].y += redc[j][tid + stride].y;
            }
        }
        __syncthreads();
    }
    const long long row = frame * a.S + chunk;
    for (int c = tid; c < a.C; c += NT) a.pc[row * a.C + c] = redc[c % V][c / V];
    for (int g = tid; g < a.G; g += NT) {
        float2 acc = make_float2(0.f, 0.f);
        for (int c = g * cg; c < (g + 1) * cg; ++c) {
            const float2 r = redc[c % V][c / V];
            const float gc = a.gamma ? a.gamma[c] : 1.f;
            acc.x = fmaf(gc, r.y, acc.x);
            acc.y = fmaf(gc, r.x, acc.y);
        }
        a.pg[row * a.G + g] = acc;
    }
}

// dx (+ add) of one (frame, chunk), given the frame's group means gst[g] =
// (mean g, mean g * xhat).
template <typename T>
__device__ __forceinline__ void gn_bwd_apply_unit(const GnBwdArgs<T>& a, long long frame, int chunk, uint8_t* sm,
                                                  uint64_t* bar, const float2* gst) {
    constexpr int V = V8<T>::N;
    const int tid = threadIdx.x;
    const int vpv = a.C / V, cg = a.C / a.G;
    const int c0 = (tid % vpv) * V;
    const int nt = a.add ? 3 : 2;
    const long long bytes = gn_bwd_stage(a, frame, chunk, sm, bar, nt);
    // h = x * hs + hb; dx = rstd * (dh * gamma - m1 - xhat * m2) = ka * dh + (k0 + k1 * x)
    // with xhat = (x - mean) * rstd
    float hs[V], hb[V], ka[V], k0[V], k1[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int g = (c0 + j) / cg;
        const float2 st = a.stats[frame * a.G + g];
        const float2 gs = gst[g];
        const float ga = a.gamma ? a.gamma[c0 + j] : 1.f, be = a.beta ? a.beta[c0 + j] : 0.f;
        const float mu = st.x, rs = st.y;
        hs[j] = rs * ga;
        hb[j] = fmaf(-mu * rs, ga, be);
        ka[j] = rs * ga;
        k1[j] = -rs * rs * gs.y;
        k0[j] = fmaf(rs * rs * gs.y, mu, -rs * gs.x);
    }
    const long long e0 = (frame * a.vpf + (long long)chunk * NT * a.vpt) * V;
    for (int sg = 0; sg < GN_BWD_SEGS; ++sg) {
        const long long b = min((long long)GN_BWD_SEG, bytes - (long long)sg * GN_BWD_SEG);
        if (b <= 0) break;
        if (!mbar_wait(&bar[sg], 0, a.status, a.wait_ns)) return;
        const uint4* qx = reinterpret_cast<const uint4*>(sm + sg * GN_BWD_SEG);
        const uint4* qg = reinterpret_cast<const uint4*>(sm + (GN_BWD_SEGS + sg) * GN_BWD_SEG);
        const uint4* qa = reinterpret_cast<const uint4*>(sm + (2 * GN_BWD_SEGS + sg) * GN_BWD_SEG);
        const int n = (int)(b / 16), i0 = sg * (GN_BWD_SEG / 16);
        for (int i = tid; i < n; i += NT) {
            float xv[V], gv[V], av[V], r[V];
            unpack<T>(*reinterpret_cast<const typename Raw<T>::type*>(qx + i), xv);
            unpack<T>(*reinterpret_cast<const typename Raw<T>::type*>(qg + i), gv);
            if (a.add) unpack<T>(*reinterpret_cast<const typename Raw<T>::type*>(qa + i), av);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float h = fmaf(xv[j], hs[j], hb[j]);
                const float sg1 = gn_bwd_sigmoid<T>(h);
                const float dh = gv[j] * sg1 * fmaf(h, 1.f - sg1, 1.f);
                r[j] = fmaf(ka[j], dh, fmaf(k1[j], xv[j], k0[j]));
                if (a.add) r[j] += av[j];
            }
            stv(a.dx + e0 + (long long)(i0 + i) * V, r);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(NT, 3) gn_bwd_reduce_kernel(const __grid_constant__ GnBwdArgs<T> a) {
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ float2 redc[V8<T>::N][NT];  // [channel slot][thread]: consecutive threads, consecutive banks
    __shared__ uint64_t bar[GN_BWD_SEGS];
    gn_bwd_reduce_unit<T>(a, blockIdx.y, blockIdx.x, sm, bar, redc);
}

// Per (frame, group) the chunk sums, one warp each (lanes take chunks lane,
// lane + 32, ...; a fixed shuffle tree combines them).
__global__ void gn_bwd_finalize_kernel(const float2* __restrict__ pg, long long frames, int S, int G, float inv_n,
                                       float2* __restrict__ gstat) {
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (wid >= frames * G) return;
    const long long frame = wid / G;
    const int g = (int)(wid % G);
    float s0 = 0.f, s1 = 0.f;
    for (int c = lane; c < S; c += 32) {
        const float2 v = pg[(frame * S + c) * G + g];
        s0 += v.x;
        s1 += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) gstat[wid] = make_float2(s0 * inv_n, s1 * inv_n);
}

template <typename T>
__global__ void __launch_bounds__(NT, 2) gn_bwd_apply_kernel(const __grid_constant__ GnBwdArgs<T> a) {
    extern __shared__ __align__(128) uint8_t sm[];
    __shared__ uint64_t bar[GN_BWD_SEGS];
    gn_bwd_apply_unit<T>(a, blockIdx.y, blockIdx.x, sm, bar, a.gstat + (long long)blockIdx.y * a.G);
}

// Per channel over all (frame, chunk) rows, in two steps: blocks of 32 channels
// x 8 row lanes sum a band of rows into q[band][C], then one warp per channel
// sums the bands.
constexpr int GN_BANDS = 128;

__global__ void __launch_bounds__(256) gn_bwd_channel_kernel(const float2* __restrict__ pc, long long rows, int C,
                                                             float2* __restrict__ q) {
    __shared__ float2 red[8][32];
    const int cx = threadIdx.x % 32, ry = threadIdx.x / 32;
    const int c = blockIdx.x * 32 + cx, band = blockIdx.y;
    const long long r0 = rows * band / GN_BANDS, r1 = rows * (band + 1) / GN_BANDS;
    float a = 0.f, b = 0.f;
    if (c < C)
        for (long long r = r0 + ry; r < r1; r += 8) {
            const float2 v = pc[r * C + c];
            a += v.x;
            b += v.y;
        }
    red[ry][cx] = make_float2(a, b);
    __syncthreads();
    if (ry == 0 && c < C) {
        float2 t = red[0][cx];
        for (int l = 1; l < 8; ++l) {
            t.x += red[l][cx].x;
            t.y += red[l][cx].y;
        }
        q[(long long)band * C + c] = t;
    }
}

__global__ void gn_bwd_channel_final_kernel(const float2* __restrict__ q, int C, float* __restrict__ dgamma,
                                            float* __restrict__ dbeta) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (c >= C) return;
    float a = 0.f, b = 0.f;
    for (int i = lane; i < GN_BANDS; i += 32) {
        a += q[(long long)i * C + c].x;
        b += q[(long long)i * C + c].y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        if (dgamma) dgamma[c] = a;
        if (dbeta) dbeta[c] = b;
    }
}

// ------------------------------------------------------------- STE / mask

template <typename T>
__global__ void ste_bwd_kernel(const T* __restrict__ dcodes, int Cd, const float* __restrict__ z,
                               const uint32_t* __restrict__ keep_bits, long long ntok, int Wq, FsqConsts f,
                               T* __restrict__ dz, int Co) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    bool keep = true;
    if (keep_bits) {
        const int nwords = (Wq + 31) / 32;
        const long long row = t / Wq;
        const int w = (int)(t % Wq);
        keep = (keep_bits[row * nwords + w / 32] >> (w % 32)) & 1u;
    }
    for (int c = 0; c < Co; ++c) {
        float v = 0.f;
        if (c < f.nlev && keep) {
            const float th = tanhf(z[t * f.nlev + c] + f.shift[c]);
            v = ldf(dcodes + t * Cd + c) * f.half_l[c] * (1.f - th * th) / (float)f.half_w[c];
        }
        stf(dz + t * Co + c, v);
    }
}

// Dequantised codes with dropped tokens zeroed (the decoder input of a training step).
template <typename T>
__global__ void codes_kernel(const int32_t* __restrict__ idx, long long ntok, FsqConsts f, T* __restrict__ codes) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    const int id = idx[t];
    for (int i = 0; i < f.nlev; ++i) {
        const int d = (id / f.basis[i]) % f.levels[i];
        stf(codes + t * f.nlev + i, (float)(d - f.half_w[i]) / (float)f.half_w[i]);
    }
}

// ------------------------------------------------------------------ s2d

template <typename Ti, typename To>
__global__ void s2d_kernel(const Ti* __restrict__ d, int N, int oT, int oH, int oW, int C, int rt, int rh, int rw,
                           int drop_t, int T, int H, int W, int Cpad, To* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N * T * H * W * Cpad;
    if (t >= total) return;
    long long r = t;
    const int co = (int)(r % Cpad); r /= Cpad;
    const int w = (int)(r % W); r /= W;
    const int h = (int)(r % H); r /= H;
    const int tt = (int)(r % T);
    const int n = (int)(r / T);
    float v = 0.f;
    if (co < C * rt * rh * rw) {
        const int ch = co % C, sub = co / C;
        const int c = sub % rw, b = (sub / rw) % rh, a = sub / (rw * rh);
        const int ot = tt * rt + a - drop_t, oh = h * rh + b, ow = w * rw + c;
        if (ot >= 0 && ot < oT && oh < oH && ow < oW)
            v = ldf(d + ((((long long)n * oT + ot) * oH + oh) * oW + ow) * C + ch);
    }
    stf(out + t, v);
}

// 16-byte forms of the two gradient reshapes (bf16, channel counts multiples of
// 8): a thread moves 8 consecutive channels, which share one sub-position.
__global__ void s2d_vec8_kernel(const uint4* __restrict__ d, int N, int oT, int oH, int oW, int C, int rt, int rh,
                                int rw, int drop_t, int T, int H, int W, int Cpad, uint4* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int G = Cpad / 8;
    const long long total = (long long)N * T * H * W * G;
    if (t >= total) return;
    long long r = t / G;
    const int co0 = (int)(t - r * G) * 8;
    const int w = (int)(r % W); r /= W;
    const int h = (int)(r % H); r /= H;
    const int tt = (int)(r % T);
    const int n = (int)(r / T);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (co0 < C * rt * rh * rw) {
        const int sub = co0 / C, ch0 = co0 - sub * C;
        const int c = sub % rw, b = (sub / rw) % rh, a = sub / (rw * rh);
        const int ot = tt * rt + a - drop_t, oh = h * rh + b, ow = w * rw + c;
        if (ot >= 0 && ot < oT && oh < oH && ow < oW)
            v = d[(((((long long)n * oT + ot) * oH + oh) * oW + ow) * C + ch0) / 8];
    }
    out[t] = v;
}

__global__ void zero_insert_vec8_kernel(const uint4* __restrict__ dy, int N, int To, int Ho, int Wo, int C, int Tin,
                                        int Hin, int Win, int st, int sh, int sw, uint4* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int G = C / 8;
    const long long total = (long long)N * Tin * Hin * Win * G;
    if (t >= total) return;
    long long r = t / G;
    const int g = (int)(t - r * G);
    const int w = (int)(r % Win); r /= Win;
    const int h = (int)(r % Hin); r /= Hin;
    const int tt = (int)(r % Tin);
    const int n = (int)(r / Tin);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (tt % st == 0 && h % sh == 0 && w % sw == 0) {
        const int a = tt / st, b = h / sh, e = w / sw;
        if (a < To && b < Ho && e < Wo) v = dy[((((long long)n * To + a) * Ho + b) * Wo + e) * G + g];
    }
    out[t] = v;
}

// The pixel head's gradient (fp32 frames -> bf16 rows of Cpad channels): one
// thread per output voxel writes its row in 16-byte pieces.
__global__ void s2d_head_kernel(const float* __restrict__ d, int N, int oT, int oH, int oW, int C, int rt, int rh,
                                int rw, int drop_t, int T, int H, int W, int Cpad, uint4* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N * T * H * W;
    if (t >= total) return;
    long long r = t;
    const int w = (int)(r % W); r /= W;
    const int h = (int)(r % H); r /= H;
    const int tt = (int)(r % T);
    const int n = (int)(r / T);
    const int used = C * rt * rh * rw;
    for (int co0 = 0; co0 < Cpad; co0 += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int co = co0 + j;
            v[j] = 0.f;
            if (co < used) {
                const int sub = co / C, ch = co - sub * C;
                const int c = sub % rw, b = (sub / rw) % rh, a = sub / (rw * rh);
                const int ot = tt * rt + a - drop_t, oh = h * rh + b, ow = w * rw + c;
                if (ot >= 0 && ot < oT && oh < oH && ow < oW)
                    v[j] = d[((((long long)n * oT + ot) * oH + oh) * oW + ow) * C + ch];
            }
        }
        out[t * (Cpad / 8) + co0 / 8] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                                                   pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
    }
}

template <typename T>
__global__ void zero_insert_kernel(const T* __restrict__ dy, int N, int To, int Ho, int Wo, int C, int Tin, int Hin,
                                   int Win, int st, int sh, int sw, T* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N * Tin * Hin * Win * C;
    if (t >= total) return;
    long long r = t;
    const int c = (int)(r % C); r /= C;
    const int w = (int)(r % Win); r /= Win;
    const int h = (int)(r % Hin); r /= Hin;
    const int tt = (int)(r % Tin);
    const int n = (int)(r / Tin);
    float v = 0.f;
    if (tt % st == 0 && h % sh == 0 && w % sw == 0) {
        const int a = tt / st, b = h / sh, e = w / sw;
        if (a < To && b < Ho && e < Wo) v = ldf(dy + ((((long long)n * To + a) * Ho + b) * Wo + e) * C + c);
    }
    stf(out + t, v);
}

// ------------------------------------------------------------------ MSE

template <typename T>
__global__ void mse_partial_kernel(const float* __restrict__ xh, const T* __restrict__ x, long long n, float scale,
                                   float* __restrict__ dxh, float* __restrict__ part) {
    __shared__ float red[256];
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = xh[i] - ldf(x + i);
        s += d * d;
        if (dxh) dxh[i] = scale * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void mse_final_kernel(const float* __restrict__ part, int nb, float inv_n, float* __restrict__ loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += part[i];
        *loss = (float)(s * inv_n);
    }
}

// ---------------------------------------------------------- weight packs

// Adjoint-conv weights: Wf[ci][tap'][co] with tap' the spatio-temporal flip
// of tap (k = 3) or identity (k = 1); rows padded to rows_pad, the co axis to
// cpad per tap. `corr` selects the replicate-pad correction weights (k = 3):
// two temporal taps d'' with V[0] = W[dt=0] + W[dt=1], V[1] = W[dt=0], both
// spatially flipped.
template <typename T>
__global__ void __launch_bounds__(256) pack_adjoint_kernel(const float* __restrict__ w, int Cout, int Cin, int k,
                                                           int rows_pad, int cpad, int corr, T* __restrict__ out) {
    // one output tap, 32 input channels (rows) x 32 output channels (columns),
    // transposed through shared memory so reads run along ci and writes along co
    __shared__ float tile[32][33];
    // corr 0: the adjoint taps; 1: the frame-0 correction (2 taps); 2: the adjoint taps of
    // output frame 0, where the correction is folded in (sum of W over dt <= k-1-dtp)
    const int taps_out = corr == 1 ? 2 * k * k : k * k * k;
    const int tap = blockIdx.z, co0 = blockIdx.x * 32, ci0 = blockIdx.y * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    const int k2 = k * k;
    const int dwp = tap % k, dhp = (tap / k) % k, dtp = tap / k2;
    const int dh = k - 1 - dhp, dw = k - 1 - dwp;
    auto W = [&](int co, int dt, int ci) { return w[(((long long)co * k + dt) * k2 + dh * k + dw) * Cin + ci]; };
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + ty + 8 * i, ci = ci0 + tx;
        float v = 0.f;
        if (co < Cout && ci < Cin) {
            if (corr == 0) {
                v = W(co, k - 1 - dtp, ci);
            } else if (corr == 1) {
                v = dtp == 0 ? W(co, 0, ci) + W(co, 1, ci) : W(co, 0, ci);
            } else {
                for (int dt = 0; dt <= k - 1 - dtp; ++dt) v += W(co, dt, ci);
            }
        }
        tile[ty + 8 * i][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ci = ci0 + ty + 8 * i, co = co0 + tx;
        if (ci < rows_pad && co < cpad) stf(out + ((long long)ci * taps_out + tap) * cpad + co, tile[tx][ty + 8 * i]);
    }
}

// All three BF16 layouts of a 3x3x3 conv from one read of its master weights
// W[co][dt][dh][dw][ci]: the forward rows fwd[co][tap * Cin + ci], the adjoint
// taps wt[ci][tap'][co] (tap' = the flipped tap) and the frame-0 adjoint taps
// wf0[ci][tap'][co] (sum of W over dt <= 2 - dt'). A block takes 32 output x
// 32 input channels of one spatial tap (dh, dw) for all three dt; the two
// adjoint layouts go through a shared-memory transpose.
__device__ __forceinline__ void pack3_tile(const float* __restrict__ w, int Cout, int Cin, int Cout_pad, int Kpad,
                                           int rows_pad, int cpad, __nv_bfloat16* __restrict__ fwd,
                                           __nv_bfloat16* __restrict__ wt, __nv_bfloat16* __restrict__ wf0, int bx,
                                           int by, int hw, float (&tile)[3][32][33]) {
    const int dh = hw / 3, dw = hw % 3;
    const int co0 = bx * 32, ci0 = by * 32;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
    for (int dt = 0; dt < 3; ++dt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int co = co0 + ty + 8 * i, ci = ci0 + tx;
            const float v = (co < Cout && ci < Cin) ? w[(((long long)co * 3 + dt) * 9 + dh * 3 + dw) * Cin + ci] : 0.f;
            tile[dt][ty + 8 * i][tx] = v;
            const int tap = (dt * 3 + dh) * 3 + dw;
            if (co < Cout_pad && ci < Cin) fwd[(long long)co * Kpad + (long long)tap * Cin + ci] = __float2bfloat16_rn(v);
        }
    __syncthreads();
    // adjoint taps: tap' = (dt', dh', dw') with W(2 - dt', 2 - dh', 2 - dw')
    const int tp_hw = (2 - dh) * 3 + (2 - dw);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ci = ci0 + ty + 8 * i, co = co0 + tx;
        if (ci >= rows_pad || co >= cpad) continue;
        const float w0 = tile[0][tx][ty + 8 * i], w1 = tile[1][tx][ty + 8 * i], w2 = tile[2][tx][ty + 8 * i];
        const long long base = (long long)ci * 27;
#pragma unroll
        for (int dtp = 0; dtp < 3; ++dtp) {
            const int tp = dtp * 9 + tp_hw;
            const float vt = dtp == 0 ? w2 : (dtp == 1 ? w1 : w0);
            const float vf = dtp == 0 ? w0 + w1 + w2 : (dtp == 1 ? w0 + w1 : w0);
            wt[(base + tp) * cpad + co] = __float2bfloat16_rn(vt);
            wf0[(base + tp) * cpad + co] = __float2bfloat16_rn(vf);
        }
    }
}

__global__ void __launch_bounds__(256) pack3_kernel(const float* __restrict__ w, int Cout, int Cin, int Cout_pad,
                                                    int Kpad, int rows_pad, int cpad, __nv_bfloat16* __restrict__ fwd,
                                                    __nv_bfloat16* __restrict__ wt, __nv_bfloat16* __restrict__ wf0) {
    __shared__ float tile[3][32][33];
    pack3_tile(w, Cout, Cin, Cout_pad, Kpad, rows_pad, cpad, fwd, wt, wf0, blockIdx.x, blockIdx.y, blockIdx.z, tile);
}

// All the 3x3x3 convs of a network in one launch: block b belongs to the job whose
// first block is the largest block0 <= b (jobs in order of block0).
__global__ void __launch_bounds__(256) pack3_batch_kernel(const Pack3Job* __restrict__ jobs, int njobs) {
    __shared__ float tile[3][32][33];
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (jobs[mid].block0 <= (long long)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const Pack3Job& J = jobs[s_job];
    const long long lb = (long long)blockIdx.x - J.block0;
    const int bx = (int)(lb % J.gx), by = (int)((lb / J.gx) % J.gy), hw = (int)(lb / ((long long)J.gx * J.gy));
    pack3_tile(J.w, J.Cout, J.Cin, J.Cout_pad, J.Kpad, J.rows_pad, J.cpad, J.fwd, J.wt, J.wf0, bx, by, hw, tile);
}

// p -= lr * g, four floats per thread when both are 16-byte aligned (the tail and
// unaligned vectors one at a time).
__global__ void sgd_kernel(float* __restrict__ p, const float* __restrict__ g, long long n, float lr) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g)) & 15u) == 0;
    if (vec) {
        const long long i = 4 * t;
        if (i + 4 <= n) {
            float4 pv = *reinterpret_cast<const float4*>(p + i);
            const float4 gv = *reinterpret_cast<const float4*>(g + i);
            pv.x -= lr * gv.x;
            pv.y -= lr * gv.y;
            pv.z -= lr * gv.z;
            pv.w -= lr * gv.w;
            *reinterpret_cast<float4*>(p + i) = pv;
        } else {
            for (long long k = i; k < n; ++k) p[k] -= lr * g[k];
        }
    } else {
        for (long long k = 4 * t; k < 4 * t + 4 && k < n; ++k) p[k] -= lr * g[k];
    }
}

}  // namespace

// ======================================================================= host

size_t wgrad_partial_floats(int Cout, int K, int S) { return (size_t)S * Cout * K + (size_t)S * Cout; }

int wgrad_splits(const WgradArgs& a, int num_sms, size_t max_partial_floats) {
    const long long tiles = (long long)((a.Cout + WB - 1) / WB) * ((a.K + WB - 1) / WB);
    long long S = (4LL * num_sms + tiles - 1) / tiles;
    S = std::max(1LL, std::min(S, (a.V + 255) / 256));
    while (S > 1 && wgrad_partial_floats(a.Cout, a.K, (int)S) > max_partial_floats) --S;
    return (int)std::min(S, 256LL);
}

template <typename T>
int launch_wgrad(const T* dy, const T* x, WgradArgs a, int S, float* part, float* dw, float* db, cudaStream_t s) {
    if (a.V <= 0) return 0;
    a.vchunk = ((a.V + S - 1) / S + WV - 1) / WV * WV;
    float* dbpart = part + (size_t)S * a.Cout * a.K;
    dim3 grid((a.Cout + WB - 1) / WB, (a.K + WB - 1) / WB, S);
    wgrad_kernel<T><<<grid, 256, 0, s>>>(dy, x, a, part, dbpart);
    const long long n = std::max<long long>((long long)a.Cout * a.K, a.Cout);
    wgrad_reduce_kernel<<<blocks_for(n, 256), 256, 0, s>>>(part, dbpart, S, a.Cout, a.K, dw, db);
    return (int)cudaGetLastError();
}
template int launch_wgrad<float>(const float*, const float*, WgradArgs, int, float*, float*, float*, cudaStream_t);
template int launch_wgrad<__nv_bfloat16>(const __nv_bfloat16*, const __nv_bfloat16*, WgradArgs, int, float*, float*,
                                         float*, cudaStream_t);

// Scratch layout of the GN backward (float2 each): pg[frames*S*G],
// pc[frames*S*C], gstat[frames*G], q[GN_BANDS*C]; S = chunks per frame.
size_t gn_bwd_scratch_bytes(long long frames, int S, int C, int G) {
    return ((size_t)frames * S * G + (size_t)frames * S * C + (size_t)frames * G + (size_t)GN_BANDS * C) *
               sizeof(float2) +
           256;
}

int gn_bwd_vectors_per_thread() { return GN_BWD_VPT; }
int gn_bwd_chunks_per_frame(long long HW, int C, int vec) {
    const long long vpf = HW * C / vec;
    return (int)std::max<long long>(1, (vpf + (long long)NT * GN_BWD_VPT - 1) / ((long long)NT * GN_BWD_VPT));
}

// stats: (mean, rstd) per (frame, group) from the forward statistics pass;
// S chunks of NT * vpt vectors per frame (vpt <= GN_BWD_VPT).
template <typename T>
int launch_gn_silu_bwd(const T* x, const T* dy, const float2* stats, const float* gamma, const float* beta,
                       const T* add, long long frames, long long HW, int C, int G, int vpt, int S, void* scratch,
                       float* dgamma, float* dbeta, T* dx, int* status, unsigned long long wait_ns, cudaStream_t s) {
    constexpr int V = V8<T>::N;
    const int vpv = C / V;
    if (C % V || C % G || vpv > NT || (vpv & (vpv - 1)) || vpt < 1 || vpt > GN_BWD_VPT ||
        (long long)S * NT * vpt < HW * C / V)
        return (int)cudaErrorInvalidValue;
    static std::atomic<unsigned long long> done_r{0}, done_a{0};
    if (smem_attr_once(gn_bwd_reduce_kernel<T>, 2 * GN_BWD_SEGS * GN_BWD_SEG, done_r) != cudaSuccess ||
        smem_attr_once(gn_bwd_apply_kernel<T>, 3 * GN_BWD_SEGS * GN_BWD_SEG, done_a) != cudaSuccess)
        return (int)cudaGetLastError();
    GnBwdArgs<T> a;
    a.x = x;
    a.dy = dy;
    a.stats = stats;
    a.gamma = gamma;
    a.beta = beta;
    a.add = add;
    a.dx = dx;
    a.frames = frames;
    a.vpf = HW * C / V;
    a.C = C;
    a.G = G;
    a.S = S;
    a.vpt = vpt;
    a.pg = static_cast<float2*>(scratch);
    a.pc = a.pg + frames * S * G;
    a.gstat = a.pc + frames * S * C;
    a.status = status;
    a.wait_ns = wait_ns;
    float2* q = a.gstat + frames * G;
    const dim3 grid(S, (unsigned)frames);
    gn_bwd_reduce_kernel<T><<<grid, NT, 2 * GN_BWD_SEGS * GN_BWD_SEG, s>>>(a);
    gn_bwd_finalize_kernel<<<blocks_for(frames * G * 32, 256), 256, 0, s>>>(a.pg, frames, S, G,
                                                                           1.f / (float)(HW * (C / G)), a.gstat);
    gn_bwd_channel_kernel<<<dim3((C + 31) / 32, GN_BANDS), 256, 0, s>>>(a.pc, frames * S, C, q);
    gn_bwd_channel_final_kernel<<<blocks_for((long long)C * 32, 256), 256, 0, s>>>(q, C, dgamma, dbeta);
    gn_bwd_apply_kernel<T><<<grid, NT, (add ? 3 : 2) * GN_BWD_SEGS * GN_BWD_SEG, s>>>(a);
    return (int)cudaGetLastError();
}
template int launch_gn_silu_bwd<float>(const float*, const float*, const float2*, const float*, const float*,
                                       const float*, long long, long long, int, int, int, int, void*, float*, float*,
                                       float*, int*, unsigned long long, cudaStream_t);
template int launch_gn_silu_bwd<__nv_bfloat16>(const __nv_bfloat16*, const __nv_bfloat16*, const float2*,
                                               const float*, const float*, const __nv_bfloat16*, long long, long long,
                                               int, int, int, int, void*, float*, float*, __nv_bfloat16*,
                                               int*, unsigned long long, cudaStream_t);

template <typename T>
int launch_ste_bwd(const T* dcodes, int Cd, const float* z, const uint32_t* keep_bits, long long ntok, int Wq,
                   const FsqConsts& f, T* dz, int Co, cudaStream_t s) {
    if (ntok <= 0) return 0;
    ste_bwd_kernel<T><<<blocks_for(ntok, 256), 256, 0, s>>>(dcodes, Cd, z, keep_bits, ntok, Wq, f, dz, Co);
    return (int)cudaGetLastError();
}
template int launch_ste_bwd<float>(const float*, int, const float*, const uint32_t*, long long, int, const FsqConsts&,
                                   float*, int, cudaStream_t);
template int launch_ste_bwd<__nv_bfloat16>(const __nv_bfloat16*, int, const float*, const uint32_t*, long long, int,
                                           const FsqConsts&, __nv_bfloat16*, int, cudaStream_t);

template <typename T>
int launch_codes(const int32_t* idx, long long ntok, const FsqConsts& f, T* codes, cudaStream_t s) {
    if (ntok <= 0) return 0;
    codes_kernel<T><<<blocks_for(ntok, 256), 256, 0, s>>>(idx, ntok, f, codes);
    return (int)cudaGetLastError();
}
template int launch_codes<float>(const int32_t*, long long, const FsqConsts&, float*, cudaStream_t);
template int launch_codes<__nv_bfloat16>(const int32_t*, long long, const FsqConsts&, __nv_bfloat16*, cudaStream_t);

template <typename Ti, typename To>
int launch_s2d(const Ti* d, int N, int oT, int oH, int oW, int C, int rt, int rh, int rw, int drop_t, int T, int H,
               int W, int Cpad, To* out, cudaStream_t s) {
    const long long n = (long long)N * T * H * W * Cpad;
    if (n <= 0) return 0;
    if constexpr (sizeof(Ti) == 2 && sizeof(To) == 2) {
        if (C % 8 == 0 && Cpad % 8 == 0) {
            s2d_vec8_kernel<<<blocks_for(n / 8, 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(d), N, oT, oH, oW,
                                                                    C, rt, rh, rw, drop_t, T, H, W, Cpad,
                                                                    reinterpret_cast<uint4*>(out));
            return (int)cudaGetLastError();
        }
    }
    if constexpr (sizeof(Ti) == 4 && sizeof(To) == 2) {
        if (Cpad % 8 == 0) {
            s2d_head_kernel<<<blocks_for(n / Cpad, 128), 128, 0, s>>>(d, N, oT, oH, oW, C, rt, rh, rw, drop_t, T, H,
                                                                      W, Cpad, reinterpret_cast<uint4*>(out));
            return (int)cudaGetLastError();
        }
    }
    s2d_kernel<Ti, To><<<blocks_for(n, 256), 256, 0, s>>>(d, N, oT, oH, oW, C, rt, rh, rw, drop_t, T, H, W, Cpad, out);
    return (int)cudaGetLastError();
}
template int launch_s2d<float, float>(const float*, int, int, int, int, int, int, int, int, int, int, int, int, int,
                                      float*, cudaStream_t);
template int launch_s2d<float, __nv_bfloat16>(const float*, int, int, int, int, int, int, int, int, int, int, int, int,
                                              int, __nv_bfloat16*, cudaStream_t);
template int launch_s2d<__nv_bfloat16, __nv_bfloat16>(const __nv_bfloat16*, int, int, int, int, int, int, int, int,
                                                      int, int, int, int, int, __nv_bfloat16*, cudaStream_t);

template <typename T>
int launch_zero_insert(const T* dy, int N, int To, int Ho, int Wo, int C, int Tin, int Hin, int Win, int st, int sh,
                       int sw, T* out, cudaStream_t s) {
    const long long n = (long long)N * Tin * Hin * Win * C;
    if (n <= 0) return 0;
    if (sizeof(T) == 2 && C % 8 == 0) {
        zero_insert_vec8_kernel<<<blocks_for(n / 8, 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(dy), N, To, Ho,
                                                                        Wo, C, Tin, Hin, Win, st, sh, sw,
                                                                        reinterpret_cast<uint4*>(out));
        return (int)cudaGetLastError();
    }
    zero_insert_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(dy, N, To, Ho, Wo, C, Tin, Hin, Win, st, sh, sw, out);
    return (int)cudaGetLastError();
}
template int launch_zero_insert<float>(const float*, int, int, int, int, int, int, int, int, int, int, int, float*,
                                       cudaStream_t);
template int launch_zero_insert<__nv_bfloat16>(const __nv_bfloat16*, int, int, int, int, int, int, int, int, int, int,
                                               int, __nv_bfloat16*, cudaStream_t);

template <typename T>
int launch_mse(const float* xh, const T* x, long long n, float* dxh, float* loss, float* scratch, cudaStream_t s) {
    const int nb = 592;
    mse_partial_kernel<T><<<nb, 256, 0, s>>>(xh, x, n, 2.f / (float)n, dxh, scratch);
    mse_final_kernel<<<1, 32, 0, s>>>(scratch, nb, 1.f / (float)n, loss);
    return (int)cudaGetLastError();
}
template int launch_mse<float>(const float*, const float*, long long, float*, float*, float*, cudaStream_t);
template int launch_mse<__nv_bfloat16>(const float*, const __nv_bfloat16*, long long, float*, float*, float*,
                                       cudaStream_t);

template <typename T>
int launch_pack_adjoint(const float* w, int Cout, int Cin, int k, int rows_pad, int cpad, int corr, T* out,
                        cudaStream_t s) {
    const int taps_out = corr == 1 ? 2 * k * k : k * k * k;
    dim3 grid((cpad + 31) / 32, (rows_pad + 31) / 32, taps_out);
    pack_adjoint_kernel<T><<<grid, 256, 0, s>>>(w, Cout, Cin, k, rows_pad, cpad, corr, out);
    return (int)cudaGetLastError();
}
template int launch_pack_adjoint<float>(const float*, int, int, int, int, int, int, float*, cudaStream_t);
template int launch_pack_adjoint<__nv_bfloat16>(const float*, int, int, int, int, int, int, __nv_bfloat16*,
                                                cudaStream_t);

int launch_pack3(const float* w, int Cout, int Cin, int Cout_pad, int Kpad, int rows_pad, int cpad,
                 __nv_bfloat16* fwd, __nv_bfloat16* wt, __nv_bfloat16* wf0, cudaStream_t s) {
    const int cmax = std::max(Cout_pad, cpad), rmax = std::max(Cin, rows_pad);
    dim3 grid((cmax + 31) / 32, (rmax + 31) / 32, 9);
    pack3_kernel<<<grid, 256, 0, s>>>(w, Cout, Cin, Cout_pad, Kpad, rows_pad, cpad, fwd, wt, wf0);
    return (int)cudaGetLastError();
}

Pack3Job pack3_job(const float* w, int Cout, int Cin, int Cout_pad, int Kpad, int rows_pad, int cpad,
                   __nv_bfloat16* fwd, __nv_bfloat16* wt, __nv_bfloat16* wf0, long long block0) {
    Pack3Job j;
    j.w = w;
    j.fwd = fwd;
    j.wt = wt;
    j.wf0 = wf0;
    j.Cout = Cout;
    j.Cin = Cin;
    j.Cout_pad = Cout_pad;
    j.Kpad = Kpad;
    j.rows_pad = rows_pad;
    j.cpad = cpad;
    j.gx = (std::max(Cout_pad, cpad) + 31) / 32;
    j.gy = (std::max(Cin, rows_pad) + 31) / 32;
    j.block0 = block0;
    return j;
}

int launch_pack3_batch(const Pack3Job* d_jobs, int njobs, long long blocks, cudaStream_t s) {
    if (njobs <= 0 || blocks <= 0) return 0;
    pack3_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs);
    return (int)cudaGetLastError();
}

int launch_sgd(float* p, const float* g, long long n, float lr, cudaStream_t s) {
    if (n <= 0) return 0;
    sgd_kernel<<<blocks_for((n + 3) / 4, 256), 256, 0, s>>>(p, g, n, lr);
    return (int)cudaGetLastError();
}

}  // namespace tok
