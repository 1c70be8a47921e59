// Gather kernels feeding the tensor-core convolution where the input has too
// few channels for 64-channel K blocks: the pixel stem (3 channels) and the
// decoder input (the nlev FSQ code channels, dequantised on the fly). Each
// builds the im2col matrix A (M x Kpad, BF16) of one causal conv, with
// K = (tap, ci), zero columns up to Kpad, the time-causal pad (history frames,
// replicate or zero), zero spatial pad, and, for pixels, edge extension of the
// frame from H x W to the padded Hp x Wp. Also the edge pad used by the FP32
// path. All bandwidth-bound; one thread writes 8 consecutive K entries.
#include "common.cuh"
#include "conv_args.h"

namespace tok {

namespace {

// Source location of (output voxel, tap) or -1 for a zero tap.
// Returns (frame index into `x` or into `hist` (flag), h, w).
__device__ __forceinline__ bool gather_src(const GatherGeo& g, int n, int to, int ho, int wo, int tap,
                                           bool* from_hist, long long* frame, int* hi, int* wi) {
    const int dw = tap % g.kw, dh = (tap / g.kw) % g.kh, dt = tap / (g.kw * g.kh);
    int h = ho * g.sh + dh - (g.kh - 1) / 2;
    int w = wo * g.sw + dw - (g.kw - 1) / 2;
    if (h < 0 || h >= g.Hp || w < 0 || w >= g.Wp) return false;
    *hi = h < g.H ? h : g.H - 1;  // edge extension of the padded frame
    *wi = w < g.W ? w : g.W - 1;
    const int ti = to * g.st + dt + g.t_off;
    *from_hist = false;
    if (ti >= 0) {
        *frame = (long long)n * g.Tin + ti;
    } else if (g.hist_T > 0) {
        *from_hist = true;
        *frame = (long long)n * g.hist_T + g.hist_T + ti;
    } else if (g.pad_mode == 0) {
        *frame = (long long)n * g.Tin;
    } else {
        return false;
    }
    return true;
}

__global__ void im2col_pixels_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ hist,
                                     GatherGeo g, __nv_bfloat16* __restrict__ A) {
    const long long M = (long long)g.N * g.Tout * g.Hout * g.Wout;
    const int kg = g.Kpad / 8;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * kg) return;
    const long long m = t / kg;
    const int k0 = (int)(t % kg) * 8;
    long long mm = m;
    const int wo = (int)(mm % g.Wout); mm /= g.Wout;
    const int ho = (int)(mm % g.Hout); mm /= g.Hout;
    const int to = (int)(mm % g.Tout);
    const int n = (int)(mm / g.Tout);
    const int K = g.kt * g.kh * g.kw * g.Cin;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        v[e] = 0.f;
        const int k = k0 + e;
        if (k < K) {
            bool fh;
            long long fr;
            int hi, wi;
            if (gather_src(g, n, to, ho, wo, k / g.Cin, &fh, &fr, &hi, &wi)) {
                const __nv_bfloat16* src = fh ? hist : x;
                v[e] = __bfloat162float(src[((fr * g.H + hi) * g.W + wi) * g.Cin + (k % g.Cin)]);
            }
        }
    }
    uint4 o;
    o.x = pack_bf16x2(v[0], v[1]);
    o.y = pack_bf16x2(v[2], v[3]);
    o.z = pack_bf16x2(v[4], v[5]);
    o.w = pack_bf16x2(v[6], v[7]);
    reinterpret_cast<uint4*>(A)[t] = o;
}

__device__ __forceinline__ float code_of(int id, const FsqConsts& f, int i) {
    const int d = (id / f.basis[i]) % f.levels[i];
    return (float)(d - f.half_w[i]) / (float)f.half_w[i];
}

__global__ void im2col_tokens_kernel(const int32_t* __restrict__ idx, const int32_t* __restrict__ hist, GatherGeo g,
                                     FsqConsts f, __nv_bfloat16* __restrict__ A) {
    const long long M = (long long)g.N * g.Tout * g.Hout * g.Wout;
    const int kg = g.Kpad / 8;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * kg) return;
    const long long m = t / kg;
    const int k0 = (int)(t % kg) * 8;
    long long mm = m;
    const int wo = (int)(mm % g.Wout); mm /= g.Wout;
    const int ho = (int)(mm % g.Hout); mm /= g.Hout;
    const int to = (int)(mm % g.Tout);
    const int n = (int)(mm / g.Tout);
    const int K = g.kt * g.kh * g.kw * g.Cin;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        v[e] = 0.f;
        const int k = k0 + e;
        if (k < K) {
            bool fh;
            long long fr;
            int hi, wi;
            if (gather_src(g, n, to, ho, wo, k / g.Cin, &fh, &fr, &hi, &wi)) {
                const int32_t* src = fh ? hist : idx;
                v[e] = code_of(src[(fr * g.H + hi) * g.W + wi], f, k % g.Cin);
            }
        }
    }
    uint4 o;
    o.x = pack_bf16x2(v[0], v[1]);
    o.y = pack_bf16x2(v[2], v[3]);
    o.z = pack_bf16x2(v[4], v[5]);
    o.w = pack_bf16x2(v[6], v[7]);
    reinterpret_cast<uint4*>(A)[t] = o;
}

// Row-per-thread form of the pixel gather for the stem's shape (3x3x3 taps,
// CIN channels, KQ 16-byte groups per row): each thread resolves a tap's
// source once and emits its CIN values in order, so the register buffer
// indices are compile-time; the block stages its rows in shared memory and
// writes them out as contiguous 16-byte stores.
constexpr int ROWS_PER_BLOCK = 128;

template <int CIN, int KQ>
__global__ void __launch_bounds__(ROWS_PER_BLOCK) im2col_rows_kernel(const __nv_bfloat16* __restrict__ src,
                                                                     const __nv_bfloat16* __restrict__ hist,
                                                                     GatherGeo g, __nv_bfloat16* __restrict__ A) {
    __shared__ uint4 stage[ROWS_PER_BLOCK][KQ + 1];
    const long long M = (long long)g.N * g.Tout * g.Hout * g.Wout;
    const long long m0 = (long long)blockIdx.x * ROWS_PER_BLOCK;
    const long long m = m0 + threadIdx.x;
    if (m < M) {
        long long mm = m;
        const int wo = (int)(mm % g.Wout); mm /= g.Wout;
        const int ho = (int)(mm % g.Hout); mm /= g.Hout;
        const int to = (int)(mm % g.Tout);
        const int n = (int)(mm / g.Tout);
        float buf[KQ * 8];
#pragma unroll
        for (int tap = 0; tap < 27; ++tap) {
            bool fh;
            long long fr;
            int hi, wi;
            const bool ok = gather_src(g, n, to, ho, wo, tap, &fh, &fr, &hi, &wi);
            const long long pix = ok ? (fr * g.H + hi) * g.W + wi : 0;
            const __nv_bfloat16* s16 = fh ? hist : src;
#pragma unroll
            for (int c = 0; c < CIN; ++c) buf[tap * CIN + c] = ok ? __bfloat162float(s16[pix * CIN + c]) : 0.f;
        }
#pragma unroll
        for (int k = 27 * CIN; k < KQ * 8; ++k) buf[k] = 0.f;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
            uint4 o;
            o.x = pack_bf16x2(buf[8 * q + 0], buf[8 * q + 1]);
            o.y = pack_bf16x2(buf[8 * q + 2], buf[8 * q + 3]);
            o.z = pack_bf16x2(buf[8 * q + 4], buf[8 * q + 5]);
            o.w = pack_bf16x2(buf[8 * q + 6], buf[8 * q + 7]);
            stage[threadIdx.x][q] = o;
        }
    }
    __syncthreads();
    uint4* out = reinterpret_cast<uint4*>(A) + m0 * KQ;
    const long long rows = M - m0 < ROWS_PER_BLOCK ? M - m0 : ROWS_PER_BLOCK;
    for (int i = threadIdx.x; i < rows * KQ; i += ROWS_PER_BLOCK) out[i] = stage[i / KQ][i % KQ];
}

// The stem's pixel gather (3x3x3 taps, 3 channels, stride 2 in h and w, Kpad
// = 128): a block forms the im2col rows of STEM_VOX consecutive output voxels
// of one output row. It first stages the input it reads -- 3 frames x 3 rows
// x (2 * STEM_VOX + 1) pixels, with the causal time padding, the edge
// extension of the frame and zero padding applied -- in shared memory with
// coalesced loads; then thread t forms the 16-byte chunk t % 16 (K = 8q ..
// 8q+7, its 8 shared-memory offsets fixed per thread) of successive rows, so
// every warp stores 512 contiguous bytes.
constexpr int STEM_VOX = 128;
constexpr int STEM_PX = 2 * STEM_VOX + 1;  // input pixels of a row segment

__global__ void __launch_bounds__(128) im2col_stem_kernel(const __nv_bfloat16* __restrict__ x,
                                                          const __nv_bfloat16* __restrict__ hist, GatherGeo g,
                                                          __nv_bfloat16* __restrict__ A) {
    __shared__ __nv_bfloat16 tile[9 * STEM_PX * 3];
    const int wo0 = blockIdx.x * STEM_VOX, ho = blockIdx.y;
    const int nto = blockIdx.z;  // n * Tout + to
    const int n = nto / g.Tout, to = nto - n * g.Tout;
    const int tid = threadIdx.x;
    // 1. stage the input: row r = dt * 3 + dh, pixel p <-> w = 2 * wo0 - 1 + p. Per row, the
    //    source frame (or none) is decided once; the loads go out in batches of 8 per thread.
    const uint16_t* rsrc[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int dt = r / 3, dh = r - dt * 3;
        const int h = ho * g.sh + dh - 1, ti = to * g.st + dt + g.t_off;
        const __nv_bfloat16* src = nullptr;
        long long fr = 0;
        if (h >= 0 && h < g.Hp) {
            if (ti >= 0) {
                src = x;
                fr = (long long)n * g.Tin + ti;
            } else if (g.hist_T > 0) {
                src = hist;
                fr = (long long)n * g.hist_T + g.hist_T + ti;
            } else if (g.pad_mode == 0) {
                src = x;
                fr = (long long)n * g.Tin;
            }
        }
        const int hi = h < g.H ? h : g.H - 1;
        rsrc[r] = src ? reinterpret_cast<const uint16_t*>(src) + (fr * g.H + hi) * g.W * 3 : nullptr;
    }
    // Each row segment: the pixels inside the frame, [p_lo, p_hi), are copied as they lie in
    // memory; pixels left of the frame are zero, those right of it repeat the last column
    // (edge extension) up to the padded width and are zero beyond.
    uint16_t* t16w = reinterpret_cast<uint16_t*>(tile);
    const int w_first = wo0 * g.sw - 1;
    const int p_lo = max(0, -w_first);
    const int p_hi = max(p_lo, min(STEM_PX, g.W - w_first));
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        uint16_t* dst = t16w + r * STEM_PX * 3;
        const uint16_t* rs = rsrc[r];
        if (!rs) {
            for (int e = tid; e < STEM_PX * 3; e += blockDim.x) dst[e] = 0;
            continue;
        }
        // all of a thread's loads of the row in flight at once (a row is 3 * STEM_PX elements)
        const uint16_t* src = rs + (long long)w_first * 3;
        constexpr int RB = (3 * STEM_PX + 127) / 128;
        uint16_t v[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int e = 3 * p_lo + u * 128 + tid;
            v[u] = e < 3 * p_hi ? __ldg(src + e) : (uint16_t)0;
        }
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int e = 3 * p_lo + u * 128 + tid;
            if (e < 3 * p_hi) dst[e] = v[u];
        }
        for (int e = tid; e < 3 * p_lo; e += blockDim.x) dst[e] = 0;
        for (int e = 3 * p_hi + tid; e < 3 * STEM_PX; e += blockDim.x) {
            const int px = e / 3, c = e - px * 3;
            dst[e] = (w_first + px < g.Wp) ? __ldg(rs + (long long)(g.W - 1) * 3 + c) : (uint16_t)0;
        }
    }
    __syncthreads();
    // 2. rows: thread t forms chunk q = t % 16 (K = 8q + j, j < 8) of voxels v = t / 16 + 8 i
    const int q = tid & 15;
    int off[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = 8 * q + j;
        if (k < 81) {
            const int tap = k / 3, c = k - tap * 3;
            const int dt = tap / 9, dh = (tap / 3) % 3, dw = tap % 3;
            off[j] = ((dt * 3 + dh) * STEM_PX + dw) * 3 + c;
        } else {
            off[j] = -1;
        }
    }
    const long long m0 = ((long long)nto * g.Hout + ho) * g.Wout + wo0;
    const int nv = min(STEM_VOX, g.Wout - wo0);
    const uint16_t* t16 = reinterpret_cast<const uint16_t*>(tile);
    uint4* out = reinterpret_cast<uint4*>(A);
    for (int v = tid >> 4; v < nv; v += blockDim.x >> 4) {
        uint32_t u[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) u[j] = off[j] >= 0 ? t16[off[j] + 6 * v] : 0u;
        out[(m0 + v) * 16 + q] = make_uint4(u[0] | (u[1] << 16), u[2] | (u[3] << 16), u[4] | (u[5] << 16),
                                            u[6] | (u[7] << 16));
    }
}

template <typename T>
__global__ void edge_pad_kernel(const T* __restrict__ x, long long frames, int H, int W, int Hp, int Wp, int C,
                                T* __restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = frames * Hp * Wp * C;
    if (t >= total) return;
    long long r = t;
    const int c = (int)(r % C); r /= C;
    const int w = (int)(r % Wp); r /= Wp;
    const int h = (int)(r % Hp);
    const long long f = r / Hp;
    const int hi = h < H ? h : H - 1, wi = w < W ? w : W - 1;
    y[t] = x[((f * H + hi) * W + wi) * C + c];
}

template <typename T>
__global__ void pack_weights_kernel(const float* __restrict__ w, int Cout, int K, int Cout_pad, int Kpad,
                                    T* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)Cout_pad * Kpad) return;
    const int co = (int)(t / Kpad), k = (int)(t % Kpad);
    const float v = (co < Cout && k < K) ? w[(long long)co * K + k] : 0.f;
    if constexpr (sizeof(T) == 2)
        out[t] = __float2bfloat16_rn(v);
    else
        out[t] = v;
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

static bool taps27(const GatherGeo& g) { return g.kt == 3 && g.kh == 3 && g.kw == 3; }

int launch_im2col_pixels(const __nv_bfloat16* x, const __nv_bfloat16* hist, const GatherGeo& g, __nv_bfloat16* A,
                         cudaStream_t s) {
    const long long M = (long long)g.N * g.Tout * g.Hout * g.Wout;
    if (M <= 0) return 0;
    if (taps27(g) && g.Cin == 3 && g.Kpad == 128 && g.sh == 2 && g.sw == 2 && g.N * g.Tout <= 65535 &&
        g.Hout <= 65535) {
        const dim3 grid((unsigned)((g.Wout + STEM_VOX - 1) / STEM_VOX), (unsigned)g.Hout, (unsigned)(g.N * g.Tout));
        im2col_stem_kernel<<<grid, 128, 0, s>>>(x, hist, g, A);
    } else if (taps27(g) && g.Cin == 3 && g.Kpad == 128) {
        im2col_rows_kernel<3, 16><<<blocks_for(M, ROWS_PER_BLOCK), ROWS_PER_BLOCK, 0, s>>>(x, hist, g, A);
    } else {
        im2col_pixels_kernel<<<blocks_for(M * (g.Kpad / 8), 256), 256, 0, s>>>(x, hist, g, A);
    }
    return (int)cudaGetLastError();
}

int launch_im2col_tokens(const int32_t* idx, const int32_t* hist, const GatherGeo& g, const FsqConsts& f,
                         __nv_bfloat16* A, cudaStream_t s) {
    const long long M = (long long)g.N * g.Tout * g.Hout * g.Wout;
    if (M <= 0) return 0;
    im2col_tokens_kernel<<<blocks_for(M * (g.Kpad / 8), 256), 256, 0, s>>>(idx, hist, g, f, A);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_edge_pad(const T* x, long long frames, int H, int W, int Hp, int Wp, int C, T* y, cudaStream_t s) {
    const long long n = frames * Hp * Wp * C;
    if (n <= 0) return 0;
    edge_pad_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(x, frames, H, W, Hp, Wp, C, y);
    return (int)cudaGetLastError();
}
template int launch_edge_pad<float>(const float*, long long, int, int, int, int, int, float*, cudaStream_t);
template int launch_edge_pad<int32_t>(const int32_t*, long long, int, int, int, int, int, int32_t*, cudaStream_t);

namespace {
__global__ void fill_i32_kernel(int32_t* p, long long n, int32_t v) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = v;
}
}  // namespace

int launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t s) {
    if (n <= 0) return 0;
    fill_i32_kernel<<<blocks_for(n, 256), 256, 0, s>>>(p, n, v);
    return (int)cudaGetLastError();
}

// Weights of a narrow 3x3x3 head for the forms in which spatial taps are MMA
// rows (W[co][dt][dh][dw][ci]; rows_out rows, the unused ones zero):
//   tr = 3 (at most 16 channels): out[dw * 16 + co][(dt * 3 + dh) * Cin + ci], K = 9 Cin;
//   tr = 9 (9 * Cout <= 128):     out[(dh * 3 + dw) * Cout + co][dt * Cin + ci], K = 3 Cin.
__global__ void pack_weights_taprows_kernel(const float* __restrict__ w, int Cout, int Cin, int rows_out, int tr,
                                            __nv_bfloat16* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long K = (tr == 9 ? 3LL : 9LL) * Cin;
    if (t >= (long long)rows_out * K) return;
    const int r = (int)(t / K);
    const long long k = t - (long long)r * K;
    const int ci = (int)(k % Cin), kk = (int)(k / Cin);  // kk: dt * 3 + dh (tr = 3) or dt (tr = 9)
    float v = 0.f;
    if (tr == 9) {
        const int tap = r / Cout, co = r - tap * Cout;  // tap = dh * 3 + dw
        if (tap < 9) v = w[((long long)co * 27 + kk * 9 + tap) * Cin + ci];
    } else {
        const int dw = r / 16, co = r - dw * 16;
        if (dw < 3 && co < Cout) v = w[((long long)co * 27 + kk * 3 + dw) * Cin + ci];
    }
    out[t] = __float2bfloat16_rn(v);
}

int launch_pack_weights_taprows(const float* w, int Cout, int Cin, int rows_out, int tr, __nv_bfloat16* out,
                                cudaStream_t s) {
    if (tr != 3 && tr != 9) return (int)cudaErrorInvalidValue;
    const long long n = (long long)rows_out * (tr == 9 ? 3 : 9) * Cin;
    if (n <= 0) return 0;
    pack_weights_taprows_kernel<<<blocks_for(n, 256), 256, 0, s>>>(w, Cout, Cin, rows_out, tr, out);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_pack_weights(const float* w, int Cout, int K, int Cout_pad, int Kpad, T* out, cudaStream_t s) {
    const long long n = (long long)Cout_pad * Kpad;
    if (n <= 0) return 0;
    pack_weights_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(w, Cout, K, Cout_pad, Kpad, out);
    return (int)cudaGetLastError();
}
template int launch_pack_weights<float>(const float*, int, int, int, int, float*, cudaStream_t);
template int launch_pack_weights<__nv_bfloat16>(const float*, int, int, int, int, __nv_bfloat16*, cudaStream_t);

}  // namespace tok
