// GoP boundary smoothing (Sec. 6.1): blending of the first n frames of a GoP
// with the last n of the previous one (Eq. 2) and the boundary loss with its
// gradient (Eq. 1). All bandwidth-bound; the loss reduction is deterministic
// (fixed chunks, fixed-order sums).
#include "common.cuh"

namespace tok {

namespace {

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// out[s, t] = a * prev[s, Tp - n + t] + (1 - a) * curr[s, t], a = (n - 1 - t) / n, for t < n;
// out[s, t] = curr[s, t] otherwise. Four elements per thread (E % 4 == 0).
__global__ void gop_blend_kernel(const float4* __restrict__ prev, const float4* __restrict__ curr,
                                 float4* __restrict__ out, long long N, int Tp, int T, long long E4, int n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * T * E4) return;
    const long long e = i % E4;
    const int t = (int)((i / E4) % T);
    const long long s = i / (E4 * T);
    float4 c = curr[i];
    if (t < n) {
        // explicitly rounded, as the blend fused into the pixel head's epilogue
        const float a = __fdiv_rn((float)(n - 1 - t), (float)n), b = __fsub_rn(1.f, a);
        const float4 p = prev[(s * Tp + (Tp - n + t)) * E4 + e];
        c = make_float4(__fmaf_rn(a, p.x, __fmul_rn(b, c.x)), __fmaf_rn(a, p.y, __fmul_rn(b, c.y)),
                        __fmaf_rn(a, p.z, __fmul_rn(b, c.z)), __fmaf_rn(a, p.w, __fmul_rn(b, c.w)));
    }
    out[i] = c;
}

__global__ void gop_blend1_kernel(const float* __restrict__ prev, const float* __restrict__ curr,
                                  float* __restrict__ out, long long N, int Tp, int T, long long E, int n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * T * E) return;
    const long long e = i % E;
    const int t = (int)((i / E) % T);
    const long long s = i / (E * T);
    float c = curr[i];
    if (t < n) {
        const float a = __fdiv_rn((float)(n - 1 - t), (float)n);
        c = __fmaf_rn(a, prev[(s * Tp + (Tp - n + t)) * E + e], __fmul_rn(__fsub_rn(1.f, a), c));
    }
    out[i] = c;
}

constexpr int LT = 256, LPER = 16, LCHUNK = LT * LPER;

// partial sums of squared differences per (sample, boundary frame, chunk)
__global__ void tloss_partial_kernel(const float* __restrict__ xc, const float* __restrict__ xp, int Tc, int Tp,
                                     long long E, int n, long long chunks, double* __restrict__ part) {
    __shared__ double red[LT];
    const long long blk = blockIdx.x;
    const long long ch = blk % chunks;
    const int i = (int)((blk / chunks) % n);
    const long long s = blk / (chunks * n);
    const float* a = xc + (s * Tc + i) * E;
    const float* b = xp + (s * Tp + (Tp - n + i)) * E;
    float acc = 0.f;  // 16 squares in float32, then FP64 across the block
    if ((E & 3) == 0 && ((reinterpret_cast<uintptr_t>(xc) | reinterpret_cast<uintptr_t>(xp)) & 15u) == 0) {
        // four float4 per thread, all requested before use (thread covers 4 runs of 4)
        float4 va[LPER / 4], vb[LPER / 4];
#pragma unroll
        for (int j = 0; j < LPER / 4; ++j) {
            const long long e = ch * LCHUNK + ((long long)j * LT + threadIdx.x) * 4;
            va[j] = e < E ? *reinterpret_cast<const float4*>(a + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            vb[j] = e < E ? *reinterpret_cast<const float4*>(b + e) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < LPER / 4; ++j) {
            const float d0 = va[j].x - vb[j].x, d1 = va[j].y - vb[j].y, d2 = va[j].z - vb[j].z,
                        d3 = va[j].w - vb[j].w;
            acc = fmaf(d0, d0, acc);
            acc = fmaf(d1, d1, acc);
            acc = fmaf(d2, d2, acc);
            acc = fmaf(d3, d3, acc);
        }
    } else {
        for (int j = 0; j < LPER; ++j) {
            const long long e = ch * LCHUNK + (long long)j * LT + threadIdx.x;
            if (e < E) {
                const float d = a[e] - b[e];
                acc = fmaf(d, d, acc);
            }
        }
    }
    red[threadIdx.x] = (double)acc;
    __syncthreads();
    for (int o = LT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blk] = red[0];
}

// norms of the N*n boundary differences (a warp per difference, lanes over chunks, fixed
// shuffle tree), the gradient scales 1/(N n ||d||), and the loss (one warp, fixed order)
__global__ void tloss_norm_kernel(const double* __restrict__ part, long long pairs, long long chunks, long long Nn,
                                  float* __restrict__ scale, double* __restrict__ norms) {
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (q >= pairs) return;
    double ss = 0.0;
    for (long long c = lane; c < chunks; c += 32) ss += part[q * chunks + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if (lane == 0) {
        const double nrm = sqrt(ss);
        norms[q] = nrm;
        scale[q] = nrm > 0.0 ? (float)(1.0 / ((double)Nn * nrm)) : 0.f;
    }
}

__global__ void tloss_sum_kernel(const double* __restrict__ norms, long long pairs, long long Nn,
                                 float* __restrict__ loss) {
    const int lane = threadIdx.x;
    double acc = 0.0;
    for (long long q = lane; q < pairs; q += 32) acc += norms[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) *loss = (float)(acc / (double)Nn);
}

// the same, four elements per thread (E % 4 == 0, 16-byte aligned frames)
__global__ void tloss_grad4_kernel(const float4* __restrict__ xc, const float4* __restrict__ xp, int Tc, int Tp,
                                   long long E4, int n, long long N, const float* __restrict__ scale,
                                   float4* __restrict__ g) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N * Tc * E4) return;
    const long long e = k % E4;
    const int t = (int)((k / E4) % Tc);
    const long long s = k / (E4 * Tc);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < n) {
        const float4 c = xc[k], p = xp[(s * Tp + (Tp - n + t)) * E4 + e];
        const float sc = scale[s * n + t];
        v = make_float4((c.x - p.x) * sc, (c.y - p.y) * sc, (c.z - p.z) * sc, (c.w - p.w) * sc);
    }
    g[k] = v;
}

__global__ void tloss_grad_kernel(const float* __restrict__ xc, const float* __restrict__ xp, int Tc, int Tp,
                                  long long E, int n, long long N, const float* __restrict__ scale,
                                  float* __restrict__ g) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N * Tc * E) return;
    const long long e = k % E;
    const int t = (int)((k / E) % Tc);
    const long long s = k / (E * Tc);
    float v = 0.f;
    if (t < n) v = (xc[k] - xp[(s * Tp + (Tp - n + t)) * E + e]) * scale[s * n + t];
    g[k] = v;
}

}  // namespace

int launch_gop_blend(const float* prev, int Tp, const float* curr, float* out, long long N, int T, long long E, int n,
                     cudaStream_t s) {
    const long long total = N * T * E;
    if (total <= 0) return 0;
    const bool vec = E % 4 == 0 && ((uintptr_t)prev % 16) == 0 && ((uintptr_t)curr % 16) == 0 &&
                     ((uintptr_t)out % 16) == 0;
    if (vec)
        gop_blend_kernel<<<blocks_for(total / 4, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(prev),
                                                                    reinterpret_cast<const float4*>(curr),
                                                                    reinterpret_cast<float4*>(out), N, Tp, T, E / 4,
                                                                    n);
    else
        gop_blend1_kernel<<<blocks_for(total, 256), 256, 0, s>>>(prev, curr, out, N, Tp, T, E, n);
    return (int)cudaGetLastError();
}

size_t temporal_loss_workspace_bytes(long long N, int n, long long E) {
    const long long chunks = (E + LCHUNK - 1) / LCHUNK;
    return (size_t)(N * n * chunks) * sizeof(double) + (size_t)(N * n) * (sizeof(double) + sizeof(float)) + 512;
}

int launch_temporal_loss(const float* xc, const float* xp, long long N, int Tc, int Tp, long long E, int n,
                         float* loss, float* grad, void* ws, cudaStream_t s) {
    if (N <= 0 || n <= 0 || E <= 0) return 0;
    const long long chunks = (E + LCHUNK - 1) / LCHUNK;
    double* part = static_cast<double*>(ws);
    double* norms = part + N * n * chunks;
    float* scale = reinterpret_cast<float*>(norms + N * n);
    tloss_partial_kernel<<<(unsigned)(N * n * chunks), LT, 0, s>>>(xc, xp, Tc, Tp, E, n, chunks, part);
    tloss_norm_kernel<<<blocks_for(N * n * 32, 256), 256, 0, s>>>(part, N * n, chunks, N * n, scale, norms);
    tloss_sum_kernel<<<1, 32, 0, s>>>(norms, N * n, N * n, loss);
    const bool vec4 = E % 4 == 0 && ((reinterpret_cast<uintptr_t>(xc) | reinterpret_cast<uintptr_t>(xp) |
                                      reinterpret_cast<uintptr_t>(grad)) & 15u) == 0;
    if (grad && vec4)
        tloss_grad4_kernel<<<blocks_for(N * Tc * E / 4, 256), 256, 0, s>>>(
            reinterpret_cast<const float4*>(xc), reinterpret_cast<const float4*>(xp), Tc, Tp, E / 4, n, N, scale,
            reinterpret_cast<float4*>(grad));
    else if (grad)
        tloss_grad_kernel<<<blocks_for(N * Tc * E, 256), 256, 0, s>>>(xc, xp, Tc, Tp, E, n, N, scale, grad);
    return (int)cudaGetLastError();
}

}  // namespace tok
