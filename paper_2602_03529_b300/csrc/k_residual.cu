// Pixel residuals (Sec. 6.3, Eq. 4).
//
//   residual_mean_kernel : r = x - x_hat, averaged over each window of
//                          consecutive frames (Eq. 4) and zeroed where
//                          |r| < theta; float32 with the definition's rounding
//                          steps (differences summed in frame order, one
//                          division by the window's frame count), since the
//                          threshold decides which elements exist.
//   count / scan / scatter: the sparse form, per (sample, window) segment the
//                          nonzero elements in position order (deterministic
//                          stream compaction: per-block counts, one exclusive
//                          scan, block-local scans for the scatter).
//   apply_kernel          : receiver side, every frame of a window gets that
//                          window's residual added.
// All bandwidth-bound.
#include "common.cuh"

namespace tok {

namespace {

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename T>
__device__ __forceinline__ float to_f(T v) {
    if constexpr (sizeof(T) == 2)
        return __bfloat162float(v);
    else
        return v;
}

// one thread per (sample, window, element); E = H*W*C elements per frame
template <typename T>
__global__ void residual_mean_kernel(const T* __restrict__ x, const float* __restrict__ xh, long long N, int Tf,
                                     long long E, int window, int nwin, float theta, float* __restrict__ r) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * nwin * E) return;
    const long long e = i % E;
    const long long seg = i / E;
    const int k = (int)(seg % nwin);
    const long long n = seg / nwin;
    const int t0 = k * window, t1 = min(t0 + window, Tf);
    float s = 0.f;
    for (int t = t0; t < t1; ++t) {
        const long long o = (n * Tf + t) * E + e;
        s = __fadd_rn(s, __fsub_rn(to_f(x[o]), xh[o]));
    }
    const float v = __fdiv_rn(s, (float)(t1 - t0));
    r[i] = fabsf(v) < theta ? 0.f : v;
}

// four consecutive elements per thread (E % 4 == 0, 16-byte aligned rows): same arithmetic
template <typename T>
__global__ void residual_mean4_kernel(const T* __restrict__ x, const float* __restrict__ xh, long long N, int Tf,
                                      long long E, int window, int nwin, float theta, float* __restrict__ r) {
    const long long E4 = E / 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * nwin * E4) return;
    const long long e = (i % E4) * 4;
    const long long seg = i / E4;
    const int k = (int)(seg % nwin);
    const long long n = seg / nwin;
    const int t0 = k * window, t1 = min(t0 + window, Tf);
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int t = t0; t < t1; ++t) {
        const long long o = (n * Tf + t) * E + e;
        const float4 h = *reinterpret_cast<const float4*>(xh + o);
        float v[4];
        if constexpr (sizeof(T) == 2) {
            const uint2 q = *reinterpret_cast<const uint2*>(x + o);
            const float2 a = unpack_bf16x2(q.x), b = unpack_bf16x2(q.y);
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        } else {
            const float4 q = *reinterpret_cast<const float4*>(x + o);
            v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        }
        s[0] = __fadd_rn(s[0], __fsub_rn(v[0], h.x));
        s[1] = __fadd_rn(s[1], __fsub_rn(v[1], h.y));
        s[2] = __fadd_rn(s[2], __fsub_rn(v[2], h.z));
        s[3] = __fadd_rn(s[3], __fsub_rn(v[3], h.w));
    }
    const float cnt = (float)(t1 - t0);
    float o4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float v = __fdiv_rn(s[j], cnt);
        o4[j] = fabsf(v) < theta ? 0.f : v;
    }
    *reinterpret_cast<float4*>(r + seg * E + e) = make_float4(o4[0], o4[1], o4[2], o4[3]);
}

constexpr int CH_THREADS = 256, CH_PER = 16, CHUNK = CH_THREADS * CH_PER;

// nonzero count of every CHUNK-element chunk of every segment (16-byte loads when
// the segment is 16-byte aligned: E % 4 == 0)
__global__ void count_kernel(const float* __restrict__ r, long long E, long long chunks, long long* __restrict__ cnt) {
    __shared__ int red[CH_THREADS];
    const long long seg = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const long long base = seg * E + ch * CHUNK;
    const long long lim = min((long long)CHUNK, E - ch * CHUNK);
    int c = 0;
    if ((E & 3) == 0 && (reinterpret_cast<uintptr_t>(r) & 15u) == 0) {
        float4 v[CH_PER / 4];
#pragma unroll
        for (int j = 0; j < CH_PER / 4; ++j) {
            const long long l = ((long long)j * CH_THREADS + threadIdx.x) * 4;
            v[j] = l < lim ? *reinterpret_cast<const float4*>(r + base + l) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < CH_PER / 4; ++j)
            c += (v[j].x != 0.f) + (v[j].y != 0.f) + (v[j].z != 0.f) + (v[j].w != 0.f);
    } else {
        for (int j = 0; j < CH_PER; ++j) {
            const long long l = (long long)j * CH_THREADS + threadIdx.x;
            if (l < lim && r[base + l] != 0.f) ++c;
        }
    }
    red[threadIdx.x] = c;
    __syncthreads();
    for (int o = CH_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[blockIdx.x] = red[0];
}

// exclusive scan of cnt[0..n) in place (one block, carry across rounds); cnt[n] = total
__global__ void scan_kernel(long long* __restrict__ cnt, long long n) {
    __shared__ long long buf[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < n; b += 1024) {
        const long long i = b + threadIdx.x;
        const long long v = i < n ? cnt[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const long long add = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) cnt[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[n] = carry;
}

// position-ordered scatter of the nonzeros of every chunk: CH_PER steps of
// CH_THREADS consecutive elements (coalesced), a warp ballot for the order within
// a warp and a scan of the warps' counts for the order across the block
__global__ void scatter_kernel(const float* __restrict__ r, long long E, long long chunks,
                               const long long* __restrict__ off, int32_t* __restrict__ pos,
                               float* __restrict__ val) {
    constexpr int NW = CH_THREADS / 32;
    __shared__ int wcnt[CH_PER][NW];
    const long long seg = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const long long base = seg * E + ch * CHUNK;
    const long long lim = min((long long)CHUNK, E - ch * CHUNK);
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    float v[CH_PER];
    uint32_t bal[CH_PER];
#pragma unroll
    for (int j = 0; j < CH_PER; ++j) {
        const long long l = (long long)j * CH_THREADS + threadIdx.x;
        v[j] = l < lim ? r[base + l] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < CH_PER; ++j) {
        bal[j] = __ballot_sync(0xffffffffu, v[j] != 0.f);
        if (lane == 0) wcnt[j][warp] = __popc(bal[j]);
    }
    __syncthreads();
    // nonzeros before (step j, warp): all of steps < j, then warps < warp of step j
    long long w = off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < CH_PER; ++j) {
        int before = 0, step = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int cnt = wcnt[j][k];
            before += k < warp ? cnt : 0;
            step += cnt;
        }
        if (v[j] != 0.f) {
            const long long d = w + before + __popc(bal[j] & ((1u << lane) - 1u));
            pos[d] = (int32_t)(ch * CHUNK + (long long)j * CH_THREADS + threadIdx.x);
            val[d] = v[j];
        }
        w += step;
    }
}

__global__ void seg_offsets_kernel(const long long* __restrict__ off, long long nseg, long long chunks,
                                   int64_t* __restrict__ seg_off) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nseg) return;
    seg_off[s] = off[s * chunks];  // off[nseg * chunks] is the total
}

// one thread per stored nonzero (grid over the capacity; threads past the total exit)
__global__ void apply_kernel(float* __restrict__ xh, long long N, int Tf, long long E, int window, int nwin,
                             const int32_t* __restrict__ pos, const float* __restrict__ val,
                             const int64_t* __restrict__ seg_off, long long cap) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nseg = N * nwin;
    if (i >= cap || i >= seg_off[nseg]) return;
    long long lo = 0, hi = nseg;  // the segment s with seg_off[s] <= i < seg_off[s + 1]
    while (hi - lo > 1) {
        const long long mid = (lo + hi) / 2;
        if (seg_off[mid] <= i) lo = mid;
        else hi = mid;
    }
    const long long n = lo / nwin;
    const int k = (int)(lo % nwin);
    const int t0 = k * window, t1 = min(t0 + window, Tf);
    const float v = val[i];
    float* const p0 = xh + (n * Tf + t0) * E + pos[i];
    // the window's frames are E apart (distinct elements): read them all, then write
    constexpr int MAXW = 8;
    if (t1 - t0 <= MAXW) {
        float a[MAXW];
#pragma unroll
        for (int t = 0; t < MAXW; ++t)
            if (t < t1 - t0) a[t] = p0[(long long)t * E];
#pragma unroll
        for (int t = 0; t < MAXW; ++t)
            if (t < t1 - t0) p0[(long long)t * E] = __fadd_rn(a[t], v);
    } else {
        for (int t = 0; t < t1 - t0; ++t) p0[(long long)t * E] = __fadd_rn(p0[(long long)t * E], v);
    }
}

}  // namespace

int launch_residual_mean(bool bf16, const void* x, const float* xh, long long N, int Tf, long long E, int window,
                         float theta, float* r, cudaStream_t s) {
    const int nwin = (Tf + window - 1) / window;
    const long long n = N * nwin * E;
    if (n <= 0) return 0;
    const bool vec = E % 4 == 0 && ((uintptr_t)x % 16) == 0 && ((uintptr_t)xh % 16) == 0 && ((uintptr_t)r % 16) == 0;
    if (vec) {
        const long long n4 = n / 4;
        if (bf16)
            residual_mean4_kernel<__nv_bfloat16><<<blocks_for(n4, 256), 256, 0, s>>>(
                static_cast<const __nv_bfloat16*>(x), xh, N, Tf, E, window, nwin, theta, r);
        else
            residual_mean4_kernel<float><<<blocks_for(n4, 256), 256, 0, s>>>(static_cast<const float*>(x), xh, N,
                                                                              Tf, E, window, nwin, theta, r);
        return (int)cudaGetLastError();
    }
    if (bf16)
        residual_mean_kernel<__nv_bfloat16><<<blocks_for(n, 256), 256, 0, s>>>(
            static_cast<const __nv_bfloat16*>(x), xh, N, Tf, E, window, nwin, theta, r);
    else
        residual_mean_kernel<float><<<blocks_for(n, 256), 256, 0, s>>>(static_cast<const float*>(x), xh, N, Tf, E,
                                                                        window, nwin, theta, r);
    return (int)cudaGetLastError();
}

size_t residual_sparse_workspace_bytes(long long nseg, long long E) {
    const long long chunks = (E + CHUNK - 1) / CHUNK;
    return (size_t)(nseg * chunks + 1) * sizeof(long long) + 256;
}

int launch_residual_sparse(const float* r, long long nseg, long long E, int32_t* pos, float* val, int64_t* seg_off,
                           void* ws, cudaStream_t s) {
    if (nseg <= 0 || E <= 0) return 0;
    const long long chunks = (E + CHUNK - 1) / CHUNK;
    long long* cnt = static_cast<long long*>(ws);
    count_kernel<<<(unsigned)(nseg * chunks), CH_THREADS, 0, s>>>(r, E, chunks, cnt);
    scan_kernel<<<1, 1024, 0, s>>>(cnt, nseg * chunks);
    scatter_kernel<<<(unsigned)(nseg * chunks), CH_THREADS, 0, s>>>(r, E, chunks, cnt, pos, val);
    seg_offsets_kernel<<<blocks_for(nseg + 1, 256), 256, 0, s>>>(cnt, nseg, chunks, seg_off);
    return (int)cudaGetLastError();
}

int launch_residual_apply(float* xh, long long N, int Tf, long long E, int window, const int32_t* pos,
                          const float* val, const int64_t* seg_off, long long cap, cudaStream_t s) {
    if (cap <= 0) return 0;
    const int nwin = (Tf + window - 1) / window;
    apply_kernel<<<blocks_for(cap, 256), 256, 0, s>>>(xh, N, Tf, E, window, nwin, pos, val, seg_off, cap);
    return (int)cudaGetLastError();
}

}  // namespace tok
