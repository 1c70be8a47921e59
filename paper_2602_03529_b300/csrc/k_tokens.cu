// Token-level kernels: FSQ quantise / dequantise, Philox-4x32-10 packet-drop
// masking with zero fill, and the row packetisation of the token matrix.
//
// FSQ (finite scalar quantisation, Mentzer et al. 2023) turns each latent
// vector into one integer token (the token matrix the codec transmits,
// Sec. 4.3 / Sec. 6.2). Dropped tokens and lost rows are filled with the
// zero-code index (Sec. 6.2 zero fill; random drop in training, Appendix A.2).
// All kernels are HBM- or launch-bound; one token per thread, coalesced.
#include "common.cuh"
#include "conv_args.h"

namespace tok {

namespace {

// ------------------------------------------------------------------ FSQ

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// The digit of each channel is the number of its rounding thresholds that z passes
// (see FsqThr); TMAX thresholds per channel are compared (7 when no channel has more
// than 8 levels), read from the parameter bank.
template <int TMAX>
__global__ void fsq_kernel(const float* __restrict__ z, long long ntok, FsqConsts f, const __grid_constant__ FsqThr th,
                           int32_t* __restrict__ idx, float* __restrict__ codes) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    const float* zp = z + t * f.nlev;
    int id = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < f.nlev) {
            const int d = fsq_digit<TMAX>(th, i, zp[i]);
            id += d * f.basis[i];
            if (codes) codes[t * f.nlev + i] = (float)(d - f.half_w[i]) / (float)f.half_w[i];
        }
    }
    idx[t] = id;
}

// Four tokens per thread: their 4 * NL channels are NL aligned 16-byte vectors, the
// four indices one 16-byte store (the caller checks the alignment); the last, partial
// group of tokens goes element by element.
template <int TMAX, int NL>
__global__ void fsq4_kernel(const float* __restrict__ z, long long ntok, FsqConsts f, const __grid_constant__ FsqThr th,
                            int32_t* __restrict__ idx, float* __restrict__ codes) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long t0 = g * 4;
    if (t0 >= ntok) return;
    const bool whole = t0 + 4 <= ntok;
    float v[4 * NL];
    if (whole) {
        const float4* zp = reinterpret_cast<const float4*>(z + t0 * NL);
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            const float4 q = zp[i];
            v[4 * i] = q.x;
            v[4 * i + 1] = q.y;
            v[4 * i + 2] = q.z;
            v[4 * i + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4 * NL; ++i) v[i] = t0 * NL + i < ntok * NL ? z[t0 * NL + i] : 0.f;
    }
    int id[4];
    int dg[4 * NL];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int s = 0;
#pragma unroll
        for (int c = 0; c < NL; ++c) {
            dg[k * NL + c] = fsq_digit<TMAX>(th, c, v[k * NL + c]);
            s += dg[k * NL + c] * f.basis[c];
        }
        id[k] = s;
    }
    if (codes) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int c = 0; c < NL; ++c) v[k * NL + c] = (float)(dg[k * NL + c] - f.half_w[c]) / (float)f.half_w[c];
    }
    if (whole) {
        *reinterpret_cast<int4*>(idx + t0) = make_int4(id[0], id[1], id[2], id[3]);
        if (codes) {
            float4* cp = reinterpret_cast<float4*>(codes + t0 * NL);
#pragma unroll
            for (int i = 0; i < NL; ++i) cp[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t0 + k < ntok) {
                idx[t0 + k] = id[k];
                if (codes)
#pragma unroll
                    for (int c = 0; c < NL; ++c) codes[(t0 + k) * NL + c] = v[k * NL + c];
            }
    }
}

template <int TMAX, int NL>
void launch_fsq4(const float* z, long long ntok, const FsqConsts& f, const FsqThr& th, int32_t* idx, float* codes,
                 cudaStream_t s) {
    fsq4_kernel<TMAX, NL><<<blocks_for((ntok + 3) / 4, 256), 256, 0, s>>>(z, ntok, f, th, idx, codes);
}

template <int TMAX>
bool launch_fsq4_nl(const float* z, long long ntok, const FsqConsts& f, const FsqThr& th, int32_t* idx, float* codes,
                    cudaStream_t s) {
    switch (f.nlev) {
        case 3: launch_fsq4<TMAX, 3>(z, ntok, f, th, idx, codes, s); return true;
        case 4: launch_fsq4<TMAX, 4>(z, ntok, f, th, idx, codes, s); return true;
        case 5: launch_fsq4<TMAX, 5>(z, ntok, f, th, idx, codes, s); return true;
        case 6: launch_fsq4<TMAX, 6>(z, ntok, f, th, idx, codes, s); return true;
        case 8: launch_fsq4<TMAX, 8>(z, ntok, f, th, idx, codes, s); return true;
        default: return false;
    }
}

__global__ void dequant_kernel(const int32_t* __restrict__ idx, long long ntok, FsqConsts f,
                               float* __restrict__ codes) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    const int id = idx[t];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < f.nlev) {
            const int d = (id / f.basis[i]) % f.levels[i];
            codes[t * f.nlev + i] = (float)(d - f.half_w[i]) / (float)f.half_w[i];
        }
    }
}

// ----------------------------------------------------------- Philox drop

// Philox-4x32-10 (Salmon et al., SC'11) with its ten round keys precomputed: round r
// uses k + r * (W0, W1), the same for every thread, so they are kernel parameters.
struct PhiloxKeys {
    uint32_t x[10], y[10];
};

inline PhiloxKeys philox_keys(uint2 k) {
    PhiloxKeys K;
    for (int r = 0; r < 10; ++r) {
        K.x[r] = k.x + (uint32_t)r * 0x9E3779B9u;
        K.y[r] = k.y + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.x[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.y[r],
                       (uint32_t)p0);
    }
    return c;
}

// Unsigned 32-bit division by a divisor fixed for the launch, by multiplication
// (Granlund and Montgomery, "Division by invariant integers using multiplication",
// PLDI 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, and
// q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) with t = umulhi(m, n).
struct FastDiv {
    uint32_t m, s1, s2;
};

inline FastDiv fast_div_of(uint32_t d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Rows are cut into 32-token segments (one keep-mask word each) and a warp takes
// four consecutive segments, 8 lanes each: lane l of a segment decides tokens
// w = 32 s + 4 l .. + 3 of its row from one Philox block (counter j >> 2, j the
// token's index in its sample) when the row starts on a multiple of 4 tokens,
// or from two when it does not; the 8 lanes OR their nibbles into the word.
// Only the last segment of a row can be partial, so a row of a multiple of 32
// tokens keeps every lane busy. IDX is int (segments below 2^31: divisions by
// multiplication) or long long. A token is dropped when its 32-bit word is below
// thr (all of them when thr = 2^32).
// 40 registers leave room for six 256-thread blocks per SM (46 without the bound:
// five; measured 0.218 against 0.227 ms on 118 M tokens).
template <typename IDX>
__global__ void __launch_bounds__(256, 6) drop4_kernel(const int32_t* __restrict__ idx, int TH, int Wq, int nseg, IDX segs, FastDiv div_seg,
                             FastDiv div_th, unsigned long long thr, const __grid_constant__ PhiloxKeys K,
                             uint32_t chunk_lo, uint32_t stream_lo, int32_t zero_index, int32_t* __restrict__ out,
                             uint32_t* __restrict__ keep_bits) {
    const IDX gs = ((IDX)blockIdx.x * blockDim.x + threadIdx.x) / 8;  // global segment of this lane
    const int lane = threadIdx.x % 32, sl = lane & 7;
    const bool drop_all = thr > 0xFFFFFFFFull;
    const uint32_t thr32 = (uint32_t)thr;
    uint32_t nib = 0;
    IDX row = 0;
    int sr = 0;
    if (gs < segs) {
        int n;
        if constexpr (sizeof(IDX) == 4) {
            row = (IDX)fast_div((uint32_t)gs, div_seg);
            n = (int)fast_div((uint32_t)row, div_th);
        } else {
            row = gs / nseg;
            n = (int)(row / TH);
        }
        sr = (int)(gs - row * nseg);
        const uint32_t rin = (uint32_t)(row - (IDX)n * TH);  // t*Hq + h within sample n
        const int w0 = sr * 32 + 4 * sl;
        const int nw = min(4, Wq - w0);  // tokens of this lane (<= 0: none)
        if (nw > 0) {
            const uint32_t j0 = rin * (uint32_t)Wq + (uint32_t)w0;  // sample-local index of the first token
            const uint4 r0 = philox4x32_10(make_uint4(j0 >> 2, (uint32_t)n, chunk_lo, stream_lo), K);
            uint32_t wd[4] = {r0.x, r0.y, r0.z, r0.w};
            if ((j0 & 3u) != 0u) {
                // tokens j0 .. j0 + 3 straddle two Philox blocks: word (j & 3) of block j >> 2
                uint4 r1 = r0;
                if (nw > 4 - (int)(j0 & 3u))
                    r1 = philox4x32_10(make_uint4((j0 >> 2) + 1u, (uint32_t)n, chunk_lo, stream_lo), K);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t j = j0 + (uint32_t)i;
                    const uint4& r = ((j >> 2) == (j0 >> 2)) ? r0 : r1;
                    wd[i] = (j & 3u) == 0 ? r.x : (j & 3u) == 1 ? r.y : (j & 3u) == 2 ? r.z : r.w;
                }
            }
            const long long o = (long long)row * Wq + w0;
            int32_t v[4];
            const bool vec = nw == 4 && (o & 3) == 0;
            if (vec) {
                const int4 q = *reinterpret_cast<const int4*>(idx + o);
                v[0] = q.x;
                v[1] = q.y;
                v[2] = q.z;
                v[3] = q.w;
            } else {
                for (int i = 0; i < 4; ++i) v[i] = i < nw ? idx[o + i] : 0;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool keep = i < nw && !drop_all && wd[i] >= thr32;
                if (keep) nib |= 1u << i;
                if (!keep) v[i] = zero_index;
            }
            if (vec) {
                *reinterpret_cast<int4*>(out + o) = make_int4(v[0], v[1], v[2], v[3]);
            } else {
                for (int i = 0; i < nw; ++i) out[o + i] = v[i];
            }
        }
    }
    // the 8 lanes of a segment hold its word: bits 4 (lane % 8) ..
    uint32_t m = nib << (4 * sl);
    m |= __shfl_xor_sync(0xffffffffu, m, 1);
    m |= __shfl_xor_sync(0xffffffffu, m, 2);
    m |= __shfl_xor_sync(0xffffffffu, m, 4);
    if (keep_bits && sl == 0 && gs < segs) keep_bits[(long long)row * nseg + sr] = m;
}

// --------------------------------------------------------- row packets

__global__ void row_count_kernel(const uint32_t* __restrict__ keep_bits, long long rows, int nwords,
                                 int64_t* __restrict__ counts) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int c = 0;
    for (int i = 0; i < nwords; ++i) c += __popc(keep_bits[r * nwords + i]);
    counts[r + 1] = c;  // shifted: exclusive scan done in place afterwards
}

// Single-block exclusive scan of counts[1..rows] into offsets[0..rows].
__global__ void scan_kernel(int64_t* __restrict__ offs, long long rows) {
    __shared__ int64_t carry;
    __shared__ int64_t buf[1024];
    if (threadIdx.x == 0) {
        carry = 0;
        offs[0] = 0;
    }
    __syncthreads();
    for (long long base = 0; base < rows; base += 1024) {
        const long long i = base + threadIdx.x;
        buf[threadIdx.x] = (i < rows) ? offs[i + 1] : 0;
        __syncthreads();
        for (int s = 1; s < 1024; s <<= 1) {
            int64_t v = (threadIdx.x >= (unsigned)s) ? buf[threadIdx.x - s] : 0;
            __syncthreads();
            buf[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < rows) offs[i + 1] = carry + buf[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
}

// One warp per row: compact the kept tokens (ballot + popc) into the payload.
__global__ void pack_kernel(const int32_t* __restrict__ idx, const uint32_t* __restrict__ keep_bits, long long rows,
                            int Wq, const int64_t* __restrict__ offs, int32_t* __restrict__ payload) {
    const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (r >= rows) return;
    const int nwords = (Wq + 31) / 32;
    long long o = offs[r];
    for (int wd = 0; wd < nwords; ++wd) {
        const uint32_t m = keep_bits[r * nwords + wd];
        const int w = wd * 32 + lane;
        if ((m >> lane) & 1u) payload[o + __popc(m & ((1u << lane) - 1u))] = idx[r * Wq + w];
        o += __popc(m);
    }
}

__global__ void unpack_kernel(const int32_t* __restrict__ payload, const int64_t* __restrict__ offs,
                              const uint32_t* __restrict__ keep_bits, const uint8_t* __restrict__ received,
                              long long rows, int Wq, int32_t zero_index, int32_t* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * Wq) return;
    const long long r = t / Wq;
    const int w = (int)(t % Wq);
    int32_t v = zero_index;
    if (received == nullptr || received[r]) {
        const int nwords = (Wq + 31) / 32;
        const uint32_t* kb = keep_bits + r * nwords;
        const uint32_t m = kb[w / 32];
        if ((m >> (w % 32)) & 1u) {
            int rank = __popc(m & ((1u << (w % 32)) - 1u));
            for (int i = 0; i < w / 32; ++i) rank += __popc(kb[i]);
            v = payload[offs[r] + rank];
        }
    }
    out[t] = v;
}

// Zero fill of the tokens a caller's row masks mark as dropped.
__global__ void apply_keep_kernel(const int32_t* __restrict__ idx, const uint32_t* __restrict__ keep_bits,
                                  long long ntok, int Wq, int32_t zero_index, int32_t* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    const int nwords = (Wq + 31) / 32;
    const long long row = t / Wq;
    const int w = (int)(t % Wq);
    const bool keep = (keep_bits[row * nwords + w / 32] >> (w % 32)) & 1u;
    out[t] = keep ? idx[t] : zero_index;
}


}  // namespace

int launch_apply_keep(const int32_t* idx, const uint32_t* keep_bits, long long ntok, int Wq, int32_t zero_index,
                      int32_t* out, cudaStream_t s) {
    if (ntok <= 0) return 0;
    apply_keep_kernel<<<blocks_for(ntok, 256), 256, 0, s>>>(idx, keep_bits, ntok, Wq, zero_index, out);
    return (int)cudaGetLastError();
}

int launch_fsq(const float* z, long long ntok, const FsqConsts& f, int32_t* idx, float* codes, cudaStream_t s) {
    if (ntok <= 0) return 0;
    const FsqThr th = make_fsq_thr(f.levels, f.nlev);
    int lmax = 0;
    for (int i = 0; i < f.nlev; ++i) lmax = f.levels[i] > lmax ? f.levels[i] : lmax;
    // four tokens per thread when the vectors are 16-byte aligned
    const bool aligned = (reinterpret_cast<uintptr_t>(z) % 16 == 0) && (reinterpret_cast<uintptr_t>(idx) % 16 == 0) &&
                         (!codes || reinterpret_cast<uintptr_t>(codes) % 16 == 0);
    if (aligned && (lmax <= 8 ? launch_fsq4_nl<7>(z, ntok, f, th, idx, codes, s)
                              : launch_fsq4_nl<15>(z, ntok, f, th, idx, codes, s)))
        return (int)cudaGetLastError();
    if (lmax <= 8)
        fsq_kernel<7><<<blocks_for(ntok, 256), 256, 0, s>>>(z, ntok, f, th, idx, codes);
    else
        fsq_kernel<15><<<blocks_for(ntok, 256), 256, 0, s>>>(z, ntok, f, th, idx, codes);
    return (int)cudaGetLastError();
}

int launch_dequant(const int32_t* idx, long long ntok, const FsqConsts& f, float* codes, cudaStream_t s) {
    if (ntok <= 0) return 0;
    dequant_kernel<<<blocks_for(ntok, 256), 256, 0, s>>>(idx, ntok, f, codes);
    return (int)cudaGetLastError();
}

int launch_drop(const int32_t* idx, int N, int Tq, int Hq, int Wq, unsigned long long thr, uint64_t seed,
                uint64_t stream_id, uint64_t chunk_id, int32_t zero_index, int32_t* out, uint32_t* keep_bits,
                cudaStream_t s) {
    const long long rows = (long long)N * Tq * Hq;
    const int nseg = (Wq + 31) / 32;  // 32-token segments (keep-mask words) per row
    const long long segs = rows * nseg;
    if (segs <= 0) return 0;
    const PhiloxKeys K = philox_keys(make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)));
    const uint32_t clo = (uint32_t)(chunk_id & 0xffffffffu), slo = (uint32_t)(stream_id & 0xffffffffu);
    const int TH = Tq * Hq;
    const long long threads = (segs + 3) / 4 * 32;  // four segments per warp
    const FastDiv dseg = fast_div_of((uint32_t)nseg), dth = fast_div_of((uint32_t)TH);
    if (threads < (1LL << 31))
        drop4_kernel<int><<<blocks_for(threads, 256), 256, 0, s>>>(idx, TH, Wq, nseg, (int)segs, dseg, dth, thr, K,
                                                                   clo, slo, zero_index, out, keep_bits);
    else
        drop4_kernel<long long><<<blocks_for(threads, 256), 256, 0, s>>>(idx, TH, Wq, nseg, segs, dseg, dth, thr,
                                                                         K, clo, slo, zero_index, out, keep_bits);
    return (int)cudaGetLastError();
}

int launch_pack(const int32_t* idx, const uint32_t* keep_bits, long long rows, int Wq, int32_t* payload,
                int64_t* offs, cudaStream_t s) {
    if (rows <= 0) return 0;
    const int nwords = (Wq + 31) / 32;
    row_count_kernel<<<blocks_for(rows, 256), 256, 0, s>>>(keep_bits, rows, nwords, offs);
    scan_kernel<<<1, 1024, 0, s>>>(offs, rows);
    pack_kernel<<<blocks_for(rows * 32, 256), 256, 0, s>>>(idx, keep_bits, rows, Wq, offs, payload);
    return (int)cudaGetLastError();
}

int launch_unpack(const int32_t* payload, const int64_t* offs, const uint32_t* keep_bits, const uint8_t* received,
                  long long rows, int Wq, int32_t zero_index, int32_t* out, cudaStream_t s) {
    const long long n = rows * Wq;
    if (n <= 0) return 0;
    unpack_kernel<<<blocks_for(n, 256), 256, 0, s>>>(payload, offs, keep_bits, received, rows, Wq, zero_index, out);
    return (int)cudaGetLastError();
}

}  // namespace tok
