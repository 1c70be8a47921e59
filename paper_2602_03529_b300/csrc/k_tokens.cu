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

__global__ void fsq_kernel(const float* __restrict__ z, long long ntok, FsqConsts f, int32_t* __restrict__ idx,
                           float* __restrict__ codes) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntok) return;
    const float* zp = z + t * f.nlev;
    int id = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < f.nlev) {
            const float b = tanhf(zp[i] + f.shift[i]) * f.half_l[i] - f.offset[i];
            const float q = rintf(b);
            id += ((int)q + f.half_w[i]) * f.basis[i];
            if (codes) codes[t * f.nlev + i] = q / (float)f.half_w[i];
        }
    }
    idx[t] = id;
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

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Rows are cut into 32-token segments (one keep-mask word each) and a warp takes
// four consecutive segments, 8 lanes each: lane l of a segment decides tokens
// w = 32 s + 4 l .. + 3 of its row from one Philox block (counter j >> 2, j the
// token's index in its sample) when the row starts on a multiple of 4 tokens,
// or from two when it does not; the 8 lanes OR their nibbles into the word.
// Only the last segment of a row can be partial, so a row of a multiple of 32
// tokens keeps every lane busy. IDX is int (segments below 2^31) or long long.
template <typename IDX>
__global__ void drop4_kernel(const int32_t* __restrict__ idx, int TH, int Wq, int nseg, IDX segs,
                             unsigned long long thr, uint2 key, uint32_t chunk_lo, uint32_t stream_lo,
                             int32_t zero_index, int32_t* __restrict__ out, uint32_t* __restrict__ keep_bits) {
    const IDX gs = ((IDX)blockIdx.x * blockDim.x + threadIdx.x) / 8;  // global segment of this lane
    const int lane = threadIdx.x % 32, sl = lane & 7;
    uint32_t nib = 0;
    IDX row = 0;
    int sr = 0;
    if (gs < segs) {
        row = gs / nseg;
        sr = (int)(gs - row * nseg);
        const int n = (int)(row / TH);
        const uint32_t rin = (uint32_t)(row - (IDX)n * TH);  // t*Hq + h within sample n
        const int w0 = sr * 32 + 4 * sl;
        const int nw = min(4, Wq - w0);  // tokens of this lane (<= 0: none)
        if (nw > 0) {
            const uint32_t j0 = rin * (uint32_t)Wq + (uint32_t)w0;  // sample-local index of the first token
            const uint4 r0 = philox4x32_10(make_uint4(j0 >> 2, (uint32_t)n, chunk_lo, stream_lo), key);
            uint4 r1 = r0;
            if ((j0 & 3u) != 0u && nw > 4 - (int)(j0 & 3u))
                r1 = philox4x32_10(make_uint4((j0 >> 2) + 1u, (uint32_t)n, chunk_lo, stream_lo), key);
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
                const uint32_t j = j0 + (uint32_t)i;
                const uint4& r = ((j >> 2) == (j0 >> 2)) ? r0 : r1;
                const uint32_t word32 = (j & 3u) == 0 ? r.x : (j & 3u) == 1 ? r.y : (j & 3u) == 2 ? r.z : r.w;
                const bool keep = i < nw && !((unsigned long long)word32 < thr);
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

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

int launch_apply_keep(const int32_t* idx, const uint32_t* keep_bits, long long ntok, int Wq, int32_t zero_index,
                      int32_t* out, cudaStream_t s) {
    if (ntok <= 0) return 0;
    apply_keep_kernel<<<blocks_for(ntok, 256), 256, 0, s>>>(idx, keep_bits, ntok, Wq, zero_index, out);
    return (int)cudaGetLastError();
}

int launch_fsq(const float* z, long long ntok, const FsqConsts& f, int32_t* idx, float* codes, cudaStream_t s) {
    if (ntok <= 0) return 0;
    fsq_kernel<<<blocks_for(ntok, 256), 256, 0, s>>>(z, ntok, f, idx, codes);
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
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const uint32_t clo = (uint32_t)(chunk_id & 0xffffffffu), slo = (uint32_t)(stream_id & 0xffffffffu);
    const int TH = Tq * Hq;
    const long long threads = (segs + 3) / 4 * 32;  // four segments per warp
    if (threads < (1LL << 31))
        drop4_kernel<int><<<blocks_for(threads, 256), 256, 0, s>>>(idx, TH, Wq, nseg, (int)segs, thr, key, clo,
                                                                   slo, zero_index, out, keep_bits);
    else
        drop4_kernel<long long><<<blocks_for(threads, 256), 256, 0, s>>>(idx, TH, Wq, nseg, segs, thr, key, clo,
                                                                         slo, zero_index, out, keep_bits);
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
