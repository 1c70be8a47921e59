// FP32 CUDA-core causal 3D convolution (implicit GEMM, no tensor cores, no TF32).
//
// The plain-FP32 GPU form of the tokenizer: the same causal convolution as the
// tcgen05 path (see conv_args.h for the definition), as an implicit GEMM with
// M = output voxels, N = output channels, K = taps * Cin. A 128 x BN output
// tile per 256-thread block, K staged through shared memory 8 at a time with
// register prefetch of the next slice, 8 x (BN/16) outputs per thread.
#include "common.cuh"
#include "conv_args.h"

namespace tok {

namespace {

constexpr int BM = 128;
constexpr int BK = 8;
constexpr int NT = 256;

struct RowGeo {
    int n, to, ho, wo;
    bool valid;
};

__device__ __forceinline__ RowGeo row_geo(const ConvArgs& a, long long m, long long M) {
    RowGeo g;
    g.valid = m < M;
    long long mm = g.valid ? m : 0;
    g.wo = (int)(mm % a.Wout);
    mm /= a.Wout;
    g.ho = (int)(mm % a.Hout);
    mm /= a.Hout;
    g.to = (int)(mm % a.Tout);
    g.n = (int)(mm / a.Tout);
    return g;
}

// Address of x[n, ti, hi, wi, 0] under the causal/zero padding rules, or null.
__device__ __forceinline__ const float* src_ptr(const ConvArgs& a, const RowGeo& g, int dt, int dh, int dw) {
    if (!g.valid) return nullptr;
    int hi = g.ho * a.sh + dh - (a.kh - 1) / 2;
    int wi = g.wo * a.sw + dw - (a.kw - 1) / 2;
    if (hi < 0 || hi >= a.Hin || wi < 0 || wi >= a.Win) return nullptr;
    int ti = g.to * a.st + dt + a.t_off;
    if (ti >= a.Tin) return nullptr;  // past the last frame (adjoint convs read ahead): zeros
    const float* base = static_cast<const float*>(a.x);
    long long frame;
    if (ti < 0) {
        if (a.hist) {
            base = static_cast<const float*>(a.hist);
            frame = (long long)g.n * a.hist_T + (a.hist_T + ti);
        } else if (a.pad_mode == 0) {
            frame = (long long)g.n * a.Tin;
        } else {
            return nullptr;
        }
    } else {
        frame = (long long)g.n * a.Tin + ti;
    }
    return base + ((frame * a.Hin + hi) * a.Win + wi) * (long long)a.Cin;
}

// Output element address for conv-grid voxel g and channel co (null if cropped).
__device__ __forceinline__ long long out_offset(const ConvArgs& a, const RowGeo& g, int co) {
    if (a.mode == OUT_D2S) {
        int ch = co % a.oC;
        int sub = co / a.oC;
        int c = sub % a.rw;
        int b = (sub / a.rw) % a.rh;
        int t = sub / (a.rw * a.rh);
        int ot = g.to * a.rt + t - a.drop_t;
        int oh = g.ho * a.rh + b;
        int ow = g.wo * a.rw + c;
        if (ot < 0 || ot >= a.oT || oh >= a.oH || ow >= a.oW) return -1;
        return ((((long long)g.n * a.oT + ot) * a.oH + oh) * a.oW + ow) * a.oC + ch;
    }
    return ((((long long)g.n * a.oT + g.to) * a.oH + g.ho) * a.oW + g.wo) * a.oC + co;
}

template <int BN>
__global__ void __launch_bounds__(NT) conv_simt_kernel(ConvArgs a) {
    constexpr int TN = BN / 16;
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const long long M = (long long)a.N * a.Tout * a.Hout * a.Wout;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int taps = a.kt * a.kh * a.kw;
    const bool vec = (a.Cin % BK) == 0;
    const int nks = vec ? taps * (a.Cin / BK) : a.Kpad / BK;

    // A loader: row lr, k-half lk (4 consecutive k)
    const int lr = tid / 2, lk = (tid % 2) * 4;
    const RowGeo g = row_geo(a, m0 + lr, M);

    constexpr int BLOADS = (BN * BK + NT - 1) / NT;  // scalars of B per thread
    float ra[4], rbv[BLOADS];

    auto load_a = [&](int ks) {
        if (vec) {
            int cpt = a.Cin / BK;
            int tap = ks / cpt;
            int c0 = (ks % cpt) * BK + lk;
            int dw = tap % a.kw, dh = (tap / a.kw) % a.kh, dt = tap / (a.kw * a.kh);
            const float* p = src_ptr(a, g, dt, dh, dw);
            if (p) {
                float4 v = *reinterpret_cast<const float4*>(p + c0);
                ra[0] = v.x; ra[1] = v.y; ra[2] = v.z; ra[3] = v.w;
            } else {
                ra[0] = ra[1] = ra[2] = ra[3] = 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int k = ks * BK + lk + e;
                float v = 0.f;
                if (k < taps * a.Cin) {
                    int tap = k / a.Cin, ci = k % a.Cin;
                    int dw = tap % a.kw, dh = (tap / a.kw) % a.kh, dt = tap / (a.kw * a.kh);
                    const float* p = src_ptr(a, g, dt, dh, dw);
                    if (p) v = p[ci];
                }
                ra[e] = v;
            }
        }
    };
    // B: W[n0 + n][k0 + k], element e of thread -> linear (n, k) = tid + e*NT
    auto load_b = [&](int ks) {
        int kbase;
        if (vec) {
            int cpt = a.Cin / BK;
            kbase = (ks / cpt) * a.Cin + (ks % cpt) * BK;
        } else {
            kbase = ks * BK;
        }
        const float* w = static_cast<const float*>(a.w);
#pragma unroll
        for (int e = 0; e < BLOADS; ++e) {
            int lin = tid + e * NT;
            int nn = lin / BK, kk = lin % BK;
            float v = 0.f;
            if (lin < BN * BK && n0 + nn < a.Cout_pad) v = w[(long long)(n0 + nn) * a.Kpad + kbase + kk];
            rbv[e] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int e = 0; e < 4; ++e) As[buf][lk + e][lr] = ra[e];
#pragma unroll
        for (int e = 0; e < BLOADS; ++e) {
            int lin = tid + e * NT;
            if (lin < BN * BK) Bs[buf][lin % BK][lin / BK] = rbv[e];
        }
    };

    float acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    load_a(0);
    load_b(0);
    store(0);
    __syncthreads();
    for (int ks = 0; ks < nks; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < nks) {
            load_a(ks + 1);
            load_b(ks + 1);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float av[8], bv[TN];
            float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
            av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
            av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (ks + 1 < nks) store(buf ^ 1);
        __syncthreads();
    }

    // epilogue
    float* out = static_cast<float*>(a.out);
    const float* res = static_cast<const float*>(a.residual);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
        RowGeo og = row_geo(a, m0 + r, M);
        if (!og.valid) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int co = n0 + tx + 16 * j;
            if (co >= a.Cout) continue;
            long long off = out_offset(a, og, co);
            if (off < 0) continue;
            float v = acc[i][j] + (a.bias ? a.bias[co] : 0.f);
            if (res) v += res[off];
            out[off] = gop_blend_out(a, off, v);
        }
    }
}

}  // namespace

int launch_conv_simt(const ConvArgs& a, cudaStream_t stream) {
    const long long M = (long long)a.N * a.Tout * a.Hout * a.Wout;
    if (M == 0) return 0;
    dim3 block(NT);
    unsigned gx = (unsigned)((M + BM - 1) / BM);
    if (a.Cout_pad >= 128) {
        dim3 grid(gx, (a.Cout_pad + 127) / 128);
        conv_simt_kernel<128><<<grid, block, 0, stream>>>(a);
    } else if (a.Cout_pad >= 64) {
        dim3 grid(gx, (a.Cout_pad + 63) / 64);
        conv_simt_kernel<64><<<grid, block, 0, stream>>>(a);
    } else {
        dim3 grid(gx, (a.Cout_pad + 15) / 16);
        conv_simt_kernel<16><<<grid, block, 0, stream>>>(a);
    }
    return (int)cudaGetLastError();
}

}  // namespace tok
