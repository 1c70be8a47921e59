// Geometry and epilogue description of one causal 3D convolution launch,
// shared by the tcgen05 (BF16) and CUDA-core (FP32) conv kernels.
//
// Convolution (causal in time, zero-padded in space):
//   y[n,to,ho,wo,co] = bias[co] + sum_{dt,dh,dw,ci} W[co,dt,dh,dw,ci] * x[n,ti,hi,wi,ci]
//   ti = to*st + dt + t_off   (clip mode: t_off = -(kt-1), the causal left pad)
//   hi = ho*sh + dh - (kh-1)/2,  wi = wo*sw + dw - (kw-1)/2
// A tap with ti < 0 reads, in this order of precedence: frame (hist_T + ti)
// of the history tensor when one is given (streaming), frame 0 (replicate
// pad) or zero (zero pad). A tap with ti >= Tin (only the adjoint convs of the
// backward read ahead) and taps outside [0,H) x [0,W) read zero.
//
// Epilogue modes:
//   OUT_PLAIN : out[n,to,ho,wo,co] = y (+ residual[n,to,ho,wo,co])
//   OUT_D2S   : depth-to-space: channel co = ((a*rh+b)*rw+c)*oC + ch of y at
//               (to,ho,wo) goes to out[n, to*rt + a - drop_t, ho*rh+b, wo*rw+c, ch];
//               frames < 0 are dropped, rows/cols >= oH/oW are cropped.
//   OUT_FSQ   : out is the fp32 latent z; idx gets the FSQ token index.
// An fp32 output may be blended with the previous GoP's reconstruction at the
// GoP boundary (Sec. 6.1, Eq. 2): see blend_prev below.
#pragma once
#include <stdint.h>

#include <cmath>

namespace tok {

enum OutMode { OUT_PLAIN = 0, OUT_D2S = 1, OUT_FSQ = 2 };

// Most inputs one grouped conv launch takes (clips or stream chunks of one layer).
constexpr int kMaxConvGroup = 8;

struct FsqConsts {
    int nlev;
    int levels[8];     // L_i
    float half_l[8];   // (L-1)(1-eps)/2
    float offset[8];   // 0.5 for even L else 0
    float shift[8];    // atanh(offset/half_l)
    int half_w[8];     // L/2
    int basis[8];      // prod_{j<i} L_j
};

// FSQ rounding as thresholds on z. With b = tanh(z + s) h - o and q = round(b), the
// digit d = q + floor(L/2) exceeds k exactly when b > k + 1/2 - floor(L/2), i.e. when
// z > atanh((k + 1/2 - floor(L/2) + o) / h) - s (tanh is increasing); t[c][k] is the
// smallest float above that bound, computed in double, so a float z passes it when
// z >= t[c][k], and the digit of channel c is the number of its thresholds that z
// passes. This is the rounding of the exactly computed bounded value (a float32
// tanh would misplace z within a few ulps of a bound). NaN pads the unused entries.
struct FsqThr {
    float t[8][15];
};

inline FsqThr make_fsq_thr(const int* levels, int nlev) {
    FsqThr th;
    for (int c = 0; c < 8; ++c)
        for (int k = 0; k < 15; ++k) th.t[c][k] = NAN;
    for (int c = 0; c < nlev && c < 8; ++c) {
        const int L = levels[c], hw = L / 2;
        const double h = (L - 1) * (1.0 - 1e-3) / 2.0;
        const double o = (L % 2 == 0) ? 0.5 : 0.0;
        const double s = std::atanh(o / h);
        for (int k = 0; k < L - 1 && k < 15; ++k) {
            const double x = std::atanh((k + 0.5 - hw + o) / h) - s;
            float f = (float)x;
            if ((double)f <= x) f = std::nextafter(f, INFINITY);
            th.t[c][k] = f;
        }
    }
    return th;
}

// Digit of channel c (TMAX >= L - 1 thresholds examined; NaN entries never pass).
template <int TMAX>
__device__ __forceinline__ int fsq_digit(const FsqThr& th, int c, float z) {
    int d = 0;
#pragma unroll
    for (int k = 0; k < TMAX; ++k) d += (z >= th.t[c][k]) ? 1 : 0;
    return d;
}

// Partial GroupNorm statistics of a set of values: count, mean and the sum of
// squared deviations from the mean (merged with Chan's pairwise update).
struct GnTriple {
    float n, mean, m2;
};

struct ConvArgs {
    // input (the chunk / clip) and optional history
    const void* x;        // (N, Tin, Hin, Win, Cin)
    const void* hist;     // (N, hist_T, Hin, Win, Cin) or null
    int hist_T;
    int N, Tin, Hin, Win, Cin;
    // weights: (Cout_pad, Kpad) with K = taps*Cin laid out (tap, ci)
    const void* w;
    // weights for the tiles of output frame 0 (same layout), or null: the adjoint of
    // a replicate-padded conv, where input frame 0 also stood in for the padded frames
    const void* w0;
    // spatial taps in the weight rows of a narrow 3x3x3 stride-1 head: 0 (no), 3 (rows
    // dw * 16 + co over K = (dt, dh, ci), Cout <= 16) or 9 (rows (dh * 3 + dw) * Cout + co
    // over K = (dt, ci), 9 * Cout <= 128)
    int w_dwm;
    const float* bias;    // (Cout) fp32
    int Cout, Cout_pad, Kpad;
    int kt, kh, kw, st, sh, sw;
    int t_off, pad_mode;
    // output (pre-epilogue conv grid)
    int Tout, Hout, Wout;
    // epilogue
    int mode;
    void* out;
    int out_fp32;         // store fp32 (else bf16 on the BF16 path)
    int oT, oH, oW, oC;   // output tensor dims per sample
    int rt, rh, rw, drop_t;
    const void* residual; // same layout as out (OUT_PLAIN only) or null
    int32_t* idx;         // OUT_FSQ
    FsqConsts fsq;
    const FsqThr* fsq_thr;  // OUT_FSQ: the thresholds of fsq in device memory
    // GroupNorm statistics of the stored output (bf16 values after the residual),
    // for the GroupNorm that reads it next: per (frame, slot, group) triples, a slot
    // being a spatial tile (times the rh x rw sub-positions for OUT_D2S); groups of
    // gn_cg consecutive channels. Null: none. Only the swapped wide form writes them.
    GnTriple* gn_part;
    int gn_cg;
    // 1: the tile of a layer with statistics may depend on the frame count (a
    // training forward, which no stream of chunks has to reproduce bit for bit)
    int gn_any_tile;
    // GoP boundary blend of an fp32 output (Eq. 2): output frame ot < blend_n of
    // sample n becomes a * prev[n, blend_Tp - blend_n + ot] + (1 - a) * out with
    // a = (blend_n - 1 - ot) / blend_n; prev is (N, blend_Tp, oH, oW, oC) fp32.
    // blend_n = 0: none.
    const float* blend_prev;
    int blend_n, blend_Tp;
    // device status / bounded waits
    int* status;
    unsigned long long wait_ns;
};

#ifdef __CUDACC__
// The value an fp32 output element at flat offset `off` is stored as: itself, or
// its Eq. 2 blend with the previous GoP (the same float operations as the
// stand-alone blend kernel, so the two agree bit for bit).
__device__ __forceinline__ float gop_blend_out(const ConvArgs& a, long long off, float o) {
    if (a.blend_n <= 0) return o;
    const long long fe = (long long)a.oH * a.oW * a.oC;
    const long long f = off / fe;
    const int ot = (int)(f % a.oT);
    if (ot >= a.blend_n) return o;
    const long long n = f / a.oT;
    const float al = __fdiv_rn((float)(a.blend_n - 1 - ot), (float)a.blend_n);
    const float p = a.blend_prev[(n * a.blend_Tp + (a.blend_Tp - a.blend_n + ot)) * fe + (off - f * fe)];
    return __fmaf_rn(al, p, __fmul_rn(__fsub_rn(1.f, al), o));
}
#endif

// The tensor-core kernel form of a BF16 conv (see conv_route).
struct ConvRoute {
    bool taps3, narrow, swap, halo;
};

// Geometry of the im2col gathers (pixel stem / dequantised decoder input).
struct GatherGeo {
    int N, Tin, H, W, Hp, Wp, Cin;  // source (H,W real extent; Hp,Wp logical padded extent)
    int hist_T;
    int Tout, Hout, Wout;
    int kt, kh, kw, st, sh, sw, t_off, pad_mode;
    int Kpad;
};

// One problem of the fused BF16 stem (k_stem_tc.cu): the causal 3x3x3 conv with
// stride (st, 2, 2) from the pixels x (N, Tin, H, W, 3) to out (N, Tout, H/2,
// W/2, Cout), frames before the clip taken from hist (N, hist_T, H, W, 3) when
// it is given, else frame 0 (pad_mode 0) or zeros; zeros outside the frame.
struct StemArgs {
    const void* x;
    const void* hist;  // or null
    int hist_T;
    int N, Tin, H, W;
    int Tout, st, t_off, pad_mode;
    const void* w;       // packed (Cout_pad, Kpad) bf16, K = (dt, dh, dw, ci), zeros from 81 on
    const float* bias;   // (Cout) or null
    int Cout, Cout_pad, Kpad;
    void* out;           // bf16
    GnTriple* gn_part;   // GroupNorm statistics (N * Tout, stem_tc_gn_slots, 32) triples, or null
    int* status;
    unsigned long long wait_ns;
};

// One weight-gradient problem: dY of a conv (N,Tout,Hout,Wout,Cdy) against its input
// (N,Tin,Hin,Win,Cin); same tap rule as the forward conv.
struct WgradArgs {
    int N, Tin, Hin, Win, Cin;
    int Tout, Hout, Wout, Cout, Cdy;  // Cdy: channel stride of dY (>= Cout)
    int kt, kh, kw, st, sh, sw, t_off, pad_mode;
    int K;                            // taps * Cin
    long long V;                      // N * Tout * Hout * Wout
    long long vchunk;                 // voxels per split
    // dw rows (narrow 3x3x3 stride-1 layers): dY holds the three w-shifted copies of
    // the gradient as rows dw * 16 + co (Cout = 48 rows, cout_real real channels), and a
    // CTA slot is dt alone
    int dwrows, cout_real;
};

}  // namespace tok
