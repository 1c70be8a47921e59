/*
 * FP64 direct-loop causal 3D convolution: the oracle's convolution.
 *
 * TEST INFRASTRUCTURE ONLY. This file is part of the oracle: only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it. The
 * product path never calls it.
 *
 * What it computes (the tokenizer's "causal 3D conv", the building block of
 * the encoder f_phi and decoder g_theta of Sec. 2.4, whose causal residual
 * blocks are named in Sec. 1, challenge C2):
 *
 *   y[n,to,ho,wo,co] = b[co] + sum_{dt,dh,dw,ci} w[co,dt,dh,dw,ci]
 *                              * x[n, ti, hi, wi, ci]
 *   ti = to*st + dt - (kt-1)        (causal: left pad of kt-1 frames)
 *   hi = ho*sh + dh - (kh-1)/2      (symmetric spatial pad, zeros)
 *   wi = wo*sw + dw - (kw-1)/2
 *
 * A tap with ti < 0 reads frame 0 (pad_mode 0, replicate) or zero
 * (pad_mode 1). A tap outside [0,H) x [0,W) reads zero.
 * Layouts are channels-last: x (N,T,H,W,Cin), y (N,To,Ho,Wo,Cout),
 * w (Cout,kt,kh,kw,Cin), all contiguous doubles.
 *
 * dgrad and wgrad are the exact transposes of the loop above (same tap rule),
 * written as scatter (dgrad) and gather (wgrad) over the very same loop nest,
 * so that they are obviously the adjoint of the forward.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Resolve the input frame read by output frame `to` at temporal tap `dt`.
 * Returns -1 when the tap reads zero padding. */
static inline long src_frame(int to, int dt, int st, int kt, int pad_mode) {
    long ti = (long)to * st + dt - (kt - 1);
    if (ti < 0) return pad_mode == 0 ? 0 : -1;
    return ti;
}

static inline long src_pos(int o, int d, int s, int k, int extent) {
    long i = (long)o * s + d - (k - 1) / 2;
    if (i < 0 || i >= extent) return -1;
    return i;
}

void oracle_conv3d_fwd(const double* x, int N, int T, int H, int W, int Cin,
                       const double* w, const double* b, int Cout,
                       int kt, int kh, int kw, int st, int sh, int sw, int pad_mode,
                       double* y, int To, int Ho, int Wo) {
    const long taps = (long)kt * kh * kw;
#pragma omp parallel for collapse(3) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int to = 0; to < To; ++to)
            for (int ho = 0; ho < Ho; ++ho)
                for (int wo = 0; wo < Wo; ++wo) {
                    double* yo = y + ((((long)n * To + to) * Ho + ho) * Wo + wo) * Cout;
                    for (int co = 0; co < Cout; ++co) {
                        double acc = b ? b[co] : 0.0;
                        for (int dt = 0; dt < kt; ++dt) {
                            long ti = src_frame(to, dt, st, kt, pad_mode);
                            if (ti < 0) continue;
                            for (int dh = 0; dh < kh; ++dh) {
                                long hi = src_pos(ho, dh, sh, kh, H);
                                if (hi < 0) continue;
                                for (int dw = 0; dw < kw; ++dw) {
                                    long wi = src_pos(wo, dw, sw, kw, W);
                                    if (wi < 0) continue;
                                    const double* xp = x + ((((long)n * T + ti) * H + hi) * W + wi) * Cin;
                                    const double* wp = w + ((long)co * taps + ((long)dt * kh + dh) * kw + dw) * Cin;
                                    double s = 0.0;
#pragma omp simd reduction(+ : s)
                                    for (int ci = 0; ci < Cin; ++ci) s += wp[ci] * xp[ci];
                                    acc += s;
                                }
                            }
                        }
                        yo[co] = acc;
                    }
                }
}

/* dx = (d y / d x)^T dy. Parallel over input channels so that every thread
 * owns a disjoint slice of dx (no races, fixed summation order). */
void oracle_conv3d_dgrad(const double* dy, int N, int To, int Ho, int Wo, int Cout,
                         const double* w, int kt, int kh, int kw, int st, int sh, int sw,
                         int pad_mode, double* dx, int T, int H, int W, int Cin) {
    const long taps = (long)kt * kh * kw;
    memset(dx, 0, sizeof(double) * (size_t)N * T * H * W * Cin);
#pragma omp parallel for schedule(static)
    for (int ci = 0; ci < Cin; ++ci)
        for (int n = 0; n < N; ++n)
            for (int to = 0; to < To; ++to)
                for (int ho = 0; ho < Ho; ++ho)
                    for (int wo = 0; wo < Wo; ++wo) {
                        const double* g = dy + ((((long)n * To + to) * Ho + ho) * Wo + wo) * Cout;
                        for (int dt = 0; dt < kt; ++dt) {
                            long ti = src_frame(to, dt, st, kt, pad_mode);
                            if (ti < 0) continue;
                            for (int dh = 0; dh < kh; ++dh) {
                                long hi = src_pos(ho, dh, sh, kh, H);
                                if (hi < 0) continue;
                                for (int dw = 0; dw < kw; ++dw) {
                                    long wi = src_pos(wo, dw, sw, kw, W);
                                    if (wi < 0) continue;
                                    long tap = ((long)dt * kh + dh) * kw + dw;
                                    double s = 0.0;
                                    for (int co = 0; co < Cout; ++co)
                                        s += w[((long)co * taps + tap) * Cin + ci] * g[co];
                                    dx[((((long)n * T + ti) * H + hi) * W + wi) * Cin + ci] += s;
                                }
                            }
                        }
                    }
}

/* dw[co,tap,ci] = sum over outputs of dy[...,co] * x[src(tap),ci];
 * db[co] = sum over outputs of dy[...,co]. Parallel over output channels. */
void oracle_conv3d_wgrad(const double* dy, int N, int To, int Ho, int Wo, int Cout,
                         const double* x, int T, int H, int W, int Cin,
                         int kt, int kh, int kw, int st, int sh, int sw, int pad_mode,
                         double* dw_out, double* db_out) {
    const long taps = (long)kt * kh * kw;
#pragma omp parallel for schedule(static)
    for (int co = 0; co < Cout; ++co) {
        double* dwc = dw_out + (long)co * taps * Cin;
        for (long i = 0; i < taps * Cin; ++i) dwc[i] = 0.0;
        double bsum = 0.0;
        for (int n = 0; n < N; ++n)
            for (int to = 0; to < To; ++to)
                for (int ho = 0; ho < Ho; ++ho)
                    for (int wo = 0; wo < Wo; ++wo) {
                        double g = dy[((((long)n * To + to) * Ho + ho) * Wo + wo) * Cout + co];
                        bsum += g;
                        for (int dt = 0; dt < kt; ++dt) {
                            long ti = src_frame(to, dt, st, kt, pad_mode);
                            if (ti < 0) continue;
                            for (int dh = 0; dh < kh; ++dh) {
                                long hi = src_pos(ho, dh, sh, kh, H);
                                if (hi < 0) continue;
                                for (int dw = 0; dw < kw; ++dw) {
                                    long wi = src_pos(wo, dw, sw, kw, W);
                                    if (wi < 0) continue;
                                    long tap = ((long)dt * kh + dh) * kw + dw;
                                    const double* xp = x + ((((long)n * T + ti) * H + hi) * W + wi) * Cin;
                                    double* d = dwc + tap * Cin;
#pragma omp simd
                                    for (int ci = 0; ci < Cin; ++ci) d[ci] += g * xp[ci];
                                }
                            }
                        }
                    }
        if (db_out) db_out[co] = bsum;
    }
}

int oracle_num_threads(void) {
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}
