// Inference executor over a group of inputs: the encoder and decoder layer
// walk (Sec. 2.4, f_phi and g_theta) for 1 .. kMaxConvGroup problems at once,
// each a whole clip or the next chunk of a stream, of any size. Every conv of
// a layer is one grouped tensor-core launch over all problems and every
// GroupNorm+SiLU one grouped pass; the gathers and cache copies, which are
// small, run per problem. Each problem has its own slice of the arena.
#pragma once
#include <array>

#include "tok_internal.h"

namespace tok {
namespace {

struct GroupExec : Exec {
    struct Prob {
        Work w;
        tok_stream* st = nullptr;  // chunked streaming (null: whole clip)
        bool chunk0 = true;        // first chunk of a stream: clip-mode causal padding
        // GoP boundary blend of the decoded frames with the previous GoP (Eq. 2)
        const float* blend_prev = nullptr;
        int blend_n = 0, blend_Tp = 0;
    };
    using MAct = std::array<Act, kMaxConvGroup>;
    int P = 0;
    Prob pr[kMaxConvGroup];

    // ------------------------------------------------------------ streaming

    // A conv with temporal taps reads its left context from the stream's
    // history; stride-2 convs see chunks that start one frame after an
    // output frame, hence t_off -1 instead of -2.
    void stream_args(int p, ConvArgs& a, const std::string& name, int k, int st_t) {
        const Prob& q = pr[p];
        if (!q.st || k != 3 || q.chunk0) return;
        a.hist = q.st->hist[name];
        a.hist_T = 2;
        if (st_t == 2) a.t_off = -1;
    }

    // After a causal conv of a stream: history <- last two frames of [history | chunk].
    void stream_update(int p, const std::string& name, const void* chunk, int Tc, bool zero_index_fill = false) {
        tok_stream* st = pr[p].st;
        if (!st || err) return;
        auto it = st->hist.find(name);
        if (it == st->hist.end()) return;
        char* h = it->second;
        const size_t fb = st->frame_bytes[name];
        const char* x = static_cast<const char*>(chunk);
        auto cp = [&](void* d, const void* src, size_t n) {
            if (cudaMemcpyAsync(d, src, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ck(1);
        };
        if (pr[p].chunk0) {
            if (c->arch.time_pad == TOK_PAD_REPLICATE) {
                cp(h, x, fb);
            } else if (zero_index_fill) {
                other([&] { return launch_fill_i32(reinterpret_cast<int32_t*>(h), (long long)(fb / 4),
                                                   zero_index_of(c), s); }, (double)fb);
            } else if (cudaMemsetAsync(h, 0, fb, s) != cudaSuccess) {
                ck(1);
            }
            cp(h + fb, x + (size_t)(Tc - 1) * fb, fb);
        } else if (Tc >= 2) {
            cp(h, x + (size_t)(Tc - 2) * fb, 2 * fb);
        } else {
            cp(h, h + fb, fb);
            cp(h + fb, x, fb);
        }
    }

    // ------------------------------------------------------------ launches

    // trace_first: as[0] is batch item 0, the problem a layer trace records
    void launch_group(ConvArgs* as, const ConvW& cw, int n = -1, bool trace_first = true) {
        if (err) return;
        const int P = n < 0 ? this->P : n;
        double flop = 0;
        for (int p = 0; p < P; ++p)
            flop += 2.0 * (double)as[p].N * as[p].Tout * as[p].Hout * as[p].Wout * cw.Cout *
                    (double)(cw.k * cw.k * cw.k) * cw.Cin;
        const int e = pbegin();
        if (c->bf16()) {
            ck(launch_conv_tc_group(as, P, c->num_sms, s, c->cta_tiles));
            c->launches += 1;
        } else {
            for (int p = 0; p < P; ++p) ck(launch_conv_simt(as[p], s));
            c->launches += P;
        }
        pend(e, 0, flop, cw.name);
        if (trace_first) trace_conv(cw.name, as[0]);
    }

    void slot(int i, void** out) const {
        for (int p = 0; p < P; ++p) out[p] = pr[p].w.act[i];
    }

    // Conv (optional residual) into outs[p].
    MAct conv(const std::string& name, const MAct& in, void* const* outs, const MAct* res = nullptr, int tst = 1,
              int sh = 1, int sw = 1) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs as[kMaxConvGroup];
        MAct out;
        for (int p = 0; p < P; ++p) {
            ConvArgs& a = as[p];
            a = base_args(cw, in[p], tst, sh, sw);
            stream_args(p, a, name, cw.k, tst);
            a.mode = OUT_PLAIN;
            a.out = outs[p];
            a.residual = res ? (*res)[p].p : nullptr;
            a.oT = a.Tout;
            a.oH = a.Hout;
            a.oW = a.Wout;
            a.oC = cw.Cout;
            want_gn_stats(a, pr[p].w, cw.Cout);
            out[p] = Act{outs[p], in[p].N, a.Tout, a.Hout, a.Wout, cw.Cout};
            tag_gn_stats(out[p], a);
        }
        launch_group(as, cw);
        for (int p = 0; p < P; ++p) stream_update(p, name, in[p].p, in[p].T);
        return out;
    }
    MAct conv_slot(const std::string& name, const MAct& in, int i, const MAct* res = nullptr, int tst = 1,
                   int sh = 1, int sw = 1) {
        void* o[kMaxConvGroup];
        slot(i, o);
        return conv(name, in, o, res, tst, sh, sw);
    }

    // Conv followed by depth-to-space (rt, rh, rw), cropped to oH[p] x oW[p].
    MAct conv_d2s(const std::string& name, const MAct& in, void* const* outs, int rt, int rh, int rw, const int* oH,
                  const int* oW, bool out_fp32, bool pixels = false) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs as[kMaxConvGroup];
        MAct out;
        for (int p = 0; p < P; ++p) {
            ConvArgs& a = as[p];
            a = base_args(cw, in[p], 1, 1, 1);
            stream_args(p, a, name, cw.k, 1);
            a.mode = OUT_D2S;
            a.out = outs[p];
            a.out_fp32 = out_fp32 ? 1 : 0;
            a.rt = rt;
            a.rh = rh;
            a.rw = rw;
            // the causal trim of the first rt-1 frames belongs to the clip's start only
            a.drop_t = (pr[p].st && !pr[p].chunk0) ? 0 : rt - 1;
            a.oT = a.Tout * rt - a.drop_t;
            a.oH = oH[p];
            a.oW = oW[p];
            a.oC = cw.Cout / (rt * rh * rw);
            if (!out_fp32) want_gn_stats(a, pr[p].w, a.oC);
            if (pixels && pr[p].blend_n > 0) {
                a.blend_prev = pr[p].blend_prev;
                a.blend_n = pr[p].blend_n;
                a.blend_Tp = pr[p].blend_Tp;
            }
            out[p] = Act{outs[p], in[p].N, a.oT, oH[p], oW[p], a.oC};
            tag_gn_stats(out[p], a);
        }
        launch_group(as, cw);
        for (int p = 0; p < P; ++p) stream_update(p, name, in[p].p, in[p].T);
        return out;
    }

    // Conv over each problem's im2col matrix (BF16 path), a 1x1x1 conv over
    // (N, Tout, Hout, Wout, Kpad).
    // Problems with skip[p] set are left out (their outputs are not touched).
    MAct conv_gathered(const std::string& name, const MAct& dims, void* const* outs, int mode, int32_t* const* idx,
                       const bool* skip = nullptr) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs as[kMaxConvGroup];
        MAct out;
        int n = 0;
        for (int p = 0; p < P; ++p) {
            if (skip && skip[p]) continue;
            const Act& d = dims[p];
            Act in{pr[p].w.gather, d.N, d.T, d.H, d.W, cw.Kpad};
            ConvArgs& a = as[n++];
            a = base_args(cw, in, 1, 1, 1);
            a.Cin = cw.Kpad;
            a.kt = a.kh = a.kw = 1;
            a.t_off = 0;
            a.mode = mode;
            a.out = outs[p];
            a.idx = idx ? idx[p] : nullptr;
            a.oT = d.T;
            a.oH = d.H;
            a.oW = d.W;
            a.oC = cw.Cout;
            if (mode == OUT_PLAIN) want_gn_stats(a, pr[p].w, cw.Cout);
            out[p] = Act{outs[p], d.N, d.T, d.H, d.W, cw.Cout};
            tag_gn_stats(out[p], a);
        }
        if (n) launch_group(as, cw, n, !(skip && skip[0]));
        return out;
    }

    MAct gn_silu(const std::string& name, const MAct& in, int i) {
        const GnW& g = c->gns[c->gindex[name]];
        MAct out;
        double bytes = 0;
        for (int p = 0; p < P; ++p) {
            out[p] = in[p];
            out[p].p = pr[p].w.act[i];
            out[p].part = nullptr;
            out[p].part_S = 0;
            bytes += 2.0 * (double)in[p].N * in[p].T * in[p].H * in[p].W * in[p].C * c->esize();
        }
        if (err) return out;
        const int e = pbegin();
        if (c->bf16()) {
            GnItem<__nv_bfloat16> it[kMaxConvGroup];
            for (int p = 0; p < P; ++p)
                it[p] = {static_cast<const __nv_bfloat16*>(in[p].p), static_cast<__nv_bfloat16*>(out[p].p),
                         (long long)in[p].N * in[p].T, (long long)in[p].H * in[p].W, pr[p].w.gn, in[p].part,
                         in[p].part_S};
            ck(launch_gn_silu_group<__nv_bfloat16>(it, P, in[0].C, g.G, g.g, g.b, c->arch.gn_eps, true, s,
                                                   c->d_status));
        } else {
            GnItem<float> it[kMaxConvGroup];
            for (int p = 0; p < P; ++p)
                it[p] = {static_cast<const float*>(in[p].p), static_cast<float*>(out[p].p),
                         (long long)in[p].N * in[p].T, (long long)in[p].H * in[p].W, pr[p].w.gn};
            ck(launch_gn_silu_group<float>(it, P, in[0].C, g.G, g.g, g.b, c->arch.gn_eps, false, s, c->d_status));
        }
        pend(e, 1, bytes, name);
        c->launches += 3;
        const size_t nb = (size_t)in[0].N * in[0].T * in[0].H * in[0].W * in[0].C * c->esize();
        trace(name, in[0].p, nb, nullptr, 0, out[0].p, nb);
        return out;
    }

    // Residual block over the act slots: ix holds X; three temporaries.
    int block(const std::string& name, int ix, MAct& X) {
        int t[4], k = 0;
        for (int i = 0; i < 5 && k < 4; ++i)
            if (i != ix) t[k++] = i;
        const int iA = t[0], iH = t[1], iS = t[2], iY = t[3];
        MAct A = gn_silu(name + ".gn1", X, iA);
        MAct H = conv_slot(name + ".c1", A, iH);
        MAct A2 = gn_silu(name + ".gn2", H, iA);
        MAct res = X;
        if (c->cindex.count(name + ".sc")) res = conv_slot(name + ".sc", X, iS);
        X = conv_slot(name + ".c2", A2, iY, &res);
        return iY;
    }

    static int other_slot(int ix) { return ix == 0 ? 1 : 0; }

    const __nv_bfloat16* stream_hist_pixels(int p, GatherGeo& g, const char* name) {
        if (!pr[p].st || pr[p].chunk0) return nullptr;
        g.hist_T = 2;
        return reinterpret_cast<const __nv_bfloat16*>(pr[p].st->hist[name]);
    }

    // Pixel input of the first conv: the BF16 path gathers the im2col matrix
    // (stride (t_stem, 2, 2) for the stem, 1 for the single stage); the FP32
    // path edge-pads. A stem with temporal stride 2 sees a stream's later
    // chunks start one frame after an output frame, as the stride-2 convs do.
    MAct first_input(const char* name, const void* const* x, const int* N, const int* T, const int* H, const int* W,
                     int stride_hw, int stride_t, const bool* skip = nullptr) {
        MAct dims;
        for (int p = 0; p < P; ++p) {
            if (skip && skip[p]) continue;
            const Dims d = clip_dims(c, T[p], H[p], W[p]);
            if (c->bf16()) {
                GatherGeo g = gather_pixels(N[p], T[p], H[p], W[p], d.Hp, d.Wp, stride_hw);
                g.st = stride_t;
                g.Tout = (T[p] - 1) / stride_t + 1;
                const __nv_bfloat16* ph = stream_hist_pixels(p, g, name);
                if (ph && stride_t == 2) g.t_off = -1;
                other([&] { return launch_im2col_pixels(static_cast<const __nv_bfloat16*>(x[p]), ph, g,
                                                        reinterpret_cast<__nv_bfloat16*>(pr[p].w.gather), s); },
                      gather_bytes(g));
                stream_update(p, name, x[p], T[p]);
                dims[p] = Act{nullptr, N[p], g.Tout, d.Hp / stride_hw, d.Wp / stride_hw, 0};
            } else {
                float* P_ = reinterpret_cast<float*>(pr[p].w.gather);
                const float* xs = static_cast<const float*>(x[p]);
                if (d.Hp == H[p] && d.Wp == W[p]) {
                    dims[p] = Act{const_cast<float*>(xs), N[p], T[p], H[p], W[p], c->arch.in_ch};
                } else {
                    other([&] { return launch_edge_pad<float>(xs, (long long)N[p] * T[p], H[p], W[p], d.Hp, d.Wp,
                                                              c->arch.in_ch, P_, s); },
                          (double)N[p] * T[p] * (H[p] * W[p] + d.Hp * d.Wp) * c->arch.in_ch * 4);
                    dims[p] = Act{P_, N[p], T[p], d.Hp, d.Wp, c->arch.in_ch};
                }
            }
        }
        return dims;
    }

    // BF16 stem with its im2col rows formed on chip (one launch, no gather pass)
    // for the problems whose frame needs no edge extension: done[p] marks them
    // (the others take the im2col gather and the 1x1x1 conv), so that a problem
    // takes the same path in a group as alone. A stream's later chunks read the
    // two frames before them from its history, as the gather does.
    void stem_fused(const char* name, const void* const* x, const int* N, const int* T, const int* H, const int* W,
                    int stride_t, void* const* outs, MAct* X, bool* done) {
        for (int p = 0; p < P; ++p) done[p] = false;
        if (!c->bf16()) return;
        const ConvW& cw = c->convs[c->cindex[name]];
        StemArgs as[kMaxConvGroup];
        int at[kMaxConvGroup];
        int n = 0;
        for (int p = 0; p < P; ++p) {
            const Dims d = clip_dims(c, T[p], H[p], W[p]);
            if (d.Hp != H[p] || d.Wp != W[p]) continue;
            GatherGeo g = gather_pixels(N[p], T[p], H[p], W[p], d.Hp, d.Wp, 2);
            const __nv_bfloat16* ph = stream_hist_pixels(p, g, name);
            as[n] = stem_args(cw, x[p], ph, N[p], T[p], H[p], W[p], stride_t, ph && stride_t == 2 ? -1 : -2, outs[p],
                              pr[p].w);
            if (!stem_tc_accepts(&as[n], 1)) continue;
            at[n++] = p;
        }
        if (!n || !stem_launch(as, n, cw, at[0] == 0)) return;
        for (int i = 0; i < n; ++i) {
            const int p = at[i];
            stream_update(p, name, x[p], T[p]);
            (*X)[p] = stem_out(as[i]);
            done[p] = true;
        }
    }

    // Last encoder conv: latent z (fp32) and FSQ token indices.
    void out_conv(const std::string& name, const MAct& A, float* const* z, int32_t* const* idx) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs as[kMaxConvGroup];
        for (int p = 0; p < P; ++p) {
            ConvArgs& a = as[p];
            a = base_args(cw, A[p], 1, 1, 1);
            stream_args(p, a, name, cw.k, 1);
            a.out = z[p];
            a.oT = a.Tout;
            a.oH = a.Hout;
            a.oW = a.Wout;
            a.oC = cw.Cout;
            if (c->bf16()) {
                a.mode = OUT_FSQ;
                a.idx = idx[p];
            } else {
                a.mode = OUT_PLAIN;
                a.out_fp32 = 1;
            }
        }
        launch_group(as, cw);
        if (!c->bf16())
            for (int p = 0; p < P; ++p) {
                if (!idx[p]) continue;
                const long long ntok = (long long)A[p].N * as[p].Tout * as[p].Hout * as[p].Wout;
                other([&] { return launch_fsq(z[p], ntok, c->fsq, idx[p], nullptr, s); },
                      (double)ntok * (4 * cw.Cout + 4));
            }
        for (int p = 0; p < P; ++p) stream_update(p, name, A[p].p, A[p].T);
    }

    // ---------------------------------------------------------------- encode
    void encode(const void* const* x, const int* N, const int* T, const int* H, const int* W, float* const* z_in,
                int32_t* const* idx) {
        const tok_arch& ar = c->arch;
        float* z[kMaxConvGroup];
        for (int p = 0; p < P; ++p) z[p] = z_in[p] ? z_in[p] : reinterpret_cast<float*>(pr[p].w.zbuf);
        void* s0[kMaxConvGroup];
        slot(0, s0);
        int ix = 0;
        MAct X;
        if (ar.kind == TOK_ARCH_STAGE) {
            MAct in = first_input("stage.c0", x, N, T, H, W, 1, 1);
            if (c->bf16())
                X = conv_gathered("stage.c0", in, s0, OUT_PLAIN, nullptr);
            else
                X = conv("stage.c0", in, s0);
            MAct Y = conv_slot("stage.c1", X, 1, nullptr, 1, 2, 2);
            MAct A = gn_silu("stage.gn", Y, 2);
            out_conv("stage.out", A, z, idx);
            return;
        }
        bool fused[kMaxConvGroup];
        stem_fused("enc.stem", x, N, T, H, W, ar.t_stem, s0, &X, fused);
        int nf = 0;
        for (int p = 0; p < P; ++p) nf += fused[p] ? 1 : 0;
        if (nf < P) {
            MAct in = first_input("enc.stem", x, N, T, H, W, 2, ar.t_stem, fused);
            if (c->bf16()) {
                const MAct G = conv_gathered("enc.stem", in, s0, OUT_PLAIN, nullptr, fused);
                for (int p = 0; p < P; ++p)
                    if (!fused[p]) X[p] = G[p];
            } else {
                X = conv("enc.stem", in, s0, nullptr, ar.t_stem, 2, 2);
            }
        }
        for (int l = 0; l < ar.nlevels; ++l) {
            for (int b = 0; b < ar.blocks; ++b) ix = block("enc.l" + std::to_string(l) + ".b" + std::to_string(b), ix, X);
            if (l < ar.nlevels - 1) {
                const int iy = other_slot(ix);
                X = conv_slot("enc.down" + std::to_string(l), X, iy, nullptr, 2, 2, 2);
                ix = iy;
            }
        }
        MAct A = gn_silu("enc.out_gn", X, other_slot(ix));
        out_conv("enc.out", A, z, idx);
    }

    // ---------------------------------------------------------------- decode
    void decode(const int32_t* const* idx, const int* N, const int* Tq, const int* Hq, const int* Wq, const int* H,
                const int* W, float* const* xhat) {
        const tok_arch& ar = c->arch;
        void* s0[kMaxConvGroup];
        slot(0, s0);
        int ix = 0;
        MAct X;
        if (c->bf16()) {
            MAct dims;
            for (int p = 0; p < P; ++p) {
                GatherGeo g;
                memset(&g, 0, sizeof(g));
                g.N = N[p];
                g.Tin = Tq[p];
                g.H = g.Hp = Hq[p];
                g.W = g.Wp = Wq[p];
                g.Cin = ar.nlev;
                g.hist_T = 0;
                g.Tout = Tq[p];
                g.Hout = Hq[p];
                g.Wout = Wq[p];
                g.kt = g.kh = g.kw = 3;
                g.st = g.sh = g.sw = 1;
                g.t_off = -2;
                g.pad_mode = ar.time_pad;
                g.Kpad = round_up(27 * ar.nlev, 64);
                const int32_t* th = nullptr;
                if (pr[p].st && !pr[p].chunk0) {
                    th = reinterpret_cast<const int32_t*>(pr[p].st->hist["dec.in"]);
                    g.hist_T = 2;
                }
                other([&] { return launch_im2col_tokens(idx[p], th, g, c->fsq,
                                                        reinterpret_cast<__nv_bfloat16*>(pr[p].w.gather), s); },
                      gather_bytes(g));
                stream_update(p, "dec.in", idx[p], Tq[p], true);
                dims[p] = Act{nullptr, N[p], Tq[p], Hq[p], Wq[p], 0};
            }
            X = conv_gathered("dec.in", dims, s0, OUT_PLAIN, nullptr);
        } else {
            MAct in;
            for (int p = 0; p < P; ++p) {
                float* codes = reinterpret_cast<float*>(pr[p].w.zbuf);
                const long long nt = (long long)N[p] * Tq[p] * Hq[p] * Wq[p];
                other([&] { return launch_dequant(idx[p], nt, c->fsq, codes, s); }, (double)nt * (4 + 4 * ar.nlev));
                in[p] = Act{codes, N[p], Tq[p], Hq[p], Wq[p], ar.nlev};
            }
            X = conv("dec.in", in, s0);
        }
        for (int l = ar.nlevels - 1; l >= 0; --l) {
            for (int b = 0; b < ar.blocks; ++b) ix = block("dec.l" + std::to_string(l) + ".b" + std::to_string(b), ix, X);
            if (l > 0) {
                const int iy = other_slot(ix);
                void* o[kMaxConvGroup];
                slot(iy, o);
                int oh[kMaxConvGroup], ow[kMaxConvGroup];
                for (int p = 0; p < P; ++p) {
                    oh[p] = X[p].H * 2;
                    ow[p] = X[p].W * 2;
                }
                X = conv_d2s("dec.up" + std::to_string(l - 1), X, o, 2, 2, 2, oh, ow, false);
                ix = iy;
            }
        }
        MAct A = gn_silu("dec.out_gn", X, other_slot(ix));
        void* o[kMaxConvGroup];
        for (int p = 0; p < P; ++p) o[p] = xhat[p];
        conv_d2s("dec.out", A, o, ar.t_stem, 2, 2, H, W, true, true);
    }
};

}  // namespace
}  // namespace tok
