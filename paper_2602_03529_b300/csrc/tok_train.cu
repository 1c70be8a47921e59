// Training step of the tokenizer: forward with kept block inputs, MSE loss,
// and the hand-written backward (see include/tok.h, "Training").
//
// Backward per residual block y = skip(x) + c2(SiLU(GN2(c1(SiLU(GN1(x)))))):
// A1 = SiLU(GN1(x)), H = c1(A1), A2 = SiLU(GN2(H)) are either kept from the
// forward (TOK_TRAIN_KEEP) or rebuilt from the kept x and the kept GroupNorm
// statistics (TOK_TRAIN_RECOMPUTE: the apply pass with the forward's mean and
// rstd, then c1 on the same kernel and tile as the forward, so the rebuilt
// tensors are bitwise the forward's); then dW(c2), dA2 = c2^T(dy);
// dH = GN2^T(dA2); dW(c1), dA1 = c1^T(dH); dx = GN1^T(dA1) + skip^T(dy). Input gradients of convs (c^T) run on the
// same conv kernels as the forward with flipped/transposed weights reading
// ahead in time; stride-2 convs see dY spread onto their input grid; under
// replicate padding a two-tap correction adds the clamped taps into frame 0.
// Weight gradients use the split-K kernel of k_backward.cu.
#include <array>

#include "tok_internal.h"

namespace {

struct TrainBufs {
    std::vector<char*> enc[4];  // per level: inputs of blocks 0..B-1, then the level output
    std::vector<char*> dec[4];
    float* z = nullptr;
    int32_t* idx = nullptr;
    int32_t* idx_d = nullptr;
    uint32_t* keep = nullptr;
    char* codes = nullptr;
    char* dz = nullptr;
    char* dcodes = nullptr;
    char* R1 = nullptr;
    char* R2 = nullptr;
    char* R3 = nullptr;
    char* GA = nullptr;
    char* GB = nullptr;
    char* G3 = nullptr;
    char* G4 = nullptr;
    char* Z = nullptr;
    char* gather = nullptr;
    char* gn = nullptr;
    char* gnb = nullptr;
    char* gnpart = nullptr;  // GroupNorm statistics reduced by the forward convs
    size_t gnpart_bytes = 0;
    // kept from the forward for the backward: per residual block its GN1 output,
    // first conv output and GN2 output (TOK_TRAIN_KEEP only); the output
    // GroupNorms' outputs; and every GroupNorm's scratch, which holds the
    // (mean, rstd) its backward (and a recomputation) reuses
    bool keep_blocks = false;
    std::map<std::string, std::array<char*, 3>> blk;
    std::map<std::string, char*> gn_out;
    std::map<std::string, char*> gn_sc;
    float* wpart = nullptr;
    size_t wpart_floats = 0;
    float* mse = nullptr;
    size_t total = 0;
};

constexpr size_t kMaxWgradPartialFloats = 64ull << 20;  // 256 MB of split-K partials

int adj_cpad(const tok_ctx* c, int Cout) { return c->bf16() ? round_up(Cout, 64) : round_up(Cout, 8); }
int adj_rows(const tok_ctx* c, int Cin) {
    if (!c->bf16()) return round_up(Cin, 16);
    const int c16 = round_up(Cin, 16);
    return conv_tc_cout_pad(c16);
}

// Bump layout of the training workspace; base == nullptr only sizes it.
TrainBufs train_layout(const tok_ctx* c, int N, int T, int H, int W, char* base, int mode) {
    TrainBufs b;
    b.keep_blocks = mode == TOK_TRAIN_KEEP;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const tok_arch& a = c->arch;
    const size_t es = c->esize();
    const int L = a.nlevels;
    int Tl[4];
    Tl[0] = stem_frames(c, T);
    for (int l = 1; l < L; ++l) Tl[l] = (Tl[l - 1] - 1) / 2 + 1;
    auto vox = [&](int l) { return (size_t)N * Tl[l] * (H >> (l + 1)) * (W >> (l + 1)); };
    size_t work = 0, gn = 0;
    for (int l = 0; l < L; ++l) {
        const int cin0 = l > 0 ? a.ch[l - 1] : a.ch[0];
        for (int k = 0; k <= a.blocks; ++k) {
            const int C = (k == 0) ? cin0 : a.ch[l];
            b.enc[l].push_back(take(vox(l) * C * es));
        }
        for (int k = 0; k <= a.blocks; ++k) b.dec[l].push_back(take(vox(l) * a.ch[l] * es));
        work = std::max(work, vox(l) * std::max(a.ch[l], cin0) * es);
        if (l > 0) work = std::max(work, vox(l) * 8 * a.ch[l - 1] * es);
        const int G = std::max(1, std::min(a.gn_groups, a.ch[l] / 2));
        gn = std::max(gn, gn_scratch_bytes((long long)N * Tl[l], (long long)(H >> (l + 1)) * (W >> (l + 1)),
                                           a.ch[l], G, c->num_sms, c->bf16() ? 8 : 4));
        {
            const long long hw = (long long)(H >> (l + 1)) * (W >> (l + 1));
            const int cmax = std::max(a.ch[l], cin0), vec = c->bf16() ? 8 : 4;
            const int smax =
                std::max(gn_bwd_chunks_per_frame(hw, a.ch[l], vec), gn_bwd_chunks_per_frame(hw, cin0, vec));
            gn = std::max(gn, gn_bwd_scratch_bytes((long long)N * Tl[l], smax, cmax, std::max(a.gn_groups, 1)));
        }
        if (l > 0) {
            const int G2 = std::max(1, std::min(a.gn_groups, cin0 / 2));
            gn = std::max(gn, gn_scratch_bytes((long long)N * Tl[l], (long long)(H >> (l + 1)) * (W >> (l + 1)),
                                               cin0, G2, c->num_sms, c->bf16() ? 8 : 4));
        }
    }
    work = std::max(work, vox(0) * (size_t)adj_cpad(c, a.in_ch * 4 * a.t_stem) * es);
    // per-layer keeps of the forward
    {
        const int vec = c->bf16() ? 8 : 4;
        auto gn_keep = [&](const std::string& name, int l, int C) {
            const int G = std::max(1, std::min(a.gn_groups, C / 2));
            b.gn_sc[name] = take(gn_scratch_bytes((long long)N * Tl[l], (long long)(H >> (l + 1)) * (W >> (l + 1)), C,
                                                  G, c->num_sms, vec));
        };
        for (int side = 0; side < 2; ++side)
            for (int l = 0; l < L; ++l)
                for (int k = 0; k < a.blocks; ++k) {
                    const std::string nm = std::string(side ? "dec.l" : "enc.l") + std::to_string(l) + ".b" +
                                           std::to_string(k);
                    const int cin = (!side && k == 0) ? (l > 0 ? a.ch[l - 1] : a.ch[0]) : a.ch[l];
                    if (b.keep_blocks)
                        b.blk[nm] = {take(vox(l) * cin * es), take(vox(l) * a.ch[l] * es),
                                     take(vox(l) * a.ch[l] * es)};
                    gn_keep(nm + ".gn1", l, cin);
                    gn_keep(nm + ".gn2", l, a.ch[l]);
                }
        b.gn_out["enc.out_gn"] = take(vox(L - 1) * a.ch[L - 1] * es);
        gn_keep("enc.out_gn", L - 1, a.ch[L - 1]);
        b.gn_out["dec.out_gn"] = take(vox(0) * a.ch[0] * es);
        gn_keep("dec.out_gn", 0, a.ch[0]);
    }
    const size_t ntok = (size_t)N * Tl[L - 1] * (H >> L) * (W >> L);
    b.z = reinterpret_cast<float*>(take(ntok * a.nlev * 4));
    b.idx = reinterpret_cast<int32_t*>(take(ntok * 4));
    b.idx_d = reinterpret_cast<int32_t*>(take(ntok * 4));
    b.keep = reinterpret_cast<uint32_t*>(take(ntok * 4));
    b.codes = take(ntok * a.nlev * es);
    b.dz = take(ntok * adj_cpad(c, a.nlev) * es);
    b.dcodes = take(ntok * adj_rows(c, a.nlev) * es);
    b.R1 = take(work);
    b.R2 = take(work);
    b.R3 = take(work);
    b.GA = take(work);
    b.GB = take(work);
    b.G3 = take(work);
    b.G4 = take(work);
    b.Z = take(work);
    size_t g = (size_t)N * Tl[0] * (H / 2) * (W / 2) * round_up(27 * a.in_ch, 64) * 2;
    g = std::max(g, ntok * (size_t)round_up(27 * a.nlev, 64) * 2);
    b.gather = take(c->bf16() ? g : 256);
    b.gn = take(gn);
    b.gnb = take(gn);
    b.gnpart_bytes = gnpart_bytes(c, N, T, H, W);
    b.gnpart = b.gnpart_bytes ? take(b.gnpart_bytes) : nullptr;
    b.wpart_floats = kMaxWgradPartialFloats;
    b.wpart = reinterpret_cast<float*>(take(b.wpart_floats * 4));
    b.mse = reinterpret_cast<float*>(take(4096));
    b.total = off;
    return b;
}

struct TrainExec : Exec {
    TrainBufs b;
    float* grads = nullptr;  // flat dL/dparams

    TrainExec() { any_tile = true; }

    void set_work() {
        w.gather = b.gather;
        w.gn = b.gn;
        w.gnpart = b.gnpart;
        w.gnpart_bytes = b.gnpart_bytes;
        w.zbuf = b.codes;
        for (int i = 0; i < 5; ++i) w.act[i] = nullptr;
    }

    // GroupNorm+SiLU whose scratch (and so its statistics) is kept for the backward.
    Act gn_kept(const std::string& name, const Act& X, void* out) {
        char* keep = w.gn;
        w.gn = b.gn_sc.at(name);
        Act A = gn_silu(name, X, out);
        w.gn = keep;
        return A;
    }

    // Residual block forward into `out`; the GN1 output, first conv output and GN2
    // output go to kept buffers (TOK_TRAIN_KEEP) or to work buffers.
    Act block_fwd(const std::string& name, const Act& X, void* out) {
        std::array<char*, 3> kb = {b.R1, b.R2, b.R1};
        if (b.keep_blocks) kb = b.blk.at(name);
        Act A1 = gn_kept(name + ".gn1", X, kb[0]);
        Act H = conv(name + ".c1", A1, kb[1]);
        Act A2 = gn_kept(name + ".gn2", H, kb[2]);
        const void* res = X.p;
        if (c->cindex.count(name + ".sc")) res = conv(name + ".sc", X, b.R3).p;
        return conv(name + ".c2", A2, out, res);
    }

    void forward(const void* x, int N, int T, int H, int W, float rate, uint64_t seed, uint64_t step,
                 const uint32_t* keep_in, float* xhat, float* loss, float* dxhat) {
        const tok_arch& ar = c->arch;
        const int L = ar.nlevels;
        Act X;
        const StemArgs sa = stem_args(c->convs[c->cindex["enc.stem"]], x, nullptr, N, T, H, W, ar.t_stem, -2,
                                      b.enc[0][0], w);
        if (stem_launch(&sa, 1, c->convs[c->cindex["enc.stem"]])) {
            X = stem_out(sa);
        } else if (c->bf16()) {
            const GatherGeo g = stem_geo(N, T, H, W);
            other([&] { return launch_im2col_pixels(static_cast<const __nv_bfloat16*>(x), nullptr, g,
                                                    reinterpret_cast<__nv_bfloat16*>(w.gather), s); },
                  gather_bytes(g));
            X = conv_gathered("enc.stem", N, g.Tout, H / 2, W / 2, b.enc[0][0], OUT_PLAIN, nullptr);
        } else {
            X = conv("enc.stem", Act{const_cast<void*>(x), N, T, H, W, ar.in_ch}, b.enc[0][0], nullptr, ar.t_stem, 2,
                     2);
        }
        for (int l = 0; l < L; ++l) {
            for (int k = 0; k < ar.blocks; ++k)
                X = block_fwd("enc.l" + std::to_string(l) + ".b" + std::to_string(k), X, b.enc[l][k + 1]);
            if (ar.blocks == 0) X.p = b.enc[l][0];
            if (l < L - 1) X = conv("enc.down" + std::to_string(l), X, b.enc[l + 1][0], nullptr, 2, 2, 2);
        }
        Act A = gn_kept("enc.out_gn", X, b.gn_out.at("enc.out_gn"));
        out_conv("enc.out", A, b.z, b.idx);
        const int Tq = X.T, Hq = X.H, Wq = X.W;
        const long long ntok = (long long)N * Tq * Hq * Wq;
        if (keep_in) {
            const size_t kb = (size_t)N * Tq * Hq * ((Wq + 31) / 32) * 4;
            if (cudaMemcpyAsync(b.keep, keep_in, kb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ck(1);
            other([&] { return launch_apply_keep(b.idx, b.keep, ntok, Wq, zero_index_of(c), b.idx_d, s); },
                  (double)ntok * 8);
        } else {
            double r = std::min(1.0, std::max(0.0, (double)rate));
            const unsigned long long thr = (unsigned long long)std::floor(r * 4294967296.0);
            other([&] { return launch_drop(b.idx, N, Tq, Hq, Wq, thr, seed, 0, step, zero_index_of(c), b.idx_d,
                                           b.keep, s); },
                  (double)ntok * 8);
        }
        // decoder input: codes of the kept tokens
        if (c->bf16()) {
            other([&] { return launch_codes<__nv_bfloat16>(b.idx_d, ntok, c->fsq,
                                                           reinterpret_cast<__nv_bfloat16*>(b.codes), s); },
                  (double)ntok * (4 + 2 * ar.nlev));
            const GatherGeo g = dec_in_geo(N, Tq, Hq, Wq);
            other([&] { return launch_im2col_tokens(b.idx_d, nullptr, g, c->fsq,
                                                    reinterpret_cast<__nv_bfloat16*>(w.gather), s); },
                  gather_bytes(g));
            X = conv_gathered("dec.in", N, Tq, Hq, Wq, b.dec[L - 1][0], OUT_PLAIN, nullptr);
        } else {
            other([&] { return launch_codes<float>(b.idx_d, ntok, c->fsq, reinterpret_cast<float*>(b.codes), s); },
                  (double)ntok * (4 + 4 * ar.nlev));
            X = conv("dec.in", Act{b.codes, N, Tq, Hq, Wq, ar.nlev}, b.dec[L - 1][0]);
        }
        for (int l = L - 1; l >= 0; --l) {
            for (int k = 0; k < ar.blocks; ++k)
                X = block_fwd("dec.l" + std::to_string(l) + ".b" + std::to_string(k), X, b.dec[l][k + 1]);
            if (ar.blocks == 0) X.p = b.dec[l][0];
            if (l > 0) X = conv_d2s("dec.up" + std::to_string(l - 1), X, b.dec[l - 1][0], 2, 2, 2, X.H * 2, X.W * 2,
                                    false);
        }
        A = gn_kept("dec.out_gn", X, b.gn_out.at("dec.out_gn"));
        conv_d2s("dec.out", A, xhat, ar.t_stem, 2, 2, H, W, true);
        const long long n = (long long)N * T * H * W * ar.in_ch;
        if (c->bf16())
            other([&] { return launch_mse<__nv_bfloat16>(xhat, static_cast<const __nv_bfloat16*>(x), n, dxhat, loss,
                                                         b.mse, s); },
                  (double)n * 10, 2);
        else
            other([&] { return launch_mse<float>(xhat, static_cast<const float*>(x), n, dxhat, loss, b.mse, s); },
                  (double)n * 12, 2);
    }

    // im2col geometry of the stem (3x3x3, stride (t_stem, 2, 2) over the pixels)
    GatherGeo stem_geo(int N, int T, int H, int W) {
        GatherGeo g = gather_pixels(N, T, H, W, H, W, 2);
        g.st = c->arch.t_stem;
        g.Tout = stem_frames(c, T);
        return g;
    }

    // im2col geometry of the decoder input conv (3x3x3 over the token codes)
    GatherGeo dec_in_geo(int N, int Tq, int Hq, int Wq) const {
        GatherGeo g;
        memset(&g, 0, sizeof(g));
        g.N = N;
        g.Tin = Tq;
        g.H = g.Hp = Hq;
        g.W = g.Wp = Wq;
        g.Cin = c->arch.nlev;
        g.hist_T = 0;
        g.Tout = Tq;
        g.Hout = Hq;
        g.Wout = Wq;
        g.kt = g.kh = g.kw = 3;
        g.st = g.sh = g.sw = 1;
        g.t_off = -2;
        g.pad_mode = c->arch.time_pad;
        g.Kpad = round_up(27 * c->arch.nlev, 64);
        return g;
    }

    // ------------------------------------------------------------ backward

    // Weight gradient of a layer whose forward ran on an im2col matrix (BF16
    // stem and decoder input): the same matrix is rebuilt in the gather
    // buffer and the gradient is that of a 1x1x1 conv over its Kpad columns,
    // of which the first 27 * Cin are the weights.
    void wgrad_gathered(const std::string& name, const Act& dy, int Cdy, int Kpad) {
        if (err) return;
        const ConvW& cw = c->convs[c->cindex[name]];
        WgradArgs a;
        memset(&a, 0, sizeof(a));
        a.N = dy.N;
        a.Tin = a.Tout = dy.T;
        a.Hin = a.Hout = dy.H;
        a.Win = a.Wout = dy.W;
        a.Cin = Kpad;
        a.Cout = cw.Cout;
        a.Cdy = Cdy;
        a.kt = a.kh = a.kw = 1;
        a.st = a.sh = a.sw = 1;
        a.t_off = 0;
        a.pad_mode = c->arch.time_pad;
        a.K = Kpad;
        a.V = (long long)dy.N * dy.T * dy.H * dy.W;
        const int kv = cw.k * cw.k * cw.k * cw.Cin;
        if (!wgrad_tc_ok(a) || kv > Kpad) {
            ck(TOK_ESHAPE);
            return;
        }
        const int e = pbegin();
        ck(launch_wgrad_tc(static_cast<const __nv_bfloat16*>(dy.p), reinterpret_cast<const __nv_bfloat16*>(w.gather),
                           a, b.wpart, b.wpart_floats, grads + cw.ow, grads + cw.ob, c->num_sms, c->d_status, kWaitNs,
                           s, kv));
        pend(e, 0, 2.0 * (double)a.V * a.Cout * kv, name + ".wgrad");
        c->launches += 4;
        trace(name + ".wgrad", nullptr, 0, dy.p, (size_t)a.V * Cdy * c->esize(), nullptr, 0);
    }

    void wgrad(const std::string& name, const Act& dy, int Cdy, const Act& xin, int tst, int ss) {
        if (err) return;
        const ConvW& cw = c->convs[c->cindex[name]];
        WgradArgs a;
        memset(&a, 0, sizeof(a));
        a.N = xin.N;
        a.Tin = xin.T;
        a.Hin = xin.H;
        a.Win = xin.W;
        a.Cin = cw.Cin;
        a.Tout = dy.T;
        a.Hout = dy.H;
        a.Wout = dy.W;
        a.Cout = cw.Cout;
        a.Cdy = Cdy;
        a.kt = a.kh = a.kw = cw.k;
        a.st = tst;
        a.sh = a.sw = ss;
        a.t_off = -(cw.k - 1);
        a.pad_mode = c->arch.time_pad;
        a.K = cw.k * cw.k * cw.k * cw.Cin;
        a.V = (long long)dy.N * dy.T * dy.H * dy.W;
        const int S = wgrad_splits(a, c->num_sms, b.wpart_floats);
        const double flop = 2.0 * (double)a.V * a.Cout * a.K;
        const int e = pbegin();
        const bool tc = c->bf16() && wgrad_tc_ok(a);
        if (tc)
            ck(launch_wgrad_tc(static_cast<const __nv_bfloat16*>(dy.p), static_cast<const __nv_bfloat16*>(xin.p), a,
                               b.wpart, b.wpart_floats, grads + cw.ow, grads + cw.ob, c->num_sms, c->d_status,
                               kWaitNs, s));
        else if (c->bf16())
            ck(launch_wgrad<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(dy.p),
                                           static_cast<const __nv_bfloat16*>(xin.p), a, S, b.wpart, grads + cw.ow,
                                           grads + cw.ob, s));
        else
            ck(launch_wgrad<float>(static_cast<const float*>(dy.p), static_cast<const float*>(xin.p), a, S, b.wpart,
                                   grads + cw.ow, grads + cw.ob, s));
        pend(e, 0, flop, name + ".wgrad");
        c->launches += tc ? 4 : 2;
        const size_t es = c->esize();
        trace(name + ".wgrad", xin.p, (size_t)xin.N * xin.T * xin.H * xin.W * cw.Cin * es, dy.p,
              (size_t)a.V * Cdy * es, nullptr, 0);
    }

    // Input gradient of a stride-1 conv: the adjoint conv over dY (cpad
    // channels) into `out` (rows_pad channels), plus the frame-0 correction.
    Act dgrad(const std::string& name, const Act& dy, void* out) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs a;
        memset(&a, 0, sizeof(a));
        a.x = dy.p;
        a.N = dy.N;
        a.Tin = dy.T;
        a.Hin = dy.H;
        a.Win = dy.W;
        a.Cin = cw.cpad;
        a.w = cw.wt;
        a.bias = nullptr;
        a.Cout = cw.rows_pad;
        a.Cout_pad = cw.rows_pad;
        a.kt = a.kh = a.kw = cw.k;
        a.Kpad = c->bf16() ? cw.k * cw.k * cw.k * cw.cpad : round_up(cw.k * cw.k * cw.k * cw.cpad, 8);
        a.st = a.sh = a.sw = 1;
        a.t_off = 0;  // reads frames t .. t+k-1 of dY (zeros past the end)
        a.pad_mode = c->arch.time_pad;
        a.Tout = dy.T;
        a.Hout = dy.H;
        a.Wout = dy.W;
        a.mode = OUT_PLAIN;
        a.out = out;
        a.oT = dy.T;
        a.oH = dy.H;
        a.oW = dy.W;
        a.oC = cw.rows_pad;
        a.status = c->d_status;
        a.wait_ns = kWaitNs;
        a.fsq = c->fsq;
        a.fsq_thr = c->d_fsq_thr;
        ConvW shadow = cw;
        shadow.Cin = cw.cpad;
        shadow.Cout = cw.rows_pad;
        shadow.name = name + ".dgrad";
        // BF16: the tiles of output frame 0 read their own taps, which fold in the
        // replicate-pad correction (input frame 0 stood for the two padded frames)
        const bool fold = c->bf16() && cw.k == 3 && c->arch.time_pad == TOK_PAD_REPLICATE && cw.wf0;
        if (fold) a.w0 = cw.wf0;
        launch(a, shadow);
        if (!fold && cw.k == 3 && c->arch.time_pad == TOK_PAD_REPLICATE) {
            // taps of output frames 0 (dt = 0, 1) and 1 (dt = 0) that were clamped to frame 0
            ConvArgs b2 = a;
            b2.w = cw.wc;
            b2.kt = 2;
            b2.Kpad = c->bf16() ? 2 * 9 * cw.cpad : round_up(2 * 9 * cw.cpad, 8);
            b2.Tout = 1;
            b2.residual = out;
            ConvW sh2 = shadow;
            sh2.name = name + ".dgrad0";
            launch(b2, sh2);
        }
        const size_t nb = (size_t)dy.N * dy.T * dy.H * dy.W * c->esize();
        trace(name + ".dgrad", dy.p, nb * cw.cpad, nullptr, 0, out, nb * cw.rows_pad);
        return Act{out, dy.N, dy.T, dy.H, dy.W, cw.rows_pad};
    }

    // GN+SiLU backward: dx = GN^T(SiLU^T(dy)) [+ add], parameter gradients into `grads`.
    void gn_bwd(const std::string& name, const Act& x, const void* dy, const void* add, void* dx) {
        if (err) return;
        const GnW& g = c->gns[c->gindex[name]];
        const long long frames = (long long)x.N * x.T, HW = (long long)x.H * x.W;
        // the forward's statistics, kept in this GroupNorm's scratch
        const int vec = c->bf16() ? 8 : 4;
        const float2* stats = gn_stats_of_scratch(b.gn_sc.at(name), frames, HW, x.C, g.G, vec);
        const int vpt = gn_bwd_vectors_per_thread(), S = gn_bwd_chunks_per_frame(HW, x.C, vec);
        const int e = pbegin();
        if (c->bf16()) {
            ck(launch_gn_silu_bwd<__nv_bfloat16>(
                static_cast<const __nv_bfloat16*>(x.p), static_cast<const __nv_bfloat16*>(dy), stats, g.g, g.b,
                static_cast<const __nv_bfloat16*>(add), frames, HW, x.C, g.G, vpt, S, b.gnb, grads + g.og,
                grads + g.ob, static_cast<__nv_bfloat16*>(dx), c->d_status, kWaitNs, s));
        } else {
            ck(launch_gn_silu_bwd<float>(static_cast<const float*>(x.p), static_cast<const float*>(dy), stats, g.g,
                                         g.b, static_cast<const float*>(add), frames, HW, x.C, g.G, vpt, S, b.gnb,
                                         grads + g.og, grads + g.ob, static_cast<float*>(dx), c->d_status, kWaitNs,
                                         s));
        }
        pend(e, 1, 4.0 * (double)frames * HW * x.C * c->esize(), name + ".bwd");
        c->launches += 5;
    }

    // GroupNorm+SiLU of X with the statistics its forward launch kept (apply pass only).
    void gn_apply_kept(const std::string& name, const Act& X, void* out) {
        if (err) return;
        const GnW& g = c->gns[c->gindex[name]];
        const long long frames = (long long)X.N * X.T, HW = (long long)X.H * X.W;
        const int e = pbegin();
        if (c->bf16())
            ck(launch_gn_apply_kept<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(X.p),
                                                   static_cast<__nv_bfloat16*>(out), frames, HW, X.C, g.G, g.g, g.b,
                                                   b.gn_sc.at(name), true, s, c->d_status));
        else
            ck(launch_gn_apply_kept<float>(static_cast<const float*>(X.p), static_cast<float*>(out), frames, HW, X.C,
                                           g.G, g.g, g.b, b.gn_sc.at(name), false, s, c->d_status));
        pend(e, 1, 2.0 * (double)frames * HW * X.C * c->esize(), name + ".recompute");
        c->launches += 1;
    }

    // Block backward; the block-output gradient G is replaced by the block-input gradient.
    void block_bwd(const std::string& name, const Act& X, Act& G) {
        const int Ch = c->convs[c->cindex[name + ".c1"]].Cout;
        std::array<char*, 3> kb = {b.R1, b.R2, b.Z};
        if (b.keep_blocks) {
            kb = b.blk.at(name);
        } else {
            // rebuild the block's interior from its input and the kept statistics; c1
            // runs without the statistics epilogue (its GN2 statistics are kept)
            gn_apply_kept(name + ".gn1", X, kb[0]);
            char* gp = w.gnpart;
            w.gnpart = nullptr;
            conv(name + ".c1", Act{kb[0], X.N, X.T, X.H, X.W, X.C}, kb[1]);
            w.gnpart = gp;
            gn_apply_kept(name + ".gn2", Act{kb[1], X.N, X.T, X.H, X.W, Ch}, kb[2]);
        }
        Act A1{kb[0], X.N, X.T, X.H, X.W, X.C};
        Act H{kb[1], X.N, X.T, X.H, X.W, Ch};
        Act A2{kb[2], X.N, X.T, X.H, X.W, Ch};
        wgrad(name + ".c2", G, G.C, A2, 1, 1);
        Act dA2 = dgrad(name + ".c2", G, b.G3);
        gn_bwd(name + ".gn2", H, dA2.p, nullptr, b.G4);
        Act dH{b.G4, H.N, H.T, H.H, H.W, H.C};
        wgrad(name + ".c1", dH, dH.C, A1, 1, 1);
        Act dA1 = dgrad(name + ".c1", dH, b.G3);
        const void* skip = G.p;
        if (c->cindex.count(name + ".sc")) {
            wgrad(name + ".sc", G, G.C, X, 1, 1);
            skip = dgrad(name + ".sc", G, b.R3).p;
        }
        gn_bwd(name + ".gn1", X, dA1.p, skip, G.p);
        G.C = X.C;
    }

    void backward(const float* dxhat) {
        const tok_arch& ar = c->arch;
        const int L = ar.nlevels;
        const int N = c->train_N, T = c->train_T, H = c->train_H, W = c->train_W;
        int Tl[4];
        Tl[0] = stem_frames(c, T);
        for (int l = 1; l < L; ++l) Tl[l] = (Tl[l - 1] - 1) / 2 + 1;
        auto lev = [&](int l, void* p, int C) { return Act{p, N, Tl[l], H >> (l + 1), W >> (l + 1), C}; };
        char* gcur = b.GA;
        char* galt = b.GB;
        // dec.out: depth-to-space (t_stem,2,2) adjoint of dL/dx_hat (the trimmed
        // first t_stem-1 frames come back as zeros)
        const ConvW& co = c->convs[c->cindex["dec.out"]];
        const int ts = ar.t_stem;
        if (c->bf16())
            other([&] { return launch_s2d<float, __nv_bfloat16>(dxhat, N, T, H, W, ar.in_ch, ts, 2, 2, ts - 1, Tl[0],
                                                                H / 2, W / 2, co.cpad,
                                                                reinterpret_cast<__nv_bfloat16*>(b.Z), s); },
                  (double)N * T * H * W * 6);
        else
            other([&] { return launch_s2d<float, float>(dxhat, N, T, H, W, ar.in_ch, ts, 2, 2, ts - 1, Tl[0], H / 2,
                                                        W / 2, co.cpad, reinterpret_cast<float*>(b.Z), s); },
                  (double)N * T * H * W * 8);
        Act dY = lev(0, b.Z, co.cpad);
        Act X0 = lev(0, b.dec[0][ar.blocks], ar.ch[0]);
        Act A = lev(0, b.gn_out.at("dec.out_gn"), ar.ch[0]);
        wgrad("dec.out", dY, co.cpad, A, 1, 1);
        Act dA = dgrad("dec.out", dY, b.G3);
        gn_bwd("dec.out_gn", X0, dA.p, nullptr, gcur);
        Act G = lev(0, gcur, ar.ch[0]);
        for (int l = 0; l < L; ++l) {
            for (int k = ar.blocks - 1; k >= 0; --k)
                block_bwd("dec.l" + std::to_string(l) + ".b" + std::to_string(k), lev(l, b.dec[l][k], ar.ch[l]), G);
            if (l < L - 1) {
                // dec.up{l}: conv at level l+1 followed by depth-to-space (2,2,2)
                const std::string nm = "dec.up" + std::to_string(l);
                Act Xu = lev(l + 1, b.dec[l + 1][ar.blocks], ar.ch[l + 1]);
                const int C8 = 8 * ar.ch[l];
                if (c->bf16())
                    other([&] { return launch_s2d<__nv_bfloat16, __nv_bfloat16>(
                                    reinterpret_cast<const __nv_bfloat16*>(G.p), N, Tl[l], H >> (l + 1), W >> (l + 1),
                                    ar.ch[l], 2, 2, 2, 1, Tl[l + 1], Xu.H, Xu.W, C8,
                                    reinterpret_cast<__nv_bfloat16*>(b.Z), s); },
                          4.0 * (double)N * Tl[l + 1] * Xu.H * Xu.W * C8);
                else
                    other([&] { return launch_s2d<float, float>(reinterpret_cast<const float*>(G.p), N, Tl[l],
                                                                H >> (l + 1), W >> (l + 1), ar.ch[l], 2, 2, 2, 1,
                                                                Tl[l + 1], Xu.H, Xu.W, C8,
                                                                reinterpret_cast<float*>(b.Z), s); },
                          8.0 * (double)N * Tl[l + 1] * Xu.H * Xu.W * C8);
                Act dU = lev(l + 1, b.Z, C8);
                wgrad(nm, dU, C8, Xu, 1, 1);
                dgrad(nm, dU, galt);
                std::swap(gcur, galt);
                G = lev(l + 1, gcur, ar.ch[l + 1]);
            }
        }
        // dec.in (input: the codes of the kept tokens)
        const int Tq = Tl[L - 1], Hq = H >> L, Wq = W >> L;
        const long long ntok = (long long)N * Tq * Hq * Wq;
        Act codes{b.codes, N, Tq, Hq, Wq, ar.nlev};
        if (c->bf16()) {
            const GatherGeo g = dec_in_geo(N, Tq, Hq, Wq);
            other([&] { return launch_im2col_tokens(b.idx_d, nullptr, g, c->fsq,
                                                    reinterpret_cast<__nv_bfloat16*>(w.gather), s); },
                  gather_bytes(g));
            wgrad_gathered("dec.in", G, G.C, g.Kpad);
        } else {
            wgrad("dec.in", G, G.C, codes, 1, 1);
        }
        const ConvW& di = c->convs[c->cindex["dec.in"]];
        dgrad("dec.in", G, b.dcodes);
        // straight-through FSQ and the drop mask
        const ConvW& eo = c->convs[c->cindex["enc.out"]];
        if (c->bf16())
            other([&] { return launch_ste_bwd<__nv_bfloat16>(reinterpret_cast<const __nv_bfloat16*>(b.dcodes),
                                                             di.rows_pad, b.z, b.keep, ntok, Wq, c->fsq,
                                                             reinterpret_cast<__nv_bfloat16*>(b.dz), eo.cpad, s); },
                  (double)ntok * 64);
        else
            other([&] { return launch_ste_bwd<float>(reinterpret_cast<const float*>(b.dcodes), di.rows_pad, b.z,
                                                     b.keep, ntok, Wq, c->fsq, reinterpret_cast<float*>(b.dz), eo.cpad,
                                                     s); },
                  (double)ntok * 64);
        Act dz{b.dz, N, Tq, Hq, Wq, eo.cpad};
        Act XL = lev(L - 1, b.enc[L - 1][ar.blocks], ar.ch[L - 1]);
        A = lev(L - 1, b.gn_out.at("enc.out_gn"), ar.ch[L - 1]);
        wgrad("enc.out", dz, eo.cpad, A, 1, 1);
        dA = dgrad("enc.out", dz, b.G3);
        gn_bwd("enc.out_gn", XL, dA.p, nullptr, gcur);
        G = lev(L - 1, gcur, ar.ch[L - 1]);
        for (int l = L - 1; l >= 0; --l) {
            for (int k = ar.blocks - 1; k >= 0; --k) {
                const int C = (k == 0) ? (l > 0 ? ar.ch[l - 1] : ar.ch[0]) : ar.ch[l];
                block_bwd("enc.l" + std::to_string(l) + ".b" + std::to_string(k), lev(l, b.enc[l][k], C), G);
            }
            if (l > 0) {
                // enc.down{l-1}: stride-2 conv from level l-1
                const std::string nm = "enc.down" + std::to_string(l - 1);
                Act Xd = lev(l - 1, b.enc[l - 1][ar.blocks], ar.ch[l - 1]);
                wgrad(nm, G, G.C, Xd, 2, 2);
                if (c->bf16())
                    other([&] { return launch_zero_insert<__nv_bfloat16>(
                                    reinterpret_cast<const __nv_bfloat16*>(G.p), N, G.T, G.H, G.W, G.C, Xd.T, Xd.H,
                                    Xd.W, 2, 2, 2, reinterpret_cast<__nv_bfloat16*>(b.Z), s); },
                          4.0 * (double)N * Xd.T * Xd.H * Xd.W * G.C);
                else
                    other([&] { return launch_zero_insert<float>(reinterpret_cast<const float*>(G.p), N, G.T, G.H,
                                                                 G.W, G.C, Xd.T, Xd.H, Xd.W, 2, 2, 2,
                                                                 reinterpret_cast<float*>(b.Z), s); },
                          8.0 * (double)N * Xd.T * Xd.H * Xd.W * G.C);
                Act Zi{b.Z, N, Xd.T, Xd.H, Xd.W, G.C};
                dgrad(nm, Zi, galt);
                std::swap(gcur, galt);
                G = lev(l - 1, gcur, ar.ch[l - 1]);
            }
        }
        // stem (stride (t_stem,2,2)) from the pixels
        Act xin{const_cast<void*>(c->train_x), N, T, H, W, ar.in_ch};
        if (c->bf16()) {
            const GatherGeo g = stem_geo(N, T, H, W);
            other([&] { return launch_im2col_pixels(static_cast<const __nv_bfloat16*>(xin.p), nullptr, g,
                                                    reinterpret_cast<__nv_bfloat16*>(w.gather), s); },
                  gather_bytes(g));
            wgrad_gathered("enc.stem", G, G.C, g.Kpad);
        } else {
            wgrad("enc.stem", G, G.C, xin, ts, 2);
        }
    }
};

// Re-pack the adjoint weights of every conv (except the stem) from the master vector.
int pack_adjoints(tok_ctx* c, cudaStream_t s) {
    for (auto& cw : c->convs) {
        if (cw.name == "enc.stem" || cw.name == "stage.c0") continue;
        cw.cpad = adj_cpad(c, cw.Cout);
        cw.rows_pad = adj_rows(c, cw.Cin);
        const int taps = cw.k * cw.k * cw.k;
        const size_t es = c->esize();
        if (!cw.wt) {
            const size_t kp = c->bf16() ? (size_t)taps * cw.cpad : (size_t)round_up(taps * cw.cpad, 8);
            if (cudaMalloc(&cw.wt, (size_t)cw.rows_pad * kp * es) != cudaSuccess) return TOK_ENOMEM;
            if (cw.k == 3 && c->bf16()) {
                // output frame 0 takes its own taps (the replicate-pad correction folded in)
                if (cudaMalloc(&cw.wf0, (size_t)cw.rows_pad * kp * es) != cudaSuccess) return TOK_ENOMEM;
            } else if (cw.k == 3) {
                const size_t kc = (size_t)round_up(18 * cw.cpad, 8);
                if (cudaMalloc(&cw.wc, (size_t)cw.rows_pad * kc * es) != cudaSuccess) return TOK_ENOMEM;
            }
        }
        const float* w = c->d_master + cw.ow;
        int e;
        if (c->bf16()) {
            e = launch_pack_adjoint<__nv_bfloat16>(w, cw.Cout, cw.Cin, cw.k, cw.rows_pad, cw.cpad, 0,
                                                   static_cast<__nv_bfloat16*>(cw.wt), s);
            if (!e && cw.wf0)
                e = launch_pack_adjoint<__nv_bfloat16>(w, cw.Cout, cw.Cin, cw.k, cw.rows_pad, cw.cpad, 2,
                                                       static_cast<__nv_bfloat16*>(cw.wf0), s);
        } else {
            e = launch_pack_adjoint<float>(w, cw.Cout, cw.Cin, cw.k, cw.rows_pad, cw.cpad, 0,
                                           static_cast<float*>(cw.wt), s);
            if (!e && cw.wc)
                e = launch_pack_adjoint<float>(w, cw.Cout, cw.Cin, cw.k, cw.rows_pad, cw.cpad, 1,
                                               static_cast<float*>(cw.wc), s);
        }
        if (e) return TOK_ECUDA;
    }
    c->adjoint_dirty = false;
    return TOK_OK;
}

bool train_shape_ok(const tok_ctx* c, int N, int T, int H, int W) {
    return c->arch.kind == TOK_ARCH_FULL && N >= 1 && T >= 1 && (T - 1) % c->s_t == 0 && H % c->s_hw == 0 &&
           W % c->s_hw == 0 && H >= c->s_hw && W >= c->s_hw;
}

}  // namespace

extern "C" {

int tok_set_train_mode(tok_ctx* c, int mode) {
    if (!c || (mode != TOK_TRAIN_RECOMPUTE && mode != TOK_TRAIN_KEEP)) return TOK_EINVAL;
    c->train_mode = mode;
    return TOK_OK;
}

int64_t tok_param_total(const tok_ctx* c) { return c ? c->param_total : 0; }

int tok_get_params(tok_ctx* c, float* d_flat, void* stream) {
    if (!c || !d_flat) return TOK_EINVAL;
    return cudaMemcpyAsync(d_flat, c->d_master, (size_t)c->param_total * 4, cudaMemcpyDeviceToDevice,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? TOK_OK
               : TOK_ECUDA;
}

float* tok_params(tok_ctx* c) { return c ? c->d_master : nullptr; }

int tok_repack(tok_ctx* c, void* stream) {
    if (!c) return TOK_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // in a training loop (adjoint layouts already allocated, BF16): the forward rows and
    // both adjoint layouts of every 3x3x3 conv from one read of its new weights, all
    // such convs in one launch
    bool adj = c->bf16();
    for (const auto& cw : c->convs)
        if (cw.name != "enc.stem" && cw.name != "stage.c0" && !cw.wt) adj = false;
    const auto fused = [&](const ConvW& cw) { return adj && cw.k == 3 && !cw.im2col && cw.wt && cw.wf0 && !cw.dwm; };
    if (adj && !c->d_pack3_jobs) {
        std::vector<Pack3Job> jobs;
        long long blocks = 0;
        for (const auto& cw : c->convs) {
            if (!fused(cw)) continue;
            jobs.push_back(pack3_job(c->d_master + cw.ow, cw.Cout, cw.Cin, cw.Cout_pad, cw.Kpad, cw.rows_pad, cw.cpad,
                                     static_cast<__nv_bfloat16*>(cw.w), static_cast<__nv_bfloat16*>(cw.wt),
                                     static_cast<__nv_bfloat16*>(cw.wf0), blocks));
            blocks += (long long)jobs.back().gx * jobs.back().gy * 9;
        }
        if (!jobs.empty()) {
            if (cudaMalloc(&c->d_pack3_jobs, jobs.size() * sizeof(Pack3Job)) != cudaSuccess) return TOK_ENOMEM;
            if (cudaMemcpy(c->d_pack3_jobs, jobs.data(), jobs.size() * sizeof(Pack3Job), cudaMemcpyHostToDevice) !=
                cudaSuccess)
                return TOK_ECUDA;
        }
        c->n_pack3_jobs = (int)jobs.size();
        c->pack3_blocks = blocks;
    }
    if (adj && c->n_pack3_jobs > 0 &&
        launch_pack3_batch(static_cast<const Pack3Job*>(c->d_pack3_jobs), c->n_pack3_jobs, c->pack3_blocks, s))
        return TOK_ECUDA;
    for (auto& cw : c->convs) {
        if (fused(cw)) {
            cw.b = c->d_master + cw.ob;
            continue;
        }
        if (upload_conv(c, cw, s) != TOK_OK) return TOK_ECUDA;
        if (adj && cw.wt &&
            launch_pack_adjoint<__nv_bfloat16>(c->d_master + cw.ow, cw.Cout, cw.Cin, cw.k, cw.rows_pad, cw.cpad, 0,
                                               static_cast<__nv_bfloat16*>(cw.wt), s))
            return TOK_ECUDA;
        if (adj && cw.wf0 &&
            launch_pack_adjoint<__nv_bfloat16>(c->d_master + cw.ow, cw.Cout, cw.Cin, cw.k, cw.rows_pad, cw.cpad, 2,
                                               static_cast<__nv_bfloat16*>(cw.wf0), s))
            return TOK_ECUDA;
    }
    c->adjoint_dirty = !adj;
    return TOK_OK;
}

int tok_set_params_device(tok_ctx* c, const float* d_flat, void* stream) {
    if (!c || !d_flat) return TOK_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d_flat != c->d_master &&
        cudaMemcpyAsync(c->d_master, d_flat, (size_t)c->param_total * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return TOK_ECUDA;
    return tok_repack(c, stream);
}

size_t tok_train_workspace_bytes(const tok_ctx* c, int N, int T, int H, int W) {
    if (!c || !train_shape_ok(c, N, T, H, W)) return 0;
    return train_layout(c, N, T, H, W, nullptr, c->train_mode).total;
}

int tok_reserve_train(tok_ctx* c, int N, int T, int H, int W) {
    if (!c) return TOK_EINVAL;
    if (!train_shape_ok(c, N, T, H, W)) return TOK_ESHAPE;
    const size_t need = train_layout(c, N, T, H, W, nullptr, c->train_mode).total;
    if (need > c->tbytes) {
        if (c->tarena) {
            cudaDeviceSynchronize();
            guarded_free(c->tarena);
            c->tarena = nullptr;
            c->tbytes = 0;
        }
        c->tarena = guarded_alloc(need);
        if (!c->tarena) return TOK_ENOMEM;
        c->tbytes = need;
    }
    return TOK_OK;
}

int tok_train_forward(tok_ctx* c, const void* x, int N, int T, int H, int W, float rate, uint64_t seed, uint64_t step,
                      const uint32_t* keep_bits, float* xhat, float* loss, float* dxhat, void* stream) {
    if (!c || !x || !xhat || !loss || !dxhat || !(rate == rate)) return TOK_EINVAL;
    if (!train_shape_ok(c, N, T, H, W)) return TOK_ESHAPE;
    const size_t need = train_layout(c, N, T, H, W, nullptr, c->train_mode).total;
    if (need > c->tbytes) return TOK_ENOMEM;
    TrainExec ex;
    ex.c = c;
    ex.s = static_cast<cudaStream_t>(stream);
    ex.b = train_layout(c, N, T, H, W, c->tarena, c->train_mode);
    ex.set_work();
    ex.forward(x, N, T, H, W, rate, seed, step, keep_bits, xhat, loss, dxhat);
    if (ex.err) return ex.err;
    c->train_N = N;
    c->train_T = T;
    c->train_H = H;
    c->train_W = W;
    c->train_x = x;
    c->train_ready = true;
    c->train_mode_fwd = c->train_mode;
    return TOK_OK;
}

int tok_backward(tok_ctx* c, const float* dxhat, float* dparams, void* stream) {
    if (!c || !dxhat || !dparams) return TOK_EINVAL;
    if (!c->train_ready || c->train_mode_fwd != c->train_mode) return TOK_ESTATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->adjoint_dirty) {
        const int e = pack_adjoints(c, s);
        if (e) return e;
    }
    TrainExec ex;
    ex.c = c;
    ex.s = s;
    ex.b = train_layout(c, c->train_N, c->train_T, c->train_H, c->train_W, c->tarena, c->train_mode_fwd);
    ex.set_work();
    ex.grads = dparams;
    ex.backward(dxhat);
    return ex.err;
}

int tok_sgd(float* p, const float* g, int64_t n, float lr, void* stream) {
    if (!p || !g || n < 0) return TOK_EINVAL;
    return launch_sgd(p, g, n, lr, static_cast<cudaStream_t>(stream)) ? TOK_ECUDA : TOK_OK;
}

}  // extern "C"
