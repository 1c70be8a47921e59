// Internal definitions shared by the tokenizer library's translation units:
// the context (parameters, device layouts, workspace), the per-stream
// causal state, the layer list, workspace layouts and the layer executor.
// Everything except tok_ctx / tok_stream lives in an anonymous namespace, so
// each including file gets its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/tok.h"
#include "launchers.h"

using namespace tok;

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded device waits: 2 s

struct ParamInfo {
    std::string name;
    int ndim;
    int64_t dims[5];
    int64_t count;
    int64_t offset;  // in floats, in the flat parameter vector (architecture order)
};

struct ConvW {
    std::string name;
    int Cin, Cout, k;
    int im2col;     // BF16 path: input is gathered to (M, Kpad) and the conv runs as 1x1x1
    int Cout_pad, Kpad;
    void* w = nullptr;    // forward layout [Cout_pad][Kpad] (bf16 / fp32)
    float* b = nullptr;   // points into the context's master parameters
    int64_t ow = 0, ob = 0;  // offsets of weight and bias in the master vector
    // adjoint (input-gradient) conv: [rows_pad][taps][cpad] flipped/transposed,
    // and for k = 3 the replicate-pad correction [rows_pad][2*k*k][cpad]
    void* wt = nullptr;
    void* wc = nullptr;
    void* wf0 = nullptr;  // BF16: adjoint taps of output frame 0 with the correction folded in
    int dwm = 0;          // BF16 narrow 3x3x3 head: spatial taps in w's rows (3: dw rows, 9: (dh, dw) rows)
    int rows_pad = 0, cpad = 0;
};

struct GnW {
    std::string name;
    int C, G;
    float* g = nullptr;  // point into the master parameters
    float* b = nullptr;
    int64_t og = 0, ob = 0;
};

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
inline size_t align256(size_t a) { return (a + 255) & ~size_t(255); }

}  // namespace

struct tok_ctx {
    tok_arch arch;
    int precision;
    int device = 0, num_sms = 148;
    int cta_tiles = 0;  // conv launches: 0 persistent, n > 0 at most n tiles per CTA
    std::vector<ParamInfo> params;
    std::map<std::string, int> pindex;
    std::vector<std::vector<float>> host;
    int64_t param_total = 0;
    float* d_master = nullptr;  // flat FP32 parameters on the device (architecture order)
    bool adjoint_dirty = true;  // adjoint weights need re-packing
    // training workspace (tok_reserve_train) and the last training forward
    char* tarena = nullptr;
    size_t tbytes = 0;
    int train_N = 0, train_T = 0, train_H = 0, train_W = 0;
    bool train_ready = false;
    const void* train_x = nullptr;
    int train_mode = TOK_TRAIN_RECOMPUTE;  // memory mode of the next reserve / forward
    int train_mode_fwd = -1;               // mode the last training forward ran in
    std::vector<ConvW> convs;
    std::map<std::string, int> cindex;
    std::vector<GnW> gns;
    std::map<std::string, int> gindex;
    FsqConsts fsq;
    FsqThr* d_fsq_thr = nullptr;  // the FSQ rounding thresholds of fsq (device)
    // the batched re-pack of the 3x3x3 convs' BF16 layouts (built once the adjoint
    // layouts exist; their addresses never change afterwards)
    void* d_pack3_jobs = nullptr;
    int n_pack3_jobs = 0;
    long long pack3_blocks = 0;
    int* d_status = nullptr;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    int64_t launches = 0;
    int s_t = 1, s_hw = 1;
    // opt-in event timing (tok_profile_enable)
    struct ProfRec {
        int cls;
        double work;
        int ev;
        char name[40];  // layer name (convs, GroupNorms) or kernel label
    };
    bool prof = false;
    std::vector<cudaEvent_t> events;
    std::vector<ProfRec> recs;
    int ev_used = 0;
    // layer traces (tok_trace_layer): copies of a named layer's tensors
    struct Trace {
        std::string name;
        void* in;
        size_t in_cap;
        void* res;
        size_t res_cap;
        void* out;
        size_t out_cap;
    };
    std::vector<Trace> traces;
    bool bf16() const { return precision == TOK_BF16; }
    size_t esize() const { return bf16() ? 2 : 4; }
};

// One video stream's causal state: for every conv with temporal taps, the
// last two frames of its input (the left context of the next chunk), plus
// chunk counters for the encoder and the decoder side.
// Guard bands: every workspace allocation (the inference arena, the training
// workspace, a stream's caches) has kGuardBytes of the byte kGuardByte before and
// after the bytes it hands out; tok_check_guards / tok_stream_check_guards read
// them back, so a kernel that wrote outside its workspace is caught by the tests.
constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;

inline char* guarded_alloc(size_t bytes) {
    char* base = nullptr;
    if (cudaMalloc(&base, bytes + 2 * kGuardBytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemset(base, kGuardByte, kGuardBytes) != cudaSuccess ||
        cudaMemset(base + kGuardBytes + bytes, kGuardByte, kGuardBytes) != cudaSuccess) {
        cudaFree(base);
        return nullptr;
    }
    return base + kGuardBytes;
}

inline void guarded_free(char* p) {
    if (p) cudaFree(p - kGuardBytes);
}

// TOK_OK, TOK_EGUARD (a band changed) or TOK_ECUDA; synchronous.
inline int guards_check(const char* p, size_t bytes) {
    if (!p) return TOK_OK;
    std::vector<unsigned char> h(2 * kGuardBytes);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h.data(), p - kGuardBytes, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(h.data() + kGuardBytes, p + bytes, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TOK_ECUDA;
    for (unsigned char b : h)
        if (b != kGuardByte) return TOK_EGUARD;
    return TOK_OK;
}

struct tok_stream {
    tok_ctx* ctx = nullptr;
    int H = 0, W = 0;
    int enc_chunk = 0, dec_chunk = 0;
    char* mem = nullptr;
    size_t bytes = 0;
    std::map<std::string, char*> hist;        // conv name -> 2 frames
    std::map<std::string, size_t> frame_bytes; // conv name -> bytes of one frame
};

namespace {

// ------------------------------------------------------------ layer list

void add_param(tok_ctx* c, const std::string& name, std::vector<int64_t> dims) {
    ParamInfo p;
    p.name = name;
    p.ndim = (int)dims.size();
    p.count = 1;
    for (int i = 0; i < 5; ++i) p.dims[i] = i < p.ndim ? dims[i] : 0;
    for (auto d : dims) p.count *= d;
    p.offset = c->param_total;
    c->param_total += p.count;
    c->pindex[name] = (int)c->params.size();
    c->params.push_back(p);
    c->host.emplace_back((size_t)p.count, 0.f);
}

void add_conv(tok_ctx* c, const std::string& name, int cout, int cin, int k, bool im2col_in) {
    add_param(c, name + ".w", {cout, k, k, k, cin});
    add_param(c, name + ".b", {cout});
    ConvW cw;
    cw.name = name;
    cw.ow = c->params[c->pindex[name + ".w"]].offset;
    cw.ob = c->params[c->pindex[name + ".b"]].offset;
    cw.Cin = cin;
    cw.Cout = cout;
    cw.k = k;
    const int taps = k * k * k;
    if (c->bf16()) {
        cw.im2col = (im2col_in || cin % 64 != 0) ? 1 : 0;
        cw.Kpad = cw.im2col ? round_up(taps * cin, 64) : taps * cin;
        const int c16 = round_up(cout, 16);
        cw.Cout_pad = conv_tc_cout_pad(c16);
    } else {
        cw.im2col = 0;
        cw.Kpad = round_up(taps * cin, 8);
        cw.Cout_pad = round_up(cout, 16);
    }
    c->cindex[name] = (int)c->convs.size();
    c->convs.push_back(cw);
}

void add_gn(tok_ctx* c, const std::string& name, int C) {
    add_param(c, name + ".g", {C});
    add_param(c, name + ".b", {C});
    GnW g;
    g.name = name;
    g.og = c->params[c->pindex[name + ".g"]].offset;
    g.ob = c->params[c->pindex[name + ".b"]].offset;
    g.C = C;
    g.G = std::max(1, std::min(c->arch.gn_groups, C / 2));
    c->gindex[name] = (int)c->gns.size();
    c->gns.push_back(g);
}

void add_block(tok_ctx* c, const std::string& name, int cin, int cout) {
    add_gn(c, name + ".gn1", cin);
    add_conv(c, name + ".c1", cout, cin, 3, false);
    add_gn(c, name + ".gn2", cout);
    add_conv(c, name + ".c2", cout, cout, 3, false);
    if (cin != cout) add_conv(c, name + ".sc", cout, cin, 1, false);
}

void build_layers(tok_ctx* c) {
    const tok_arch& a = c->arch;
    const int* ch = a.ch;
    if (a.kind == TOK_ARCH_STAGE) {
        add_conv(c, "stage.c0", ch[0], a.in_ch, 3, true);
        add_conv(c, "stage.c1", ch[1], ch[0], 3, false);
        add_gn(c, "stage.gn", ch[1]);
        add_conv(c, "stage.out", a.nlev, ch[1], 1, false);
        c->s_t = 1;
        c->s_hw = 2;
        return;
    }
    add_conv(c, "enc.stem", ch[0], a.in_ch, 3, true);
    for (int l = 0; l < a.nlevels; ++l) {
        const int cin = l > 0 ? ch[l - 1] : ch[0];
        for (int b = 0; b < a.blocks; ++b)
            add_block(c, "enc.l" + std::to_string(l) + ".b" + std::to_string(b), b == 0 ? cin : ch[l], ch[l]);
        if (l < a.nlevels - 1) add_conv(c, "enc.down" + std::to_string(l), ch[l], ch[l], 3, false);
    }
    add_gn(c, "enc.out_gn", ch[a.nlevels - 1]);
    add_conv(c, "enc.out", a.nlev, ch[a.nlevels - 1], 3, false);
    add_conv(c, "dec.in", ch[a.nlevels - 1], a.nlev, 3, true);
    for (int l = a.nlevels - 1; l >= 0; --l) {
        for (int b = 0; b < a.blocks; ++b)
            add_block(c, "dec.l" + std::to_string(l) + ".b" + std::to_string(b), ch[l], ch[l]);
        if (l > 0) add_conv(c, "dec.up" + std::to_string(l - 1), ch[l - 1] * 8, ch[l], 3, false);
    }
    add_gn(c, "dec.out_gn", ch[0]);
    add_conv(c, "dec.out", a.in_ch * 4 * a.t_stem, ch[0], 3, false);
    c->s_t = a.t_stem << (a.nlevels - 1);
    c->s_hw = 1 << a.nlevels;
}

FsqConsts make_fsq(const int* levels, int nlev) {
    FsqConsts f;
    memset(&f, 0, sizeof(f));
    f.nlev = nlev;
    int basis = 1;
    for (int i = 0; i < nlev; ++i) {
        const int L = levels[i];
        const double h = (L - 1) * (1.0 - 1e-3) / 2.0;
        const double o = (L % 2 == 0) ? 0.5 : 0.0;
        f.levels[i] = L;
        f.half_l[i] = (float)h;
        f.offset[i] = (float)o;
        f.shift[i] = (float)std::atanh(o / h);
        f.half_w[i] = L / 2;
        f.basis[i] = basis;
        basis *= L;
    }
    return f;
}

bool valid_levels(const int* levels, int nlev) {
    if (!levels || nlev < 1 || nlev > 8) return false;
    long long prod = 1;
    for (int i = 0; i < nlev; ++i) {
        if (levels[i] < 2 || levels[i] > 16) return false;
        prod *= levels[i];
    }
    return prod < (1LL << 31);
}

// Pack one conv's forward weights from the master vector into its device layout.
int upload_conv(tok_ctx* c, ConvW& cw, cudaStream_t st = 0) {
    const int K = cw.k * cw.k * cw.k * cw.Cin;
    const float* w = c->d_master + cw.ow;
    cw.b = c->d_master + cw.ob;
    int e;
    cw.dwm = (c->bf16() && cw.k == 3 && !cw.im2col && cw.Cin % 64 == 0) ? conv_tc_taprows(cw.Cout, cw.Cin, 3, 1, 1) : 0;
    if (cw.dwm)
        e = launch_pack_weights_taprows(w, cw.Cout, cw.Cin, cw.Cout_pad, cw.dwm, static_cast<__nv_bfloat16*>(cw.w),
                                        st);
    else if (c->bf16())
        e = launch_pack_weights<__nv_bfloat16>(w, cw.Cout, K, cw.Cout_pad, cw.Kpad, static_cast<__nv_bfloat16*>(cw.w),
                                               st);
    else
        e = launch_pack_weights<float>(w, cw.Cout, K, cw.Cout_pad, cw.Kpad, static_cast<float*>(cw.w), st);
    return e ? TOK_ECUDA : TOK_OK;
}

int upload_gn(tok_ctx* c, GnW& g) {
    g.g = c->d_master + g.og;
    g.b = c->d_master + g.ob;
    return TOK_OK;
}

// ------------------------------------------------------------ workspace

struct Layout {
    size_t act;       // bytes per activation buffer
    size_t gather;    // im2col (BF16) / edge-padded pixels + codes (FP32)
    size_t zbuf;      // latent when the caller passes no z
    size_t gn;        // GroupNorm scratch
    size_t gnpart;    // GroupNorm statistics reduced by the producing conv (BF16)
    size_t total;
};

struct Dims {
    int Hp, Wp, Tq, Hq, Wq;
};

Dims clip_dims(const tok_ctx* c, int T, int H, int W) {
    Dims d;
    d.Hp = round_up(H, c->s_hw);
    d.Wp = round_up(W, c->s_hw);
    d.Tq = (T - 1) / c->s_t + 1;
    d.Hq = d.Hp / c->s_hw;
    d.Wq = d.Wp / c->s_hw;
    return d;
}

// Frames out of the stem for T input frames (a whole clip or its first
// chunk); a later chunk of s_T frames gives s_T / t_stem.
int stem_frames(const tok_ctx* c, int T) {
    const int ts = c->arch.kind == TOK_ARCH_FULL ? c->arch.t_stem : 1;
    return (T - 1) / ts + 1;
}

// Upper bound on the GroupNorm statistics slots of an Hout x Wout conv output:
// tiles of at least 192 voxels (BH x BW, BW >= 8) cover it in at most
// HW/192 + Hout + Wout/8 + 1 tiles.
inline long long gn_slot_bound(long long Ho, long long Wo) { return Ho * Wo / 128 + Ho + Wo / 8 + 2; }

// Bytes of the statistics triples the largest conv output of the walk needs:
// plain outputs at every level, and depth-to-space outputs (4 sub-positions per
// tile of the up conv's input).
size_t gnpart_bytes(const tok_ctx* c, int N, int T, int Hp, int Wp) {
    const tok_arch& a = c->arch;
    if (!c->bf16() || a.kind != TOK_ARCH_FULL) return 0;
    size_t m = 0;
    int Tl = stem_frames(c, T), Tprev = Tl;
    for (int l = 0; l < a.nlevels; ++l) {
        const long long Hl = Hp >> (l + 1), Wl = Wp >> (l + 1);
        m = std::max<size_t>(m, (size_t)N * Tl * gn_slot_bound(Hl, Wl) * a.gn_groups * sizeof(GnTriple));
        if (l > 0)
            m = std::max<size_t>(m, (size_t)N * Tprev * 4 * gn_slot_bound(Hl, Wl) * a.gn_groups * sizeof(GnTriple));
        Tprev = Tl;
        Tl = (Tl - 1) / 2 + 1;
    }
    return m;
}

Layout layout_for(const tok_ctx* c, int N, int T, int H, int W) {
    Layout L;
    const Dims d = clip_dims(c, T, H, W);
    const tok_arch& a = c->arch;
    const size_t es = c->esize();
    size_t act = 0, gn = 0;
    auto gn_need = [&](long long frames, long long HW, int C) {
        const int G = std::max(1, std::min(a.gn_groups, C / 2));
        gn = std::max(gn, gn_scratch_bytes(frames, HW, C, G, c->num_sms, c->bf16() ? 8 : 4));
    };
    if (a.kind == TOK_ARCH_STAGE) {
        act = std::max<size_t>((size_t)N * T * d.Hp * d.Wp * a.ch[0], (size_t)N * T * (d.Hp / 2) * (d.Wp / 2) * a.ch[1]) * es;
        gn_need((long long)N * T, (long long)(d.Hp / 2) * (d.Wp / 2), a.ch[1]);
    } else {
        int Tl = stem_frames(c, T);
        for (int l = 0; l < a.nlevels; ++l) {
            const long long Hl = d.Hp >> (l + 1), Wl = d.Wp >> (l + 1);
            const int cmax = std::max(a.ch[l], l > 0 ? a.ch[l - 1] : a.ch[0]);
            act = std::max<size_t>(act, (size_t)N * Tl * Hl * Wl * cmax * es);
            gn_need((long long)N * Tl, Hl * Wl, a.ch[l]);
            if (l > 0) gn_need((long long)N * Tl, Hl * Wl, a.ch[l - 1]);
            Tl = (Tl - 1) / 2 + 1;
        }
    }
    L.act = align256(act);
    size_t g = 0;
    const long long ntok = (long long)N * d.Tq * d.Hq * d.Wq;
    if (c->bf16()) {
        // stem / stage.c0 im2col and dec.in im2col
        const long long m0 = a.kind == TOK_ARCH_STAGE ? (long long)N * T * d.Hp * d.Wp
                                                       : (long long)N * stem_frames(c, T) * (d.Hp / 2) * (d.Wp / 2);
        g = (size_t)m0 * round_up(27 * a.in_ch, 64) * 2;
        g = std::max(g, (size_t)ntok * round_up(27 * a.nlev, 64) * 2);
    } else {
        g = align256((size_t)N * T * d.Hp * d.Wp * a.in_ch * 4) + align256((size_t)ntok * a.nlev * 4);
    }
    L.gather = align256(g);
    L.zbuf = align256((size_t)ntok * a.nlev * 4);
    L.gn = align256(gn);
    L.gnpart = align256(gnpart_bytes(c, N, T, d.Hp, d.Wp));
    L.total = 5 * L.act + L.gather + L.zbuf + L.gn + L.gnpart;
    return L;
}

struct Work {
    char* act[5];
    char* gather;
    char* zbuf;
    char* gn;
    char* gnpart = nullptr;
    size_t gnpart_bytes = 0;
};

// Carve one problem's workspace out of the arena, starting `off` bytes in.
Work carve(tok_ctx* c, const Layout& L, size_t off = 0) {
    Work w;
    char* p = c->arena + off;
    for (int i = 0; i < 5; ++i) {
        w.act[i] = p;
        p += L.act;
    }
    w.gather = p;
    p += L.gather;
    w.zbuf = p;
    p += L.zbuf;
    w.gn = p;
    p += L.gn;
    w.gnpart = L.gnpart ? p : nullptr;
    w.gnpart_bytes = L.gnpart;
    return w;
}

// ------------------------------------------------------------ executor

int32_t zero_index_of(const tok_ctx* c) {
    int32_t z = 0, b = 1;
    for (int i = 0; i < c->arch.nlev; ++i) {
        z += (c->arch.levels[i] / 2) * b;
        b *= c->arch.levels[i];
    }
    return z;
}

// Every conv with temporal taps and the bytes of one frame of its input, for
// one stream of H x W pixels (N = 1). On the BF16 path the stem and the
// decoder input keep the raw pixels / token indices their gathers read.
std::vector<std::pair<std::string, size_t>> stream_frames(const tok_ctx* c, int H, int W) {
    std::vector<std::pair<std::string, size_t>> v;
    const tok_arch& a = c->arch;
    const Dims d = clip_dims(c, 1, H, W);
    const size_t es = c->esize();
    const size_t pix = c->bf16() ? (size_t)H * W * a.in_ch * 2 : (size_t)d.Hp * d.Wp * a.in_ch * 4;
    if (a.kind == TOK_ARCH_STAGE) {
        v.push_back({"stage.c0", pix});
        v.push_back({"stage.c1", (size_t)d.Hp * d.Wp * a.ch[0] * es});
        return v;
    }
    v.push_back({"enc.stem", pix});
    for (int l = 0; l < a.nlevels; ++l) {
        const size_t hw = (size_t)(d.Hp >> (l + 1)) * (d.Wp >> (l + 1));
        const int cin = l > 0 ? a.ch[l - 1] : a.ch[0];
        for (int b = 0; b < a.blocks; ++b) {
            const std::string n = "enc.l" + std::to_string(l) + ".b" + std::to_string(b);
            v.push_back({n + ".c1", hw * (b == 0 ? cin : a.ch[l]) * es});
            v.push_back({n + ".c2", hw * a.ch[l] * es});
        }
        if (l < a.nlevels - 1) v.push_back({"enc.down" + std::to_string(l), hw * a.ch[l] * es});
    }
    const size_t hwq = (size_t)d.Hq * d.Wq;
    v.push_back({"enc.out", hwq * a.ch[a.nlevels - 1] * es});
    v.push_back({"dec.in", c->bf16() ? hwq * 4 : hwq * a.nlev * 4});
    for (int l = a.nlevels - 1; l >= 0; --l) {
        const size_t hw = (size_t)(d.Hp >> (l + 1)) * (d.Wp >> (l + 1));
        for (int b = 0; b < a.blocks; ++b) {
            const std::string n = "dec.l" + std::to_string(l) + ".b" + std::to_string(b);
            v.push_back({n + ".c1", hw * a.ch[l] * es});
            v.push_back({n + ".c2", hw * a.ch[l] * es});
        }
        if (l > 0) v.push_back({"dec.up" + std::to_string(l - 1), hw * a.ch[l] * es});
    }
    v.push_back({"dec.out", (size_t)(d.Hp >> 1) * (d.Wp >> 1) * a.ch[0] * es});
    return v;
}

struct Act {
    void* p;
    int N, T, H, W, C;
    const GnTriple* part = nullptr;  // GroupNorm statistics the producing conv reduced
    int part_S = 0;                  // their slots per frame
};

struct Exec {
    tok_ctx* c;
    cudaStream_t s;
    Work w;
    int err = 0;
    // conv tiles may depend on the frame count also where GroupNorm statistics
    // are reduced (no stream of chunks has to match this pass bit for bit)
    bool any_tile = false;
    void ck(int e) {
        if (e && !err) err = TOK_ECUDA;
    }

    // profiling: record an event pair around a launch (class 0 conv, 1 GN, 2 other)
    int pbegin() {
        if (!c->prof || c->ev_used + 2 > (int)c->events.size()) return -1;
        const int e = c->ev_used;
        c->ev_used += 2;
        cudaEventRecord(c->events[e], s);
        return e;
    }
    void pend(int e, int cls, double work, const std::string& name = std::string()) {
        if (e < 0) return;
        cudaEventRecord(c->events[e + 1], s);
        tok_ctx::ProfRec r;
        r.cls = cls;
        r.work = work;
        r.ev = e;
        snprintf(r.name, sizeof(r.name), "%s", name.c_str());
        c->recs.push_back(r);
    }

    ConvArgs base_args(const ConvW& cw, const Act& in, int st, int sh, int sw) {
        ConvArgs a;
        memset(&a, 0, sizeof(a));
        a.x = in.p;
        a.N = in.N;
        a.Tin = in.T;
        a.Hin = in.H;
        a.Win = in.W;
        a.Cin = in.C;
        a.w = cw.w;
        a.w_dwm = cw.dwm;
        a.gn_any_tile = any_tile ? 1 : 0;
        a.bias = cw.b;
        a.Cout = cw.Cout;
        a.Cout_pad = cw.Cout_pad;
        a.Kpad = cw.Kpad;
        a.kt = a.kh = a.kw = cw.k;
        a.st = st;
        a.sh = sh;
        a.sw = sw;
        a.t_off = -(cw.k - 1);
        a.pad_mode = c->arch.time_pad;
        a.Tout = (in.T - 1) / st + 1;
        a.Hout = (in.H + 2 * ((cw.k - 1) / 2) - cw.k) / sh + 1;
        a.Wout = (in.W + 2 * ((cw.k - 1) / 2) - cw.k) / sw + 1;
        a.status = c->d_status;
        a.wait_ns = kWaitNs;
        a.fsq = c->fsq;
        a.fsq_thr = c->d_fsq_thr;
        return a;
    }

    // Ask a BF16 conv for the GroupNorm statistics of its output (Cgn channels)
    // when its kernel form reduces them and the workspace region holds them.
    void want_gn_stats(ConvArgs& a, const Work& wk, int Cgn) {
        a.gn_part = nullptr;
        a.gn_cg = 0;
        if (!c->bf16() || !wk.gnpart) return;
        const int G = std::max(1, std::min(c->arch.gn_groups, Cgn / 2));
        if (Cgn % G) return;
        a.gn_cg = Cgn / G;
        if (!conv_tc_gn_fusable(a)) {
            a.gn_cg = 0;
            return;
        }
        const size_t need = (size_t)a.N * a.oT * conv_tc_gn_slots(a) * G * sizeof(GnTriple);
        if (need <= wk.gnpart_bytes)
            a.gn_part = reinterpret_cast<GnTriple*>(wk.gnpart);
        else
            a.gn_cg = 0;
    }
    static void tag_gn_stats(Act& o, const ConvArgs& a) {
        if (a.gn_part) {
            o.part = a.gn_part;
            o.part_S = conv_tc_gn_slots(a);
        }
    }

    void launch(ConvArgs& a, const ConvW& cw) {
        if (err) return;
        const double flop = 2.0 * (double)a.N * a.Tout * a.Hout * a.Wout * cw.Cout * (double)(cw.k * cw.k * cw.k) *
                            cw.Cin;
        const int e = pbegin();
        if (c->bf16())
            ck(launch_conv_tc_group(&a, 1, c->num_sms, s, 0));
        else
            ck(launch_conv_simt(a, s));
        pend(e, 0, flop, cw.name);
        c->launches += 1;
    }

    // Layer trace (a test hook): device-to-device copies, on the executor's
    // stream, of the tensors of a traced layer; a buffer too small for its
    // tensor makes the call fail with TOK_EINVAL.
    void trace(const std::string& name, const void* in, size_t in_b, const void* res, size_t res_b, const void* out,
               size_t out_b) {
        if (err || c->traces.empty()) return;
        for (const auto& t : c->traces) {
            if (t.name != name) continue;
            const std::pair<const void*, size_t> src[3] = {{in, in_b}, {res, res_b}, {out, out_b}};
            void* const dst[3] = {t.in, t.res, t.out};
            const size_t cap[3] = {t.in_cap, t.res_cap, t.out_cap};
            for (int i = 0; i < 3; ++i) {
                if (!dst[i] || !src[i].first) continue;
                if (src[i].second > cap[i]) {
                    err = TOK_EINVAL;
                    return;
                }
                if (cudaMemcpyAsync(dst[i], src[i].first, src[i].second, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                    ck(1);
            }
        }
    }
    void trace_conv(const std::string& name, const ConvArgs& a) {
        if (c->traces.empty()) return;
        const size_t es = c->esize();
        const size_t in_b = (size_t)a.N * a.Tin * a.Hin * a.Win * a.Cin * es;
        const size_t o_vox = (size_t)a.N * a.oT * a.oH * a.oW;
        const size_t res_b = o_vox * a.oC * es;
        const size_t out_b = a.mode == OUT_FSQ ? (size_t)a.N * a.Tout * a.Hout * a.Wout * c->arch.nlev * 4
                                               : o_vox * a.oC * (a.out_fp32 ? 4 : es);
        trace(name, a.x, in_b, a.residual, res_b, a.out, out_b);
    }

    // Other (bandwidth-bound) kernels: bytes of algorithmic traffic.
    template <typename F>
    void other(F&& f, double bytes, int nk = 1, const char* label = "other") {
        if (err) return;
        const int e = pbegin();
        ck(f());
        pend(e, 2, bytes, label);
        c->launches += nk;
    }

    // Plain conv (optional residual) into `out`.
    Act conv(const std::string& name, const Act& in, void* out, const void* residual = nullptr, int tst = 1,
             int sh = 1, int sw = 1) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs a = base_args(cw, in, tst, sh, sw);
        a.mode = OUT_PLAIN;
        a.out = out;
        a.residual = residual;
        a.oT = a.Tout;
        a.oH = a.Hout;
        a.oW = a.Wout;
        a.oC = cw.Cout;
        want_gn_stats(a, w, cw.Cout);
        launch(a, cw);
        trace_conv(cw.name, a);
        Act o{out, in.N, a.Tout, a.Hout, a.Wout, cw.Cout};
        tag_gn_stats(o, a);
        return o;
    }

    // Conv followed by depth-to-space (r = (rt, rh, rw)), cropped to oH x oW.
    Act conv_d2s(const std::string& name, const Act& in, void* out, int rt, int rh, int rw, int oH, int oW,
                 bool out_fp32) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs a = base_args(cw, in, 1, 1, 1);
        a.mode = OUT_D2S;
        a.out = out;
        a.out_fp32 = out_fp32 ? 1 : 0;
        a.rt = rt;
        a.rh = rh;
        a.rw = rw;
        a.drop_t = rt - 1;  // causal trim of the clip's first rt-1 frames
        a.oT = a.Tout * rt - a.drop_t;
        a.oH = oH;
        a.oW = oW;
        a.oC = cw.Cout / (rt * rh * rw);
        if (!out_fp32) want_gn_stats(a, w, a.oC);
        launch(a, cw);
        trace_conv(cw.name, a);
        Act o{out, in.N, a.oT, oH, oW, a.oC};
        tag_gn_stats(o, a);
        return o;
    }

    // Conv whose input is first gathered into an im2col matrix (BF16 path):
    // runs as a 1x1x1 conv over (N, Tout, Hout, Wout, Kpad).
    Act conv_gathered(const std::string& name, int N, int Tout, int Hout, int Wout, void* out, int mode,
                      int32_t* idx_out) {
        const ConvW& cw = c->convs[c->cindex[name]];
        Act in{w.gather, N, Tout, Hout, Wout, cw.Kpad};
        ConvArgs a = base_args(cw, in, 1, 1, 1);
        a.Cin = cw.Kpad;
        a.kt = a.kh = a.kw = 1;
        a.t_off = 0;
        a.mode = mode;
        a.out = out;
        a.idx = idx_out;
        a.oT = Tout;
        a.oH = Hout;
        a.oW = Wout;
        a.oC = cw.Cout;
        if (mode == OUT_PLAIN) want_gn_stats(a, w, cw.Cout);
        launch(a, cw);
        trace_conv(cw.name, a);
        Act o{out, N, Tout, Hout, Wout, cw.Cout};
        tag_gn_stats(o, a);
        return o;
    }

    // One problem of the fused BF16 stem: pixels x (N, T, H, W, 3) (H, W the padded
    // extent) with the stream history hist or null, into out; the GroupNorm
    // statistics of the output go to wk.gnpart when its 32 groups fit there.
    StemArgs stem_args(const ConvW& cw, const void* x, const void* hist, int N, int T, int H, int W, int st, int t_off,
                       void* out, const Work& wk) const {
        StemArgs a;
        memset(&a, 0, sizeof(a));
        a.x = x;
        a.hist = hist;
        a.hist_T = hist ? 2 : 0;
        a.N = N;
        a.Tin = T;
        a.H = H;
        a.W = W;
        a.Tout = (T - 1) / st + 1;
        a.st = st;
        a.t_off = t_off;
        a.pad_mode = c->arch.time_pad;
        a.w = cw.w;
        a.bias = cw.b;
        a.Cout = cw.Cout;
        a.Cout_pad = cw.Cout_pad;
        a.Kpad = cw.Kpad;
        a.out = out;
        a.status = c->d_status;
        a.wait_ns = kWaitNs;
        const int G = std::max(1, std::min(c->arch.gn_groups, cw.Cout / 2));
        if (wk.gnpart && G == 32 && cw.Cout % 32 == 0) {
            const size_t need = (size_t)N * a.Tout * stem_tc_gn_slots(H, W) * 32 * sizeof(GnTriple);
            if (need <= wk.gnpart_bytes) a.gn_part = reinterpret_cast<GnTriple*>(wk.gnpart);
        }
        return a;
    }

    // The fused stem over as[0 .. count): false, with nothing enqueued, where a
    // problem is outside its form (the caller then gathers the im2col matrix).
    // trace_first: as[0] is the problem a layer trace records (batch item 0).
    bool stem_launch(const StemArgs* as, int count, const ConvW& cw, bool trace_first = true) {
        if (!c->bf16() || !stem_tc_accepts(as, count)) return false;
        if (err) return true;
        double flop = 0;
        for (int p = 0; p < count; ++p)
            flop += 2.0 * (double)as[p].N * as[p].Tout * (as[p].H / 2) * (as[p].W / 2) * cw.Cout *
                    (double)(cw.k * cw.k * cw.k) * cw.Cin;
        const int e = pbegin();
        ck(launch_stem_tc(as, count, c->num_sms, s, c->cta_tiles));
        pend(e, 0, flop, cw.name);
        c->launches += 1;
        const StemArgs& a = as[0];
        if (trace_first) trace(cw.name, a.x, (size_t)a.N * a.Tin * a.H * a.W * 3 * 2, nullptr, 0, a.out,
              (size_t)a.N * a.Tout * (a.H / 2) * (a.W / 2) * cw.Cout * 2);
        return true;
    }
    static Act stem_out(const StemArgs& a) {
        Act o{a.out, a.N, a.Tout, a.H / 2, a.W / 2, a.Cout};
        if (a.gn_part) {
            o.part = a.gn_part;
            o.part_S = stem_tc_gn_slots(a.H, a.W);
        }
        return o;
    }

    Act gn_silu(const std::string& name, const Act& in, void* out) {
        const GnW& g = c->gns[c->gindex[name]];
        if (err) return Act{out, in.N, in.T, in.H, in.W, in.C};
        const long long frames = (long long)in.N * in.T, HW = (long long)in.H * in.W;
        const int e = pbegin();
        if (c->bf16()) {
            GnItem<__nv_bfloat16> it{static_cast<const __nv_bfloat16*>(in.p), static_cast<__nv_bfloat16*>(out), frames,
                                     HW, w.gn, in.part, in.part_S};
            ck(launch_gn_silu_group<__nv_bfloat16>(&it, 1, in.C, g.G, g.g, g.b, c->arch.gn_eps, true, s, c->d_status));
        } else
            ck(launch_gn_silu<float>(static_cast<const float*>(in.p), static_cast<float*>(out), frames, HW, in.C, g.G,
                                     g.g, g.b, c->arch.gn_eps, w.gn, c->num_sms, false, s, c->d_status));
        pend(e, 1, 2.0 * (double)frames * HW * in.C * c->esize(), name);
        c->launches += 3;
        const size_t nb = (size_t)frames * HW * in.C * c->esize();
        trace(name, in.p, nb, nullptr, 0, out, nb);
        return Act{out, in.N, in.T, in.H, in.W, in.C};
    }

    // Last encoder conv: latent z (fp32) and FSQ token indices.
    void out_conv(const std::string& name, const Act& A, float* z, int32_t* idx) {
        const ConvW& cw = c->convs[c->cindex[name]];
        ConvArgs a = base_args(cw, A, 1, 1, 1);
        a.out = z;
        a.oT = a.Tout;
        a.oH = a.Hout;
        a.oW = a.Wout;
        a.oC = cw.Cout;
        const long long ntok = (long long)A.N * a.Tout * a.Hout * a.Wout;
        if (c->bf16()) {
            a.mode = OUT_FSQ;
            a.idx = idx;
            launch(a, cw);
            trace_conv(cw.name, a);
        } else {
            a.mode = OUT_PLAIN;
            a.out_fp32 = 1;
            launch(a, cw);
            trace_conv(cw.name, a);
            if (idx) other([&] { return launch_fsq(z, ntok, c->fsq, idx, nullptr, s); }, (double)ntok * (4 * cw.Cout + 4));
        }
    }

    GatherGeo gather_pixels(int N, int T, int H, int W, int Hp, int Wp, int stride_hw) {
        GatherGeo g;
        g.N = N;
        g.Tin = T;
        g.H = H;
        g.W = W;
        g.Hp = Hp;
        g.Wp = Wp;
        g.Cin = c->arch.in_ch;
        g.hist_T = 0;
        g.Tout = T;
        g.Hout = Hp / stride_hw;
        g.Wout = Wp / stride_hw;
        g.kt = g.kh = g.kw = 3;
        g.st = 1;
        g.sh = g.sw = stride_hw;
        g.t_off = -2;
        g.pad_mode = c->arch.time_pad;
        g.Kpad = round_up(27 * g.Cin, 64);
        return g;
    }

    static double gather_bytes(const GatherGeo& g) {
        return (double)g.N * g.Tout * g.Hout * g.Wout * g.Kpad * 2;
    }
};

// A stream's caches may be advanced by any context with the same architecture
// and precision (a serving loop runs chunks of one stream on several lanes).
bool compatible(const tok_ctx* a, const tok_ctx* b) {
    return a == b || (a && b && a->precision == b->precision && memcmp(&a->arch, &b->arch, sizeof(tok_arch)) == 0);
}

int check_cuda_device(int* num_sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOK_EDEVICE;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return TOK_EDEVICE;
    *num_sms = p.multiProcessorCount;
    return (p.major == 10) ? TOK_OK : TOK_EDEVICE;
}

}  // namespace
