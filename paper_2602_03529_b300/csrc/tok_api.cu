// C-ABI of the tokenizer library: context, parameters, workspace and the
// layer executor of the encoder f_phi / decoder g_theta (see include/tok.h).
//
// The executor walks the layer list of the descriptor and launches, per
// layer, the kernels of the selected precision path:
//   BF16: tcgen05 implicit-GEMM convs (k_conv_tc.cu), BF16 GroupNorm+SiLU,
//         im2col gathers for the 3-channel stem and the code-vector input,
//         FSQ fused into the last encoder conv, depth-to-space fused into the
//         decoder's upsampling convs.
//   FP32: CUDA-core implicit-GEMM convs (k_conv_simt.cu), FP32 GroupNorm+SiLU,
//         stand-alone FSQ / dequantisation.
// All work is enqueued on the caller's stream; nothing here synchronises
// except tok_set_param / tok_status / allocation calls.
#include "exec_group.h"

// ======================================================================= C ABI

extern "C" {

void tok_arch_default(tok_arch* a) {
    if (!a) return;
    memset(a, 0, sizeof(*a));
    a->kind = TOK_ARCH_FULL;
    a->in_ch = 3;
    a->nlevels = 3;
    a->ch[0] = 128;
    a->ch[1] = 256;
    a->ch[2] = 512;
    a->blocks = 2;
    a->nlev = 6;
    const int lv[6] = {8, 8, 8, 5, 5, 5};
    for (int i = 0; i < 6; ++i) a->levels[i] = lv[i];
    a->gn_groups = 32;
    a->gn_eps = 1e-6f;
    a->time_pad = TOK_PAD_REPLICATE;
    a->t_stem = 1;
}

}  // extern "C"

namespace {

// Whether an architecture descriptor is one the library builds (TOK_OK) on the
// given path (TOK_BF16 needs channel counts that are multiples of 64).
int arch_error(const tok_arch& a, int precision) {
    if (a.in_ch != 3 || !valid_levels(a.levels, a.nlev)) return TOK_EINVAL;
    if (a.kind == TOK_ARCH_FULL) {
        if (a.nlevels < 1 || a.nlevels > 4 || a.blocks < 0) return TOK_EINVAL;
        if (a.t_stem != 1 && a.t_stem != 2) return TOK_EINVAL;
    } else if (a.kind != TOK_ARCH_STAGE) {
        return TOK_EINVAL;
    }
    const int nch = a.kind == TOK_ARCH_STAGE ? 2 : a.nlevels;
    for (int i = 0; i < nch; ++i) {
        const int C = a.ch[i];
        if (C < 16 || C % 16 != 0) return TOK_EINVAL;
        if (precision == TOK_BF16 && C % 64 != 0) return TOK_EINVAL;
    }
    return TOK_OK;
}

// ---- weights file: the flat FP32 parameters with the descriptor they belong to.
// Little-endian, 104-byte header:
//   0 "TOKW"   4 version (1)   8 kind   12 in_ch   16 nlevels   20 ch[4]   36 blocks
//   40 nlev   44 levels[8]   76 gn_groups   80 gn_eps (float32 bits)   84 time_pad
//   88 t_stem   92 0   96 parameter count n (int64)
// then n float32 values in the order of tok_param_info, then the 64-bit FNV-1a hash
// of those 4 n bytes.
constexpr uint32_t kWeightsMagic = 0x574B4F54u;  // "TOKW" read as a little-endian word
constexpr uint32_t kWeightsVersion = 1;
constexpr size_t kWeightsHeader = 104;

void put_u32(uint8_t* p, uint32_t v) {
    for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
uint32_t get_u32(const uint8_t* p) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
void put_u64(uint8_t* p, uint64_t v) {
    for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
uint64_t get_u64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

uint64_t fnv1a64(const uint8_t* p, size_t n) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

bool host_little_endian() {
    const uint32_t one = 1;
    uint8_t b;
    memcpy(&b, &one, 1);
    return b == 1;
}

void encode_weights_header(const tok_arch& a, int64_t n, uint8_t* h) {
    memset(h, 0, kWeightsHeader);
    put_u32(h + 0, kWeightsMagic);
    put_u32(h + 4, kWeightsVersion);
    put_u32(h + 8, (uint32_t)a.kind);
    put_u32(h + 12, (uint32_t)a.in_ch);
    put_u32(h + 16, (uint32_t)a.nlevels);
    for (int i = 0; i < 4; ++i) put_u32(h + 20 + 4 * i, (uint32_t)a.ch[i]);
    put_u32(h + 36, (uint32_t)a.blocks);
    put_u32(h + 40, (uint32_t)a.nlev);
    for (int i = 0; i < 8; ++i) put_u32(h + 44 + 4 * i, (uint32_t)a.levels[i]);
    put_u32(h + 76, (uint32_t)a.gn_groups);
    uint32_t eps;
    memcpy(&eps, &a.gn_eps, 4);
    put_u32(h + 80, eps);
    put_u32(h + 84, (uint32_t)a.time_pad);
    put_u32(h + 88, (uint32_t)a.t_stem);
    put_u64(h + 96, (uint64_t)n);
}

bool decode_weights_header(const uint8_t* h, tok_arch* a, int64_t* n) {
    if (get_u32(h) != kWeightsMagic || get_u32(h + 4) != kWeightsVersion) return false;
    memset(a, 0, sizeof(*a));
    a->kind = (int)get_u32(h + 8);
    a->in_ch = (int)get_u32(h + 12);
    a->nlevels = (int)get_u32(h + 16);
    for (int i = 0; i < 4; ++i) a->ch[i] = (int)get_u32(h + 20 + 4 * i);
    a->blocks = (int)get_u32(h + 36);
    a->nlev = (int)get_u32(h + 40);
    for (int i = 0; i < 8; ++i) a->levels[i] = (int)get_u32(h + 44 + 4 * i);
    a->gn_groups = (int)get_u32(h + 76);
    const uint32_t eps = get_u32(h + 80);
    memcpy(&a->gn_eps, &eps, 4);
    a->time_pad = (int)get_u32(h + 84);
    a->t_stem = (int)get_u32(h + 88);
    *n = (int64_t)get_u64(h + 96);
    return true;
}

// Parameter count of an architecture (the host-side layer list only).
int64_t arch_param_total(const tok_arch& a) {
    tok_ctx tmp;
    tmp.arch = a;
    tmp.precision = TOK_BF16;
    tmp.fsq = make_fsq(a.levels, a.nlev);
    build_layers(&tmp);
    return tmp.param_total;
}

// Reads and checks a weights file's header (descriptor buildable, parameter count
// that of the descriptor, file size header + 4 n + 8).
int read_weights_header(FILE* f, tok_arch* a, int64_t* n) {
    uint8_t h[kWeightsHeader];
    if (fread(h, 1, kWeightsHeader, f) != kWeightsHeader) return TOK_EFILE;
    if (!decode_weights_header(h, a, n)) return TOK_EFILE;
    if (arch_error(*a, TOK_FP32) != TOK_OK || a->time_pad < 0 || a->time_pad > 1 || !(a->gn_eps > 0.f)) return TOK_EFILE;
    if (*n <= 0 || *n != arch_param_total(*a)) return TOK_EFILE;
    if (fseek(f, 0, SEEK_END) != 0) return TOK_EFILE;
    const long size = ftell(f);
    if (size < 0 || (uint64_t)size != kWeightsHeader + 4ull * (uint64_t)*n + 8ull) return TOK_EFILE;
    if (fseek(f, (long)kWeightsHeader, SEEK_SET) != 0) return TOK_EFILE;
    return TOK_OK;
}

}  // namespace

extern "C" {

int tok_read_weights_header(const char* path, tok_arch* arch, int64_t* param_total) {
    if (!path || !arch || !param_total) return TOK_EINVAL;
    if (!host_little_endian()) return TOK_EFILE;
    FILE* f = fopen(path, "rb");
    if (!f) return TOK_EFILE;
    const int e = read_weights_header(f, arch, param_total);
    fclose(f);
    return e;
}

int tok_save_params(tok_ctx* c, const char* path) {
    if (!c || !path) return TOK_EINVAL;
    if (!host_little_endian()) return TOK_EFILE;
    std::vector<float> p((size_t)c->param_total);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(p.data(), c->d_master, p.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TOK_ECUDA;
    uint8_t h[kWeightsHeader], tail[8];
    encode_weights_header(c->arch, c->param_total, h);
    put_u64(tail, fnv1a64(reinterpret_cast<const uint8_t*>(p.data()), p.size() * 4));
    // written next to the target and renamed into place, so a reader never sees half a file
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return TOK_EFILE;
    bool ok = fwrite(h, 1, kWeightsHeader, f) == kWeightsHeader && fwrite(p.data(), 4, p.size(), f) == p.size() &&
              fwrite(tail, 1, 8, f) == 8;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return TOK_EFILE;
    }
    return TOK_OK;
}

int tok_create_from_file(const char* path, int precision, tok_ctx** out) {
    if (!path || !out) return TOK_EINVAL;
    *out = nullptr;
    if (!host_little_endian()) return TOK_EFILE;
    FILE* f = fopen(path, "rb");
    if (!f) return TOK_EFILE;
    tok_arch a;
    int64_t n = 0;
    int e = read_weights_header(f, &a, &n);
    std::vector<float> p;
    if (!e) {
        p.resize((size_t)n);
        uint8_t tail[8];
        if (fread(p.data(), 4, p.size(), f) != p.size() || fread(tail, 1, 8, f) != 8 ||
            get_u64(tail) != fnv1a64(reinterpret_cast<const uint8_t*>(p.data()), p.size() * 4))
            e = TOK_EFILE;
    }
    fclose(f);
    if (e) return e;
    tok_ctx* c = nullptr;
    e = tok_create(&a, precision, &c);
    if (e) return e;
    for (size_t i = 0; i < c->params.size(); ++i)
        std::copy(p.begin() + c->params[i].offset, p.begin() + c->params[i].offset + c->params[i].count,
                  c->host[i].begin());
    if (cudaMemcpy(c->d_master, p.data(), p.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) e = TOK_ECUDA;
    if (!e) e = tok_repack(c, nullptr);
    if (!e && cudaDeviceSynchronize() != cudaSuccess) e = TOK_ECUDA;
    if (e) {
        tok_destroy(c);
        return e;
    }
    *out = c;
    return TOK_OK;
}

const char* tok_strerror(int code) {
    switch (code) {
        case TOK_OK: return "ok";
        case TOK_EINVAL: return "invalid argument";
        case TOK_ESHAPE: return "unsupported shape";
        case TOK_ENOMEM: return "out of device memory or workspace too small";
        case TOK_ECUDA: return "CUDA call failed";
        case TOK_ETIMEOUT: return "device-side bounded wait timed out";
        case TOK_EDEVICE: return "no usable sm_100-family device";
        case TOK_ESTATE: return "call out of order";
        case TOK_EFILE: return "weights file unreadable or malformed";
        case TOK_EGUARD: return "a workspace guard band was overwritten";
        default: return "unknown error";
    }
}

int tok_create(const tok_arch* arch, int precision, tok_ctx** out) {
    if (!arch || !out) return TOK_EINVAL;
    *out = nullptr;
    if (precision != TOK_BF16 && precision != TOK_FP32) return TOK_EINVAL;
    if (const int ea = arch_error(*arch, precision)) return ea;
    int nsm = 0;
    int e = check_cuda_device(&nsm);
    if (e) return e;
    tok_ctx* c = new tok_ctx();
    c->arch = *arch;
    c->precision = precision;
    c->num_sms = nsm;
    cudaGetDevice(&c->device);
    c->fsq = make_fsq(arch->levels, arch->nlev);
    build_layers(c);
    // initial values: He-style zeros for weights, ones for GN gamma
    for (auto& g : c->gns) std::fill(c->host[c->pindex[g.name + ".g"]].begin(), c->host[c->pindex[g.name + ".g"]].end(), 1.f);
    bool ok = cudaMalloc(&c->d_status, sizeof(int)) == cudaSuccess;
    if (ok) ok = cudaMemset(c->d_status, 0, sizeof(int)) == cudaSuccess;
    if (ok) ok = cudaMalloc(&c->d_fsq_thr, sizeof(FsqThr)) == cudaSuccess;
    if (ok) {
        const FsqThr th = make_fsq_thr(arch->levels, arch->nlev);
        ok = cudaMemcpy(c->d_fsq_thr, &th, sizeof(th), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (ok) ok = cudaMalloc(&c->d_master, (size_t)c->param_total * 4) == cudaSuccess;
    for (size_t i = 0; ok && i < c->params.size(); ++i)
        ok = cudaMemcpy(c->d_master + c->params[i].offset, c->host[i].data(), c->params[i].count * 4,
                        cudaMemcpyHostToDevice) == cudaSuccess;
    for (auto& cw : c->convs) {
        if (!ok) break;
        ok = cudaMalloc(&cw.w, (size_t)cw.Cout_pad * cw.Kpad * c->esize()) == cudaSuccess;
        if (ok) ok = upload_conv(c, cw) == TOK_OK;
    }
    for (auto& g : c->gns) {
        if (!ok) break;
        ok = upload_gn(c, g) == TOK_OK;
    }
    if (ok) ok = cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        tok_destroy(c);
        return TOK_ENOMEM;
    }
    *out = c;
    return TOK_OK;
}

void tok_destroy(tok_ctx* c) {
    if (!c) return;
    for (auto& cw : c->convs) {
        if (cw.w) cudaFree(cw.w);
        if (cw.wt) cudaFree(cw.wt);
        if (cw.wc) cudaFree(cw.wc);
        if (cw.wf0) cudaFree(cw.wf0);
    }
    if (c->d_master) cudaFree(c->d_master);
    guarded_free(c->tarena);
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_fsq_thr) cudaFree(c->d_fsq_thr);
    if (c->d_pack3_jobs) cudaFree(c->d_pack3_jobs);
    guarded_free(c->arena);
    for (auto e : c->events) cudaEventDestroy(e);
    delete c;
}

int tok_param_count(const tok_ctx* c) { return c ? (int)c->params.size() : 0; }

int tok_param_info(const tok_ctx* c, int i, const char** name, int* ndim, int64_t dims[5]) {
    if (!c || i < 0 || i >= (int)c->params.size()) return TOK_EINVAL;
    const ParamInfo& p = c->params[i];
    if (name) *name = p.name.c_str();
    if (ndim) *ndim = p.ndim;
    if (dims)
        for (int k = 0; k < 5; ++k) dims[k] = p.dims[k];
    return TOK_OK;
}

int tok_set_param(tok_ctx* c, const char* name, const float* h, int64_t count) {
    if (!c || !name || !h) return TOK_EINVAL;
    auto it = c->pindex.find(name);
    if (it == c->pindex.end()) return TOK_EINVAL;
    const ParamInfo& p = c->params[it->second];
    if (count != p.count) return TOK_ESHAPE;
    std::copy(h, h + count, c->host[it->second].begin());
    if (cudaMemcpy(c->d_master + p.offset, h, count * 4, cudaMemcpyHostToDevice) != cudaSuccess) return TOK_ECUDA;
    c->adjoint_dirty = true;
    std::string n(name);
    const std::string layer = n.substr(0, n.rfind('.'));
    int e = TOK_EINVAL;
    if (c->cindex.count(layer)) e = upload_conv(c, c->convs[c->cindex[layer]]);
    if (c->gindex.count(layer)) e = upload_gn(c, c->gns[c->gindex[layer]]);
    if (e == TOK_OK && cudaDeviceSynchronize() != cudaSuccess) e = TOK_ECUDA;
    return e;
}

size_t tok_workspace_bytes(const tok_ctx* c, int N, int T, int H, int W) {
    if (!c || N < 1 || T < 1 || H < 1 || W < 1) return 0;
    return layout_for(c, N, T, H, W).total;
}

static int reserve_bytes(tok_ctx* c, size_t need);

int tok_reserve(tok_ctx* c, int N, int T, int H, int W) {
    if (!c || N < 1 || T < 1 || H < 1 || W < 1) return TOK_EINVAL;
    return reserve_bytes(c, layout_for(c, N, T, H, W).total);
}

int tok_latent_shape(const tok_ctx* c, int T, int H, int W, int* Tq, int* Hq, int* Wq) {
    if (!c || T < 1 || H < 1 || W < 1) return TOK_EINVAL;
    if ((T - 1) % c->s_t != 0) return TOK_ESHAPE;
    const Dims d = clip_dims(c, T, H, W);
    if (Tq) *Tq = d.Tq;
    if (Hq) *Hq = d.Hq;
    if (Wq) *Wq = d.Wq;
    return TOK_OK;
}

static_assert(TOK_MAX_BATCH == tok::kMaxConvGroup, "batch size of the ABI and of the grouped launch");

// Workspace of one batch item: a clip (N, T, H, W), or one chunk of a stream
// (sized as N = 1 with s_T frames).
static size_t item_bytes(const tok_ctx* c, const tok_shape& sh) { return layout_for(c, sh.N, sh.T, sh.H, sh.W).total; }

size_t tok_batch_workspace_bytes(const tok_ctx* c, const tok_shape* shapes, int count) {
    if (!c || !shapes || count < 1 || count > TOK_MAX_BATCH) return 0;
    size_t t = 0;
    for (int p = 0; p < count; ++p) {
        const tok_shape& sh = shapes[p];
        if (sh.N < 1 || sh.T < 1 || sh.H < 1 || sh.W < 1) return 0;
        t += item_bytes(c, sh);
    }
    return t;
}

static int reserve_bytes(tok_ctx* c, size_t need) {
    if (need <= c->arena_bytes) return TOK_OK;
    if (c->arena) {
        cudaDeviceSynchronize();
        guarded_free(c->arena);
        c->arena = nullptr;
        c->arena_bytes = 0;
    }
    c->arena = guarded_alloc(need);
    if (!c->arena) return TOK_ENOMEM;
    c->arena_bytes = need;
    return TOK_OK;
}

int tok_reserve_batch(tok_ctx* c, const tok_shape* shapes, int count) {
    const size_t need = tok_batch_workspace_bytes(c, shapes, count);
    if (!need) return TOK_EINVAL;
    return reserve_bytes(c, need);
}

int tok_encode_batch(tok_ctx* c, const tok_enc_item* items, int count, void* stream) {
    if (!c || !items || count < 1 || count > TOK_MAX_BATCH) return TOK_EINVAL;
    GroupExec ex;
    ex.c = c;
    ex.s = static_cast<cudaStream_t>(stream);
    ex.P = count;
    const void* x[kMaxConvGroup];
    int N[kMaxConvGroup], T[kMaxConvGroup], H[kMaxConvGroup], W[kMaxConvGroup];
    float* z[kMaxConvGroup];
    int32_t* idx[kMaxConvGroup];
    size_t off = 0;
    for (int p = 0; p < count; ++p) {
        const tok_enc_item& it = items[p];
        if (!it.d_x || it.N < 1 || it.T < 1 || it.H < 1 || it.W < 1) return TOK_EINVAL;
        tok_shape sh{it.N, it.T, it.H, it.W};
        if (tok_stream* st = it.s) {
            // one chunk of a stream: frame 0 alone, then s_T frames per chunk
            if (!compatible(st->ctx, c) || it.N != 1 || it.H != st->H || it.W != st->W) return TOK_EINVAL;
            for (int q = 0; q < p; ++q)
                if (items[q].s == st) return TOK_EINVAL;
            if (it.T != (st->enc_chunk == 0 ? 1 : c->s_t)) return TOK_ESHAPE;
            sh = tok_shape{1, c->s_t, it.H, it.W};
            ex.pr[p].st = st;
            ex.pr[p].chunk0 = st->enc_chunk == 0;
        } else if ((it.T - 1) % c->s_t != 0) {
            return TOK_ESHAPE;
        }
        const Layout L = layout_for(c, sh.N, sh.T, sh.H, sh.W);
        ex.pr[p].w = carve(c, L, off);
        off += L.total;
        x[p] = it.d_x;
        N[p] = it.N;
        T[p] = it.T;
        H[p] = it.H;
        W[p] = it.W;
        z[p] = it.d_z;
        idx[p] = it.d_idx;
    }
    if (off > c->arena_bytes) return TOK_ENOMEM;
    ex.encode(x, N, T, H, W, z, idx);
    if (!ex.err)
        for (int p = 0; p < count; ++p)
            if (items[p].s) items[p].s->enc_chunk++;
    return ex.err;
}

// The grouped decode; item 0 may take the GoP boundary blend (blend_n > 0).
static int decode_items(tok_ctx* c, const tok_dec_item* items, int count, void* stream, const float* blend_prev,
                        int blend_Tp, int blend_n) {
    if (!c || !items || count < 1 || count > TOK_MAX_BATCH) return TOK_EINVAL;
    if (c->arch.kind != TOK_ARCH_FULL) return TOK_ESTATE;
    GroupExec ex;
    ex.c = c;
    ex.s = static_cast<cudaStream_t>(stream);
    ex.P = count;
    const int32_t* idx[kMaxConvGroup];
    int N[kMaxConvGroup], Tq[kMaxConvGroup], Hq[kMaxConvGroup], Wq[kMaxConvGroup], H[kMaxConvGroup],
        W[kMaxConvGroup];
    float* xhat[kMaxConvGroup];
    size_t off = 0;
    for (int p = 0; p < count; ++p) {
        const tok_dec_item& it = items[p];
        if (!it.d_idx || !it.d_xhat || it.N < 1 || it.Tq < 1 || it.Hq < 1 || it.Wq < 1 || it.H < 1 || it.W < 1)
            return TOK_EINVAL;
        if (it.H > it.Hq * c->s_hw || it.W > it.Wq * c->s_hw) return TOK_ESHAPE;
        Layout L;
        if (tok_stream* st = it.s) {
            // one latent frame of a stream -> 1 frame (chunk 0) or s_T frames
            if (!compatible(st->ctx, c) || it.N != 1 || it.Tq != 1) return TOK_EINVAL;
            for (int q = 0; q < p; ++q)
                if (items[q].s == st) return TOK_EINVAL;
            const Dims d = clip_dims(c, 1, st->H, st->W);
            if (it.H != st->H || it.W != st->W || it.Hq != d.Hq || it.Wq != d.Wq) return TOK_ESHAPE;
            L = layout_for(c, 1, c->s_t, it.Hq * c->s_hw, it.Wq * c->s_hw);
            ex.pr[p].st = st;
            ex.pr[p].chunk0 = st->dec_chunk == 0;
        } else {
            L = layout_for(c, it.N, 1 + c->s_t * (it.Tq - 1), it.Hq * c->s_hw, it.Wq * c->s_hw);
        }
        ex.pr[p].w = carve(c, L, off);
        off += L.total;
        idx[p] = it.d_idx;
        N[p] = it.N;
        Tq[p] = it.Tq;
        Hq[p] = it.Hq;
        Wq[p] = it.Wq;
        H[p] = it.H;
        W[p] = it.W;
        xhat[p] = it.d_xhat;
    }
    if (off > c->arena_bytes) return TOK_ENOMEM;
    if (blend_n > 0) {
        ex.pr[0].blend_prev = blend_prev;
        ex.pr[0].blend_Tp = blend_Tp;
        ex.pr[0].blend_n = blend_n;
    }
    ex.decode(idx, N, Tq, Hq, Wq, H, W, xhat);
    if (!ex.err)
        for (int p = 0; p < count; ++p)
            if (items[p].s) items[p].s->dec_chunk++;
    return ex.err;
}

int tok_decode_batch(tok_ctx* c, const tok_dec_item* items, int count, void* stream) {
    return decode_items(c, items, count, stream, nullptr, 0, 0);
}

int tok_decode_gop(tok_ctx* c, const int32_t* idx, int N, int Tq, int Hq, int Wq, int H, int W, const float* prev,
                   int T_prev, int n, float* xhat, void* stream) {
    if (!c || !idx || !xhat || N < 1 || Tq < 1 || Hq < 1 || Wq < 1 || H < 1 || W < 1 || n < 0) return TOK_EINVAL;
    if (c->arch.kind != TOK_ARCH_FULL) return TOK_ESTATE;
    const int T = 1 + c->s_t * (Tq - 1);
    if (n > 0 && (!prev || T_prev < n || T < n)) return TOK_EINVAL;
    if (n > 0 && prev == xhat) return TOK_EINVAL;
    const tok_dec_item it{idx, N, Tq, Hq, Wq, H, W, xhat, nullptr};
    return decode_items(c, &it, 1, stream, prev, T_prev, n);
}

int tok_trace_layer(tok_ctx* c, const char* name, void* in, size_t in_bytes, void* res, size_t res_bytes, void* out,
                    size_t out_bytes) {
    if (!c) return TOK_EINVAL;
    if (!name) {
        c->traces.clear();
        return TOK_OK;
    }
    std::string base(name);
    for (const char* suf : {".wgrad", ".dgrad"}) {
        const size_t n = strlen(suf);
        if (base.size() > n && base.compare(base.size() - n, n, suf) == 0) {
            base.resize(base.size() - n);
            if (!c->cindex.count(base)) return TOK_EINVAL;
        }
    }
    if (!c->cindex.count(base) && !c->gindex.count(base)) return TOK_EINVAL;
    if ((!in || !in_bytes) && (!res || !res_bytes) && (!out || !out_bytes)) return TOK_EINVAL;
    c->traces.push_back(tok_ctx::Trace{name, in_bytes ? in : nullptr, in_bytes, res_bytes ? res : nullptr, res_bytes,
                                       out_bytes ? out : nullptr, out_bytes});
    return TOK_OK;
}

int tok_set_cta_tiles(tok_ctx* c, int tiles) {
    if (!c || tiles < 0) return TOK_EINVAL;
    c->cta_tiles = tiles;
    return TOK_OK;
}

int tok_encode(tok_ctx* c, const void* x, int N, int T, int H, int W, float* z, int32_t* idx, tok_stream* st,
               void* stream) {
    if (!c || !x || N < 1 || T < 1 || H < 1 || W < 1) return TOK_EINVAL;
    const tok_enc_item it{x, N, T, H, W, z, idx, st};
    return tok_encode_batch(c, &it, 1, stream);
}

int tok_decode(tok_ctx* c, const int32_t* idx, int N, int Tq, int Hq, int Wq, int H, int W, float* xhat,
               tok_stream* st, void* stream) {
    if (!c || !idx || !xhat || N < 1 || Tq < 1 || Hq < 1 || Wq < 1 || H < 1 || W < 1) return TOK_EINVAL;
    const tok_dec_item it{idx, N, Tq, Hq, Wq, H, W, xhat, st};
    return tok_decode_batch(c, &it, 1, stream);
}

int tok_quantize(const float* z, int64_t ntok, const int* levels, int nlev, int32_t* idx, float* codes,
                 void* stream) {
    if (!z || !idx || ntok < 0 || !valid_levels(levels, nlev)) return TOK_EINVAL;
    const FsqConsts f = make_fsq(levels, nlev);
    return launch_fsq(z, ntok, f, idx, codes, static_cast<cudaStream_t>(stream)) ? TOK_ECUDA : TOK_OK;
}

int tok_dequantize(const int32_t* idx, int64_t ntok, const int* levels, int nlev, float* codes, void* stream) {
    if (!idx || !codes || ntok < 0 || !valid_levels(levels, nlev)) return TOK_EINVAL;
    const FsqConsts f = make_fsq(levels, nlev);
    return launch_dequant(idx, ntok, f, codes, static_cast<cudaStream_t>(stream)) ? TOK_ECUDA : TOK_OK;
}

int32_t tok_zero_index(const int* levels, int nlev) {
    if (!valid_levels(levels, nlev)) return -1;
    int32_t z = 0, b = 1;
    for (int i = 0; i < nlev; ++i) {
        z += (levels[i] / 2) * b;
        b *= levels[i];
    }
    return z;
}

int tok_drop_mask(const int32_t* idx, int N, int Tq, int Hq, int Wq, float rate, uint64_t seed, uint64_t stream_id,
                  uint64_t chunk_id, int32_t zero_index, int32_t* out, uint32_t* keep_bits, void* stream) {
    if (!idx || !out || N < 0 || Tq < 0 || Hq < 0 || Wq < 0 || !(rate == rate)) return TOK_EINVAL;
    double r = (double)rate;
    r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
    const unsigned long long thr = (unsigned long long)std::floor(r * 4294967296.0);
    return launch_drop(idx, N, Tq, Hq, Wq, thr, seed, stream_id, chunk_id, zero_index, out, keep_bits,
                       static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

size_t tok_similarity_workspace_bytes(int N, int Tp, int Hq, int Wq) {
    if (N < 0 || Tp < 0 || Hq < 0 || Wq < 0) return 0;
    return similarity_workspace_bytes(N, Tp, (long long)Hq * Wq);
}

int tok_similarity_mask(const int32_t* idx_p, const int32_t* idx_i, int N, int Tp, int Hq, int Wq,
                        const int* levels, int nlev, float rate, int32_t* out, uint32_t* keep_bits, float* sim,
                        void* ws, size_t ws_bytes, void* stream) {
    if (!idx_p || !idx_i || !out || !ws || N < 0 || Tp < 0 || Hq < 0 || Wq < 0 || !(rate == rate) ||
        !valid_levels(levels, nlev))
        return TOK_EINVAL;
    if (ws_bytes < similarity_workspace_bytes(N, Tp, (long long)Hq * Wq)) return TOK_ENOMEM;
    const FsqConsts f = make_fsq(levels, nlev);
    double r = (double)rate;
    r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
    const long long HW = (long long)Hq * Wq;
    long long k = (long long)std::floor(r * (double)HW);
    k = k < 0 ? 0 : (k > HW ? HW : k);
    return launch_similarity_mask(idx_p, idx_i, N, Tp, Hq, Wq, f, k, tok_zero_index(levels, nlev), out, keep_bits,
                                  sim, ws, static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int tok_residual(int precision, const void* x, const float* xhat, int N, int T, int H, int W, int C, int window,
                 float theta, float* r, void* stream) {
    if (!x || !xhat || !r || N < 0 || T < 0 || H < 0 || W < 0 || C < 1 || window < 1 || !(theta == theta))
        return TOK_EINVAL;
    if (precision != TOK_BF16 && precision != TOK_FP32) return TOK_EINVAL;
    return launch_residual_mean(precision == TOK_BF16, x, xhat, N, T, (long long)H * W * C, window, theta, r,
                                static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

size_t tok_residual_sparse_workspace_bytes(int N, int nwin, int H, int W, int C) {
    if (N < 0 || nwin < 0 || H < 0 || W < 0 || C < 0) return 0;
    return residual_sparse_workspace_bytes((long long)N * nwin, (long long)H * W * C);
}

int tok_residual_sparse(const float* r, int N, int nwin, int H, int W, int C, int32_t* pos, float* val,
                        int64_t* seg_off, void* ws, size_t ws_bytes, void* stream) {
    if (!r || !pos || !val || !seg_off || !ws || N < 0 || nwin < 0 || H < 0 || W < 0 || C < 1) return TOK_EINVAL;
    const long long E = (long long)H * W * C;
    if (E > 0x7fffffffLL) return TOK_ESHAPE;
    if (ws_bytes < residual_sparse_workspace_bytes((long long)N * nwin, E)) return TOK_ENOMEM;
    return launch_residual_sparse(r, (long long)N * nwin, E, pos, val, seg_off, ws, static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int tok_residual_apply(float* xhat, int N, int T, int H, int W, int C, int window, const int32_t* pos,
                       const float* val, const int64_t* seg_off, int64_t capacity, void* stream) {
    if (!xhat || !pos || !val || !seg_off || N < 0 || T < 0 || H < 0 || W < 0 || C < 1 || window < 1 || capacity < 0)
        return TOK_EINVAL;
    return launch_residual_apply(xhat, N, T, (long long)H * W * C, window, pos, val, seg_off, capacity,
                                 static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int tok_downsample(int in_type, const void* x, int F, int H, int W, int C, int s, int out_precision, void* y,
                   void* stream) {
    if (F < 0 || H < 1 || W < 1 || C < 1 || s < 1 || s > 8) return TOK_EINVAL;
    if (in_type != TOK_PIX_U8 && in_type != TOK_PIX_BF16 && in_type != TOK_PIX_FP32) return TOK_EINVAL;
    if (out_precision != TOK_BF16 && out_precision != TOK_FP32) return TOK_EINVAL;
    if (H < s || W < s) return TOK_ESHAPE;
    if (F == 0) return TOK_OK;
    if (!x || !y) return TOK_EINVAL;
    return launch_downsample(in_type, x, F, H, W, C, s, out_precision == TOK_BF16, y,
                             static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int tok_gop_blend(const float* prev, int Tp, const float* curr, float* out, int N, int T, int H, int W, int C, int n,
                  void* stream) {
    if (!prev || !curr || !out || N < 0 || T < 0 || Tp < 0 || H < 0 || W < 0 || C < 1 || n < 0 || n > T || n > Tp)
        return TOK_EINVAL;
    return launch_gop_blend(prev, Tp, curr, out, N, T, (long long)H * W * C, n, static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

size_t tok_temporal_loss_workspace_bytes(int N, int n, int H, int W, int C) {
    if (N < 0 || n < 0 || H < 0 || W < 0 || C < 0) return 0;
    return temporal_loss_workspace_bytes(N, n, (long long)H * W * C);
}

int tok_temporal_loss(const float* xc, const float* xp, int N, int Tc, int Tp, int H, int W, int C, int n,
                      float* loss, float* grad, void* ws, size_t ws_bytes, void* stream) {
    if (!xc || !xp || !loss || !ws || N < 1 || Tc < 0 || Tp < 0 || H < 1 || W < 1 || C < 1 || n < 1 || n > Tc ||
        n > Tp)
        return TOK_EINVAL;
    if (ws_bytes < temporal_loss_workspace_bytes(N, n, (long long)H * W * C)) return TOK_ENOMEM;
    return launch_temporal_loss(xc, xp, N, Tc, Tp, (long long)H * W * C, n, loss, grad, ws,
                                static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int tok_pack_rows(const int32_t* idx, const uint32_t* keep_bits, int64_t rows, int Wq, int32_t* payload,
                  int64_t* row_offsets, void* stream) {
    if (!idx || !keep_bits || !payload || !row_offsets || rows < 0 || Wq < 1) return TOK_EINVAL;
    return launch_pack(idx, keep_bits, rows, Wq, payload, row_offsets, static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int tok_unpack_rows(const int32_t* payload, const int64_t* row_offsets, const uint32_t* keep_bits,
                    const uint8_t* row_received, int64_t rows, int Wq, int32_t zero_index, int32_t* idx,
                    void* stream) {
    if (!payload || !row_offsets || !keep_bits || !idx || rows < 0 || Wq < 1) return TOK_EINVAL;
    return launch_unpack(payload, row_offsets, keep_bits, row_received, rows, Wq, zero_index, idx,
                         static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

size_t tok_stream_bytes(const tok_ctx* c, int H, int W) {
    if (!c || H < 1 || W < 1) return 0;
    size_t total = 2 * kGuardBytes;  // the guard bands of its allocation
    for (const auto& kv : stream_frames(c, H, W)) total += align256(2 * kv.second);
    return total;
}

int tok_stream_open(tok_ctx* c, int H, int W, tok_stream** out) {
    if (!c || !out || H < 1 || W < 1) return TOK_EINVAL;
    *out = nullptr;
    const size_t bytes = tok_stream_bytes(c, H, W) - 2 * kGuardBytes;
    tok_stream* st = new tok_stream();
    st->ctx = c;
    st->H = H;
    st->W = W;
    st->mem = guarded_alloc(bytes);
    if (!st->mem) {
        delete st;
        return TOK_ENOMEM;
    }
    st->bytes = bytes;
    char* p = st->mem;
    for (const auto& kv : stream_frames(c, H, W)) {
        st->hist[kv.first] = p;
        st->frame_bytes[kv.first] = kv.second;
        p += align256(2 * kv.second);
    }
    *out = st;
    return TOK_OK;
}

void tok_stream_close(tok_stream* s) {
    if (!s) return;
    guarded_free(s->mem);
    delete s;
}

int tok_check_guards(tok_ctx* c) {
    if (!c) return TOK_EINVAL;
    const int e = guards_check(c->arena, c->arena_bytes);
    return e ? e : guards_check(c->tarena, c->tbytes);
}

int tok_selftest_guards(tok_ctx* c) {
    if (!c) return TOK_EINVAL;
    if (!c->arena) return TOK_ESTATE;
    if (tok_check_guards(c) != TOK_OK) return TOK_EGUARD;
    char* band = c->arena + c->arena_bytes;  // the trailing band
    if (cudaMemset(band + 17, kGuardByte ^ 0xFF, 1) != cudaSuccess) return TOK_ECUDA;
    const bool caught = tok_check_guards(c) == TOK_EGUARD;
    if (cudaMemset(band + 17, kGuardByte, 1) != cudaSuccess) return TOK_ECUDA;
    const bool clean = tok_check_guards(c) == TOK_OK;
    return caught && clean ? TOK_OK : TOK_EGUARD;
}

int tok_stream_check_guards(tok_stream* s) {
    if (!s) return TOK_EINVAL;
    return guards_check(s->mem, s->bytes);
}

int tok_stream_reset(tok_stream* s) {
    if (!s) return TOK_EINVAL;
    s->enc_chunk = 0;
    s->dec_chunk = 0;
    return TOK_OK;
}

size_t tok_conv3d_workspace_bytes(int precision, int Cin, int Cout, int k) {
    if ((precision != TOK_BF16 && precision != TOK_FP32) || Cin < 1 || Cout < 1 || (k != 1 && k != 3)) return 0;
    const int taps = k * k * k;
    if (precision == TOK_BF16) {
        const int c16 = round_up(Cout, 16);
        const int cp = conv_tc_cout_pad(c16);
        return align256((size_t)cp * taps * Cin * 2);
    }
    return align256((size_t)round_up(Cout, 16) * round_up(taps * Cin, 8) * 4);
}

int tok_conv3d(int precision, const void* x, int N, int T, int H, int W, int Cin, const float* w,
               const float* bias, int Cout, int k, int st, int sh, int sw, int time_pad, const void* residual,
               void* y, void* ws, size_t ws_bytes, void* stream) {
    if (!x || !w || !y || N < 1 || T < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1) return TOK_EINVAL;
    if (precision != TOK_BF16 && precision != TOK_FP32) return TOK_EINVAL;
    if ((k != 1 && k != 3) || st < 1 || st > 2 || sh < 1 || sh > 2 || sh != sw) return TOK_EINVAL;
    if (time_pad != TOK_PAD_REPLICATE && time_pad != TOK_PAD_ZERO) return TOK_EINVAL;
    const size_t need = tok_conv3d_workspace_bytes(precision, Cin, Cout, k);
    if (!ws || ws_bytes < need) return TOK_ENOMEM;
    const bool bf = precision == TOK_BF16;
    if (bf && (Cin % 64 != 0 || (sh == 2 && (H % 2 || W % 2 || k != 3)))) return TOK_ESHAPE;
    if (!bf && (Cin % 4 != 0 && Cin > 8)) return TOK_ESHAPE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nsm = 148;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int taps = k * k * k;
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    if (bf) {
        const int c16 = round_up(Cout, 16);
        a.Cout_pad = conv_tc_cout_pad(c16);
        a.Kpad = taps * Cin;
        // narrow 3x3x3 stride-1 heads: the dw taps as MMA rows (same workspace bound)
        a.w_dwm = conv_tc_taprows(Cout, Cin, k, sh, sw);
        const int e = a.w_dwm ? launch_pack_weights_taprows(w, Cout, Cin, a.Cout_pad, a.w_dwm,
                                                            static_cast<__nv_bfloat16*>(ws), s)
                              : launch_pack_weights<__nv_bfloat16>(w, Cout, taps * Cin, a.Cout_pad, a.Kpad,
                                                                   static_cast<__nv_bfloat16*>(ws), s);
        if (e) return TOK_ECUDA;
    } else {
        a.Cout_pad = round_up(Cout, 16);
        a.Kpad = round_up(taps * Cin, 8);
        if (launch_pack_weights<float>(w, Cout, taps * Cin, a.Cout_pad, a.Kpad, static_cast<float*>(ws), s))
            return TOK_ECUDA;
    }
    a.x = x;
    a.N = N;
    a.Tin = T;
    a.Hin = H;
    a.Win = W;
    a.Cin = Cin;
    a.w = ws;
    a.bias = bias;
    a.Cout = Cout;
    a.kt = a.kh = a.kw = k;
    a.st = st;
    a.sh = sh;
    a.sw = sw;
    a.t_off = -(k - 1);
    a.pad_mode = time_pad;
    a.Tout = (T - 1) / st + 1;
    a.Hout = (H + 2 * ((k - 1) / 2) - k) / sh + 1;
    a.Wout = (W + 2 * ((k - 1) / 2) - k) / sw + 1;
    a.mode = OUT_PLAIN;
    a.out = y;
    a.residual = residual;
    a.oT = a.Tout;
    a.oH = a.Hout;
    a.oW = a.Wout;
    a.oC = Cout;
    a.wait_ns = kWaitNs;
    const int e = bf ? launch_conv_tc(a, nsm, s) : launch_conv_simt(a, s);
    return e ? TOK_ECUDA : TOK_OK;
}

size_t tok_groupnorm_workspace_bytes(int precision, int64_t frames, int64_t HW, int C, int G) {
    if ((precision != TOK_BF16 && precision != TOK_FP32) || frames < 1 || HW < 1 || C < 1 || G < 1) return 0;
    int nsm = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return gn_scratch_bytes(frames, HW, C, G, nsm, precision == TOK_BF16 ? 8 : 4);
}

int tok_groupnorm_silu(int precision, const void* x, int64_t frames, int64_t HW, int C, int G, const float* gamma,
                       const float* beta, float eps, void* y, void* ws, size_t ws_bytes, void* stream) {
    if (!x || !y || frames < 1 || HW < 1 || C < 1 || G < 1 || !(eps >= 0.f)) return TOK_EINVAL;
    if (precision != TOK_BF16 && precision != TOK_FP32) return TOK_EINVAL;
    const int V = precision == TOK_BF16 ? 8 : 4;
    const int vpv = C / V;
    if (C % V || C % G || C / G < 2 || G > 64 || vpv > 256 || (vpv & (vpv - 1))) return TOK_ESHAPE;
    const int cg = C / G;
    if (!(cg % V == 0 || V % cg == 0)) return TOK_ESHAPE;
    const size_t need = tok_groupnorm_workspace_bytes(precision, frames, HW, C, G);
    if (!ws || ws_bytes < need) return TOK_ENOMEM;
    int nsm = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int e;
    if (precision == TOK_BF16)
        e = launch_gn_silu<__nv_bfloat16>(static_cast<const __nv_bfloat16*>(x), static_cast<__nv_bfloat16*>(y),
                                          frames, HW, C, G, gamma, beta, eps, ws, nsm, true, s);
    else
        e = launch_gn_silu<float>(static_cast<const float*>(x), static_cast<float*>(y), frames, HW, C, G, gamma,
                                  beta, eps, ws, nsm, false, s);
    return e ? TOK_ECUDA : TOK_OK;
}

int tok_status(tok_ctx* c) {
    if (!c) return TOK_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return TOK_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TOK_ECUDA;
    if (v) cudaMemset(c->d_status, 0, sizeof(int));
    return v;
}

int tok_selftest_timeout(tok_ctx* c, int64_t limit_ns, void* stream) {
    if (!c || limit_ns <= 0) return TOK_EINVAL;
    c->launches++;
    return launch_timeout_selftest(c->d_status, (unsigned long long)limit_ns, static_cast<cudaStream_t>(stream))
               ? TOK_ECUDA
               : TOK_OK;
}

int64_t tok_launch_count(const tok_ctx* c) { return c ? c->launches : 0; }

int tok_profile_enable(tok_ctx* c, int on) {
    if (!c) return TOK_EINVAL;
    if (on && c->events.empty()) {
        c->events.resize(8192);
        for (auto& e : c->events)
            if (cudaEventCreate(&e) != cudaSuccess) return TOK_ECUDA;
    }
    if (!on) {
        cudaDeviceSynchronize();
        for (auto e : c->events) cudaEventDestroy(e);
        c->events.clear();
    }
    c->prof = on != 0;
    c->recs.clear();
    c->ev_used = 0;
    return TOK_OK;
}

int tok_profile_records(tok_ctx* c, tok_profile_record* out, int cap, int* count) {
    if (!c || !count || cap < 0 || (cap > 0 && !out)) return TOK_EINVAL;
    *count = (int)c->recs.size();
    for (int i = 0; i < (int)c->recs.size() && i < cap; ++i) {
        const auto& r = c->recs[i];
        if (cudaEventSynchronize(c->events[r.ev + 1]) != cudaSuccess) return TOK_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->events[r.ev], c->events[r.ev + 1]);
        out[i].cls = r.cls;
        out[i].ms = ms;
        out[i].work = r.work;
        memcpy(out[i].name, r.name, sizeof(out[i].name));
    }
    return TOK_OK;
}

int tok_profile_read(tok_ctx* c, tok_profile_stats* out) {
    if (!c || !out) return TOK_EINVAL;
    memset(out, 0, sizeof(*out));
    for (const auto& r : c->recs) {
        if (cudaEventSynchronize(c->events[r.ev + 1]) != cudaSuccess) return TOK_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->events[r.ev], c->events[r.ev + 1]);
        if (r.cls == 0) {
            out->conv_launches++;
            out->conv_ms += ms;
            out->conv_flop += r.work;
        } else if (r.cls == 1) {
            out->gn_launches++;
            out->gn_ms += ms;
            out->gn_bytes += r.work;
        } else {
            out->other_launches++;
            out->other_ms += ms;
            out->other_bytes += r.work;
        }
    }
    c->recs.clear();
    c->ev_used = 0;
    return TOK_OK;
}

}  // extern "C"
