/*
 * morphe-tok: C-ABI of a B300-native causal video tokenizer (sm_103a).
 *
 * The library implements the data-parallel hot path of a VFM-based
 * generative video codec: the encoder f_phi that maps a clip
 * x_{0:T} in R^{(1+T) x H x W x 3} to a latent z_{0:T'} in
 * R^{(1+T') x H' x W' x C} with temporal factor s_T = 4 and spatial factor
 * s_HW = 8 (paper Sec. 2.4; the 4x/8x8 setting of Sec. 4.1), a finite scalar
 * quantiser that turns z into the integer token matrix that is transmitted
 * (Sec. 4.3, Sec. 6.2), packet-drop masking with zero fill of dropped tokens
 * and lost rows (Sec. 6.2; joint training with random drop, Appendix A.2),
 * and the mirrored decoder g_theta.
 *
 * Conventions for every entry point:
 *  - Tensors are channels-last, contiguous: x is (N, T, H, W, 3); latents
 *    are (N, T', H', W', C); token indices are (N, T', H', W') int32.
 *  - Pointers named d_* are device pointers (cudaMalloc'd or equivalent);
 *    h_* are host pointers. The caller owns every tensor it passes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls that take a stream are asynchronous on it: they enqueue
 *    work and return without synchronising; outputs are valid once the
 *    stream reaches that point.
 *  - Return value: TOK_OK (0) or a negative-free error code below. Argument
 *    and shape errors are detected on the host before anything is enqueued;
 *    nothing is written in that case. Device-side errors (a bounded wait that
 *    ran out) are recorded in the context's device status word and returned
 *    by tok_status() and by the next call on that context.
 *  - No entry point allocates device memory except tok_create, tok_reserve
 *    and tok_stream_open; no C++ exception crosses the ABI.
 */
#ifndef MORPHE_TOK_H
#define MORPHE_TOK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tok_ctx tok_ctx;
typedef struct tok_stream tok_stream;

enum tok_err {
    TOK_OK = 0,
    TOK_EINVAL = 1,    /* bad argument (null pointer, unknown name, bad enum) */
    TOK_ESHAPE = 2,    /* shape not supported (e.g. T != 1 mod 4) */
    TOK_ENOMEM = 3,    /* device allocation failed, or workspace too small */
    TOK_ECUDA = 4,     /* a CUDA runtime/driver call failed */
    TOK_ETIMEOUT = 5,  /* a device-side bounded wait ran out (kernel returned early) */
    TOK_EDEVICE = 6,   /* no usable sm_100-family device */
    TOK_ESTATE = 7,    /* call out of order (e.g. weights not set, stream misuse) */
    TOK_EFILE = 8,     /* weights file missing, unreadable, malformed or corrupt */
    TOK_EGUARD = 9     /* a workspace guard band was overwritten (tok_check_guards) */
};

enum tok_precision { TOK_BF16 = 1, TOK_FP32 = 2 };
enum tok_time_pad { TOK_PAD_REPLICATE = 0, TOK_PAD_ZERO = 1 };
enum tok_arch_kind { TOK_ARCH_FULL = 0, TOK_ARCH_STAGE = 1 };
/* pixel element types of tok_downsample's input (bf16 / fp32 match tok_precision) */
enum tok_pixel_type { TOK_PIX_U8 = 0, TOK_PIX_BF16 = 1, TOK_PIX_FP32 = 2 };

/* Architecture descriptor. The paper gives no layer list (it builds on a
 * published video tokenizer, Sec. 7); this descriptor is the reading used:
 *  FULL : stem conv k3 stride (t_stem,2,2) -> per level l < nlevels: `blocks`
 *         causal residual blocks at ch[l] (GN->SiLU->conv->GN->SiLU->conv,
 *         1x1x1 skip conv when channels change), a k3 stride-(2,2,2) conv
 *         between levels -> GN->SiLU->conv to zdim -> FSQ. The decoder mirrors
 *         it with k3 convs to ch[l-1]*8 channels + depth-to-space (2,2,2),
 *         and a final conv to 3*4*t_stem channels + depth-to-space
 *         (t_stem,2,2). t_stem = 1 is the 4x temporal / 8x8 spatial setting
 *         with 3 levels; t_stem = 2 the 8x temporal / 8x8 spatial one (Sec. 4.1),
 *         which makes s_T = t_stem * 2^(nlevels-1) frames per latent frame.
 *  STAGE: conv k3 in->ch[0] -> conv k3 stride (1,2,2) ch[0]->ch[1] ->
 *         GN->SiLU -> 1x1x1 conv ch[1]->zdim -> FSQ (encoder only).
 * GroupNorm statistics are per (sample, group, frame) (causal); the group
 * count of a C-channel norm is min(gn_groups, C/2). */
typedef struct tok_arch {
    int kind;            /* tok_arch_kind */
    int in_ch;           /* pixel channels, must be 3 */
    int nlevels;         /* FULL: 1..4 levels; STAGE: 2 */
    int ch[4];           /* channels per level, multiples of 64 on the BF16 path */
    int blocks;          /* residual blocks per level (FULL) */
    int nlev;            /* number of FSQ channels = latent dim (<= 8) */
    int levels[8];       /* FSQ levels, each 2..16 */
    int gn_groups;       /* 32 */
    float gn_eps;        /* 1e-6 */
    int time_pad;        /* tok_time_pad for the causal left padding */
    int t_stem;          /* FULL: temporal stride of the stem, 1 or 2 (default 1) */
} tok_arch;

/* Fill `a` with the default tokenizer: FULL, ch {128,256,512}, 2 blocks per
 * level, FSQ levels {8,8,8,5,5,5}, GroupNorm(32) eps 1e-6, replicate pad. */
void tok_arch_default(tok_arch* a);

/* Create a context on the current CUDA device. `precision` selects the
 * compute path: TOK_BF16 (tcgen05 tensor cores, BF16 activations and
 * weights, FP32 accumulation and norm statistics) or TOK_FP32 (CUDA-core FP32
 * everywhere, no TF32). Allocates the weights on the device (zeros until
 * set). Returns TOK_EDEVICE if the device is not sm_100-family. */
int tok_create(const tok_arch* arch, int precision, tok_ctx** out);
void tok_destroy(tok_ctx* ctx);

/* Weights files: the flat FP32 parameters (tok_param_info order) with the
 * descriptor they belong to. Layout (little-endian): a 104-byte header
 *   0 "TOKW"  4 version 1  8 kind  12 in_ch  16 nlevels  20 ch[4]  36 blocks
 *   40 nlev  44 levels[8]  76 gn_groups  80 gn_eps (float32)  84 time_pad
 *   88 t_stem  92 zero  96 n = parameter count (int64)
 * then n float32 values, then the 64-bit FNV-1a hash of those 4n bytes.
 * tok_save_params writes the context's parameters (synchronous; through a
 * temporary file renamed into place). tok_create_from_file creates a context
 * on the current device from such a file (as tok_create, then the weights).
 * tok_read_weights_header reads and checks a file's header on the host (no
 * device): the descriptor must be one tok_create builds, n its parameter
 * count, the file size 104 + 4n + 8. Errors: TOK_EFILE (missing, short,
 * malformed, wrong count, hash mismatch), and tok_create's. */
int tok_save_params(tok_ctx* ctx, const char* path);
int tok_create_from_file(const char* path, int precision, tok_ctx** out);
int tok_read_weights_header(const char* path, tok_arch* arch, int64_t* param_total);

/* Parameter list in the architecture's order: name (owned by the context,
 * valid until tok_destroy), rank and dims. Conv weights are
 * (Cout, kt, kh, kw, Cin); biases, GN gamma/beta are (C). */
int tok_param_count(const tok_ctx* ctx);
int tok_param_info(const tok_ctx* ctx, int i, const char** name, int* ndim, int64_t dims[5]);
/* Copy one parameter from host FP32 memory (synchronous). The BF16 path
 * rounds weights to nearest-even BF16 and re-lays them out for TMA. */
int tok_set_param(tok_ctx* ctx, const char* name, const float* h_values, int64_t count);

/* Workspace for clips of up to N x T x H x W pixels (bytes), and reserve it
 * (allocates once; later calls with larger shapes grow it). Hot calls never
 * allocate: tok_encode/tok_decode return TOK_ENOMEM if the reserved
 * workspace is smaller than they need. */
size_t tok_workspace_bytes(const tok_ctx* ctx, int N, int T, int H, int W);
int tok_reserve(tok_ctx* ctx, int N, int T, int H, int W);

/* Latent / token shape of an N x T x H x W clip: T' = 1 + (T-1)/s_T
 * (requires T = 1 mod s_T), H' = ceil(H/s_HW), W' = ceil(W/s_HW). */
int tok_latent_shape(const tok_ctx* ctx, int T, int H, int W, int* Tq, int* Hq, int* Wq);

/* Encoder f_phi (Sec. 2.4) + FSQ.
 * d_x    : (N,T,H,W,3) pixels in [-1,1]; bf16 on the BF16 path, fp32 on FP32.
 *          H and W need not be multiples of 8: the frame is edge-extended.
 * d_z    : (N,T',H',W',nlev) fp32 pre-quantisation latent, or NULL.
 * d_idx  : (N,T',H',W') int32 token indices, or NULL.
 * s      : NULL for a whole clip (causal padding at frame 0); a stream
 *          handle for chunked streaming (see tok_stream_open).
 * Errors: TOK_ESHAPE if T != 1 mod s_T in clip mode. */
int tok_encode(tok_ctx* ctx, const void* d_x, int N, int T, int H, int W,
               float* d_z, int32_t* d_idx, tok_stream* s, void* stream);

/* Decoder g_theta (Sec. 2.4): token indices -> pixels.
 * d_idx  : (N,Tq,Hq,Wq) int32 indices in [0, prod(levels)); the zero-code
 *          index stands for a dropped/lost token (Sec. 6.2).
 * d_xhat : (N, 1 + s_T*(Tq-1), H, W, 3) fp32, cropped to H x W
 *          (H <= s_HW*Hq, W <= s_HW*Wq). */
int tok_decode(tok_ctx* ctx, const int32_t* d_idx, int N, int Tq, int Hq, int Wq,
               int H, int W, float* d_xhat, tok_stream* s, void* stream);

/* Lifetime of the conv CTAs of this context's tok_encode / tok_decode
 * launches: 0 (default) one persistent CTA per SM that loops over all tiles
 * of a layer; n > 0 at most n output tiles per CTA. A context whose work runs
 * on a low-priority CUDA stream beside latency-critical work on a
 * high-priority stream sets a small n, so that the critical kernels get SMs
 * as soon as a short CTA ends rather than after a whole layer. Results do
 * not depend on n. Not in the paper: a serving control. */
int tok_set_cta_tiles(tok_ctx* ctx, int tiles);

/* Grouped encode / decode (one launch per layer over several inputs).
 * A batch holds 1 .. TOK_MAX_BATCH items of any sizes: whole clips, chunks of
 * streams (each stream at most once per batch), or both. Every convolution
 * of a layer runs as one tensor-core launch over all items, every
 * GroupNorm+SiLU as one grouped pass; tiles never span items, so each
 * item's result is the one its own tok_encode / tok_decode call gives.
 * Item fields mean what the arguments of tok_encode / tok_decode mean; the
 * workspace is the sum of the items' workspaces, laid out item after item
 * (tok_reserve_batch; a stream chunk counts as N = 1, T = s_T). Errors: the
 * first argument error of any item, before anything is launched; TOK_ENOMEM
 * if the reserved workspace is too small. Not in the paper: a serving and
 * throughput device for mixed-resolution inputs. */
#define TOK_MAX_BATCH 8
typedef struct tok_shape {
    int N, T, H, W;
} tok_shape;
typedef struct tok_enc_item {
    const void* d_x;
    int N, T, H, W;
    float* d_z;      /* or NULL */
    int32_t* d_idx;  /* or NULL */
    tok_stream* s;   /* NULL: a whole clip */
} tok_enc_item;
typedef struct tok_dec_item {
    const int32_t* d_idx;
    int N, Tq, Hq, Wq, H, W;
    float* d_xhat;
    tok_stream* s;   /* NULL: a whole clip */
} tok_dec_item;
size_t tok_batch_workspace_bytes(const tok_ctx* ctx, const tok_shape* h_shapes, int count);
int tok_reserve_batch(tok_ctx* ctx, const tok_shape* h_shapes, int count);
int tok_encode_batch(tok_ctx* ctx, const tok_enc_item* h_items, int count, void* stream);
int tok_decode_batch(tok_ctx* ctx, const tok_dec_item* h_items, int count, void* stream);

/* Stand-alone FSQ (Mentzer et al. 2023): per token of nlev channels,
 * b = tanh(z + atanh(o/h))*h - o with h = (L-1)(1-1e-3)/2, o = 0.5 for even
 * L else 0; q = round-half-even(b); idx = sum (q + L/2) * prod_{j<i} L_j;
 * codes = q / floor(L/2) (FP32). The rounding of b is taken exactly for the
 * float32 z: per channel the L-1 bounds in z where q steps (tanh is
 * increasing) are precomputed in double, and q + L/2 is the number of them z
 * passes; no tanh is evaluated. 16-byte aligned d_z and d_idx (and d_codes)
 * take a vectorised form; any alignment is accepted.
 * d_z (ntok, nlev) fp32; h_levels host array of nlev levels (<= 8);
 * d_idx (ntok) int32; d_codes (ntok, nlev) fp32 or NULL. */
int tok_quantize(const float* d_z, int64_t ntok, const int* h_levels, int nlev,
                 int32_t* d_idx, float* d_codes, void* stream);

/* Index -> code vectors: codes_i = (digit_i - L_i/2) / floor(L_i/2). */
int tok_dequantize(const int32_t* d_idx, int64_t ntok, const int* h_levels, int nlev,
                   float* d_codes, void* stream);

/* Index of the all-zero code vector (the zero-fill token of Sec. 6.2). */
int32_t tok_zero_index(const int* h_levels, int nlev);

/* Packet-drop token masking (Sec. 4.3 token dropping; Sec. 6.2 zero fill;
 * random drop of Appendix A.2). Token j = (t*Hq + h)*Wq + w of sample n is
 * dropped iff word (j & 3) of Philox-4x32-10(counter = (j>>2, n,
 * chunk_id mod 2^32, stream_id mod 2^32), key = (seed mod 2^32, seed>>32))
 * is below floor(rate * 2^32) (rate clipped to [0,1]).
 * d_idx (N,Tq,Hq,Wq) int32 in; d_out (same) gets the zero index at dropped
 * tokens (may alias d_idx); d_keep_bits, if not NULL, gets the row masks of
 * the packet headers: (N,Tq,Hq, ceil(Wq/32)) uint32, bit w%32 of word w/32 set
 * when token w of the row is kept. */
int tok_drop_mask(const int32_t* d_idx, int N, int Tq, int Hq, int Wq, float rate,
                  uint64_t seed, uint64_t stream_id, uint64_t chunk_id, int32_t zero_index,
                  int32_t* d_out, uint32_t* d_keep_bits, void* stream);

/* Similarity-based token selection (Sec. 6.3, Eq. 3). For every P-frame
 * token, S = <p, q> / (|p| |q|) between its code vector p and the code vector
 * q of the I-frame token at the same (sample, h, w) (S = 0 where either is
 * the zero vector); per sample and P latent frame the k = floor(rate * Hq*Wq)
 * tokens with the largest S are dropped (rate clipped to [0,1]; among equal S
 * the lower linear index h*Wq + w first), i.e. the threshold tau of Eq. 3 is
 * the (1 - rate)-quantile of S. S is computed in float32 with the rounding
 * steps of the definition (exact dot and squared norms, one rounded square
 * root of the squared-norm product, one rounded division), so the selection
 * is a deterministic function of the indices.
 * d_idx_p (N,Tp,Hq,Wq) int32 P tokens; d_idx_i (N,1,Hq,Wq) int32 I tokens;
 * d_out (N,Tp,Hq,Wq) int32 (zero index at dropped tokens; may alias
 * d_idx_p); d_keep_bits (N,Tp,Hq,ceil(Wq/32)) uint32 row masks as in
 * tok_drop_mask, or NULL; d_sim (N,Tp,Hq,Wq) fp32 similarities, or NULL;
 * d_ws device workspace of tok_similarity_workspace_bytes(...) bytes.
 * Errors: TOK_EINVAL (arguments, levels), TOK_ENOMEM (workspace too small). */
size_t tok_similarity_workspace_bytes(int N, int Tp, int Hq, int Wq);
int tok_similarity_mask(const int32_t* d_idx_p, const int32_t* d_idx_i, int N, int Tp, int Hq, int Wq,
                        const int* h_levels, int nlev, float rate, int32_t* d_out, uint32_t* d_keep_bits,
                        float* d_sim, void* d_ws, size_t ws_bytes, void* stream);

/* Pixel residuals (Sec. 6.3, Eq. 4). Sender: r = x - x_hat per pixel and
 * channel (x_hat a reconstruction of x, e.g. tok_decode(tok_encode(x))),
 * averaged over windows of `window` consecutive frames ([0,w), [w,2w), ...;
 * the last may be shorter): r_c = (1/T_w) sum_t r, then zeroed where
 * |r_c| < theta. float32 with the definition's rounding steps (differences
 * summed in frame order, one division), since theta decides which elements
 * are sent. precision: TOK_BF16 or TOK_FP32 for d_x (N,T,H,W,C); d_xhat
 * (N,T,H,W,C) fp32; d_r (N, ceil(T/window), H, W, C) fp32.
 * The arithmetic coding of the sparse residual (Sec. 6.3) is not part of this
 * library. */
int tok_residual(int precision, const void* d_x, const float* d_xhat, int N, int T, int H, int W, int C,
                 int window, float theta, float* d_r, void* stream);
/* Sparse form of d_r: per (sample, window) segment s = n*n_windows + k, the
 * nonzero elements in position order, position = (h*W + w)*C + c;
 * d_pos int32 / d_val fp32 hold up to N*n_windows*H*W*C entries (caller
 * allocates the worst case); d_seg_offsets int64 (N*n_windows + 1): segment s
 * occupies [off[s], off[s+1]). d_ws: tok_residual_sparse_workspace_bytes. */
size_t tok_residual_sparse_workspace_bytes(int N, int n_windows, int H, int W, int C);
int tok_residual_sparse(const float* d_r, int N, int n_windows, int H, int W, int C, int32_t* d_pos,
                        float* d_val, int64_t* d_seg_offsets, void* d_ws, size_t ws_bytes, void* stream);
/* Receiver: every frame t of window k gets that window's residual added,
 * d_xhat[n,t] += r_c[n,k] (fp32, in place). capacity = the length of
 * d_pos / d_val (entries past d_seg_offsets[N*n_windows] are ignored). */
int tok_residual_apply(float* d_xhat, int N, int T, int H, int W, int C, int window, const int32_t* d_pos,
                       const float* d_val, const int64_t* d_seg_offsets, int64_t capacity, void* stream);

/* Resolution control (Sec. 5): downsampling of frames by an integer factor
 * s before encoding (the paper uses 2x and 3x of 1080p). Reading: each output
 * pixel is the mean of the s x s input block it covers (area filter, blocks
 * anchored at the top-left corner); Ho = H/s, Wo = W/s rounded down, trailing
 * rows and columns unused. The mean is float32 in a fixed order (float input:
 * summed row by row, left to right, then one division by s*s; uint8 input:
 * exact integer sum, division by s*s, then m / 127.5 - 1 into [-1, 1]) and
 * rounded to the output type (bf16: to nearest, ties to even).
 * d_x (F,H,W,C) channels-last frames of in_type (tok_pixel_type); d_y
 * (F,Ho,Wo,C) of out_precision (TOK_BF16 or TOK_FP32). 1 <= s <= 8; F = 0
 * is a no-op (the pointers may then be NULL).
 * Errors: TOK_EINVAL (pointers, types, s), TOK_ESHAPE (H < s or W < s). */
int tok_downsample(int in_type, const void* d_x, int F, int H, int W, int C, int s, int out_precision, void* d_y,
                   void* stream);

/* GoP boundary blending (Sec. 6.1, Eq. 2): for i = 1..n, frame i of the
 * current GoP becomes a_i * prev[T_prev-n+i] + (1 - a_i) * curr[i] with
 * a_i = (n - i)/n (1-based frame numbers); the other frames are copied.
 * d_prev (N,T_prev,H,W,C), d_curr and d_out (N,T,H,W,C) fp32 (d_out may
 * alias d_curr); 0 <= n <= min(T_prev, T). */
int tok_gop_blend(const float* d_prev, int T_prev, const float* d_curr, float* d_out, int N, int T, int H, int W,
                  int C, int n, void* stream);
/* GoP boundary loss (Sec. 6.1, Eq. 1): L = (1/n) sum_{i=1..n}
 * ||xhat_curr[i] - x_prev[T_prev-n+i]||, averaged over the batch, the norm
 * being the Euclidean norm of the whole frame difference (the paper leaves it
 * open). d_loss: one fp32; d_grad (N,T_curr,H,W,C) fp32 dL/dxhat_curr or NULL
 * (zero outside the first n frames; add it to the reconstruction gradient
 * given to tok_backward). Deterministic (fixed-order FP64 sums). d_ws:
 * tok_temporal_loss_workspace_bytes. */
/* A GoP's decode with the boundary blend (Sec. 6.1, Eq. 2) fused into the
 * pixel head's epilogue: tok_decode of a whole clip (N, Tq, Hq, Wq tokens ->
 * d_xhat (N,T,H,W,3) fp32, T = 1 + s_T (Tq - 1)) whose first n frames are
 * blended as tok_gop_blend blends them, with the last n frames of the
 * previous GoP's reconstruction d_prev (N,T_prev,H,W,3) fp32; the result is
 * bitwise that of tok_decode followed by tok_gop_blend, without the extra
 * pass over the frames. n = 0: plain tok_decode. Errors: TOK_EINVAL
 * (pointers, n > min(T_prev, T), d_prev == d_xhat), as tok_decode otherwise. */
int tok_decode_gop(tok_ctx* ctx, const int32_t* d_idx, int N, int Tq, int Hq, int Wq, int H, int W,
                   const float* d_prev, int T_prev, int n, float* d_xhat, void* stream);
size_t tok_temporal_loss_workspace_bytes(int N, int n, int H, int W, int C);
int tok_temporal_loss(const float* d_xhat_curr, const float* d_x_prev, int N, int T_curr, int T_prev, int H, int W,
                      int C, int n, float* d_loss, float* d_grad, void* d_ws, size_t ws_bytes, void* stream);

/* Row packetisation (Sec. 6.2). rows = N*Tq*Hq rows of Wq tokens.
 * Sender: d_payload gets, row after row, the kept tokens of each row in
 * column order, starting at d_row_offsets[r] = number of kept tokens in rows
 * < r (d_row_offsets has rows+1 entries; both computed here). */
int tok_pack_rows(const int32_t* d_idx, const uint32_t* d_keep_bits, int64_t rows, int Wq,
                  int32_t* d_payload, int64_t* d_row_offsets, void* stream);
/* Receiver: place the kept tokens of every received row at their columns and
 * fill masked positions and every position of a lost row
 * (d_row_received[r] == 0) with zero_index. */
int tok_unpack_rows(const int32_t* d_payload, const int64_t* d_row_offsets,
                    const uint32_t* d_keep_bits, const uint8_t* d_row_received,
                    int64_t rows, int Wq, int32_t zero_index, int32_t* d_idx, void* stream);

/* Streaming (chunked causal encode/decode with per-stream conv caches on the
 * device; GoP-style segment coding, Sec. 4.2 and 4.3). Chunk 0 is one frame
 * (latent 0); every later chunk is s_T frames (frames s_T*k-3 .. s_T*k ->
 * latent k). Each causal conv keeps the last two input frames of the chunk
 * it saw, so a stream's chunks give exactly the whole-clip result.
 * tok_stream_bytes: device bytes one stream of H x W needs (for admission).
 * tok_stream_open allocates them (TOK_ENOMEM when they do not fit) and
 * tok_stream_reset starts a new video in them (chunk 0 again). A stream's
 * chunks must be encoded (decoded) in order, one at a time, but may be run
 * by any context with the same architecture and precision (serving lanes).
 * Streaming chunks have N = 1; encode takes 1 frame first, then s_T frames,
 * and returns one latent frame; decode takes one latent frame. The
 * concatenated outputs equal the whole-clip outputs bitwise. */
size_t tok_stream_bytes(const tok_ctx* ctx, int H, int W);
int tok_stream_open(tok_ctx* ctx, int H, int W, tok_stream** out);
void tok_stream_close(tok_stream* s);
int tok_stream_reset(tok_stream* s);

/* One causal 3D convolution (the K1 building block of f_phi / g_theta,
 * Sec. 2.4) on the selected precision path, without a context:
 *   y[n,to,ho,wo,co] = bias[co] + sum W[co,dt,dh,dw,ci] * x[n,ti,hi,wi,ci]
 *   ti = to*st + dt - (k-1) (frames before 0 read frame 0 under
 *   TOK_PAD_REPLICATE, zero under TOK_PAD_ZERO), hi = ho*sh + dh - (k-1)/2,
 *   wi = wo*sw + dw - (k-1)/2 (zero outside the frame).
 * d_x (N,T,H,W,Cin) and d_y (N,To,Ho,Wo,Cout), To = (T-1)/st+1,
 * Ho = (H-1)/sh+1 for k = 3 (H for k = 1), bf16 for TOK_BF16 / fp32 for
 * TOK_FP32; d_residual (same shape as d_y) is added when not NULL.
 * d_w (Cout,k,k,k,Cin) and d_bias (Cout) are fp32 device arrays; the BF16
 * path rounds the weights to bf16 into the workspace.
 * k is 1 or 3; strides are 1 or 2 with sh == sw; TOK_BF16 needs
 * Cin % 64 == 0 and even H, W when sh == 2 (TOK_ESHAPE otherwise).
 * d_workspace: at least tok_conv3d_workspace_bytes(...) bytes. */
size_t tok_conv3d_workspace_bytes(int precision, int Cin, int Cout, int k);
int tok_conv3d(int precision, const void* d_x, int N, int T, int H, int W, int Cin,
               const float* d_w, const float* d_bias, int Cout, int k, int st, int sh, int sw,
               int time_pad, const void* d_residual, void* d_y,
               void* d_workspace, size_t workspace_bytes, void* stream);

/* GroupNorm with statistics per (sample, group, frame) followed by SiLU
 * (the normalisation of every causal residual block):
 *   y = SiLU((x - mean) / sqrt(var + eps) * gamma + beta), mean/var over the
 *   C/G channels of a group and the H*W positions of one frame (biased var).
 * d_x, d_y (frames, HW, C) channels-last, bf16 (TOK_BF16) or fp32
 * (TOK_FP32), may alias. gamma/beta fp32 (C) or NULL (1/0). Needs C/G >= 2,
 * G <= 64, C a multiple of 8 (bf16) or 4 (fp32) with C/8 (C/4) a power of two
 * <= 256. d_workspace: tok_groupnorm_workspace_bytes(...) bytes. */
size_t tok_groupnorm_workspace_bytes(int precision, int64_t frames, int64_t HW, int C, int G);
int tok_groupnorm_silu(int precision, const void* d_x, int64_t frames, int64_t HW, int C, int G,
                       const float* d_gamma, const float* d_beta, float eps, void* d_y,
                       void* d_workspace, size_t workspace_bytes, void* stream);

/* Training: joint encoder/decoder optimisation through the masked decode
 * (Sec. 7, codec training; Appendix A.2, Eq. 7: tokens are dropped at random
 * and zero filled, and gradients reach the encoder through the decoder). The
 * paper's losses (L1 + optical flow + adversarial, Eq. 5-6) need networks and
 * data that are not available here; the objective is
 * L = mean((x_hat - x)^2). FSQ rounding is passed straight through:
 * d code_i / d z_i = h_i (1 - tanh^2(z_i + s_i)) / floor(L_i/2), and 0 at
 * dropped tokens. FULL architecture, H and W multiples of s_HW,
 * T = 1 mod s_T.
 *
 * Memory mode (tok_set_train_mode, before tok_reserve_train):
 *   TOK_TRAIN_RECOMPUTE (default): per residual block the forward keeps only
 *     the block's input (and the GroupNorm statistics, a few KB per norm);
 *     the backward rebuilds the block's interior, SiLU(GN1(x)), c1 of it
 *     and SiLU(GN2(.)), from them before it runs the block's backward.
 *   TOK_TRAIN_KEEP: the forward also keeps those three interior tensors and
 *     the backward recomputes nothing (more memory, e.g. about 2.3 GB more at
 *     2 x 3 x 17 x 256 x 256, and no recomputed convs).
 * Both modes give bitwise-equal gradients. tok_backward returns TOK_ESTATE
 * when the mode was changed after the forward it belongs to, and
 * tok_train_forward TOK_ENOMEM when the reserved workspace was sized for the
 * smaller mode.
 *
 * Parameters as one flat FP32 vector in the order of tok_param_info
 * (tok_param_total floats). tok_get_params copies the context's parameters
 * out, tok_set_params_device loads them from device memory (both enqueued on
 * `stream`). tok_params returns the device address of the context's own flat
 * vector (owned by the context, valid until tok_destroy): a caller may update
 * it in place (e.g. tok_sgd on it) and then call tok_repack, which rebuilds the
 * layouts the kernels read from it (the BF16 forward rows and, once a backward
 * has run, both adjoint layouts; every 3x3x3 conv's three layouts in one
 * launch); tok_set_params_device given that address skips the copy. tok_train_forward runs encode -> drop (Bernoulli(drop_rate),
 * Philox key seed, counter step) -> decode, writes x_hat (N,T,H,W,3) fp32, the
 * loss (one fp32 on the device) and dL/dx_hat (N,T,H,W,3) fp32, and keeps what
 * the backward needs; d_x must stay valid until tok_backward. A non-NULL
 * d_keep_bits (row masks in the layout tok_drop_mask writes) replaces the
 * random drop: tokens whose bit is 0 are dropped (e.g. a similarity-based
 * token selection, Sec. 4.3 Eq. 3, or lost packets). tok_backward
 * writes dL/dparams (flat FP32, every entry written) for the most recent
 * tok_train_forward, given dL/dx_hat. tok_sgd: params -= lr * grads. */
#define TOK_TRAIN_RECOMPUTE 0
#define TOK_TRAIN_KEEP 1
int tok_set_train_mode(tok_ctx* ctx, int mode);
int64_t tok_param_total(const tok_ctx* ctx);
int tok_get_params(tok_ctx* ctx, float* d_flat, void* stream);
int tok_set_params_device(tok_ctx* ctx, const float* d_flat, void* stream);
float* tok_params(tok_ctx* ctx);
int tok_repack(tok_ctx* ctx, void* stream);
size_t tok_train_workspace_bytes(const tok_ctx* ctx, int N, int T, int H, int W);
int tok_reserve_train(tok_ctx* ctx, int N, int T, int H, int W);
int tok_train_forward(tok_ctx* ctx, const void* d_x, int N, int T, int H, int W, float drop_rate,
                      uint64_t seed, uint64_t step, const uint32_t* d_keep_bits, float* d_xhat,
                      float* d_loss, float* d_dxhat, void* stream);
int tok_backward(tok_ctx* ctx, const float* d_dxhat, float* d_dparams, void* stream);
int tok_sgd(float* d_params, const float* d_grads, int64_t n, float lr, void* stream);

/* GroupNorm+SiLU without a workspace argument, for callers that cannot
 * allocate device memory (a host callback or real-time thread that may not
 * call cudaMalloc or take the allocator's locks, or an embedding with a fixed
 * memory budget). The paper has no counterpart; this is a library
 * convenience. Same computation and arguments as tok_groupnorm_silu, minus
 * the workspace: the scratch lives in one fixed array of
 * TOK_GN_NOALLOC_MAX_SCRATCH_BYTES in device global memory, held by every GPU
 * that loads the library until the process exits. Returns TOK_ENOMEM when
 * the problem needs more scratch than that (tok_groupnorm_workspace_bytes
 * tells how much it needs). Allocates nothing. The first call on a device
 * (and the first after cudaDeviceReset, or in another context) looks up the
 * array's device address, so make that first call before any stream
 * capture. TOK_EDEVICE when the current device cannot be queried. All calls
 * share the array: calls whose kernels overlap on the GPU (other streams,
 * other threads) race on it; serialise them. */
#define TOK_GN_NOALLOC_MAX_SCRATCH_BYTES (4u << 20)
int tok_groupnorm_silu_noalloc(int precision, const void* d_x, int64_t frames, int64_t HW, int C, int G,
                               const float* d_gamma, const float* d_beta, float eps, void* d_y,
                               void* stream);

/* Device status: synchronises the context's work, returns and clears the
 * first device-side error recorded since the last call. */
int tok_status(tok_ctx* ctx);
const char* tok_strerror(int code);

/* Guard bands (a check in place of a memory sanitizer): the context's
 * workspaces (inference arena, training workspace) and every stream's caches
 * are allocated with 4 KB of a fixed byte pattern before and after the bytes
 * the kernels use. tok_check_guards (the context's) and
 * tok_stream_check_guards (one stream's) synchronise the device and compare
 * the bands with the pattern: TOK_OK, or TOK_EGUARD if a kernel wrote outside
 * its workspace. tok_stream_bytes includes a stream's two bands. */
int tok_check_guards(tok_ctx* ctx);
int tok_stream_check_guards(tok_stream* s);

/* Debug/self-test: launch one kernel that waits on a device barrier nothing
 * ever signals, with a bounded wait of `limit_ns`; the kernel gives up,
 * records TOK_ETIMEOUT in the context's status word and returns. */
int tok_selftest_timeout(tok_ctx* ctx, int64_t limit_ns, void* stream);

/* Self-test of the guard bands: writes one byte of the reserved arena's
 * trailing band with cudaMemset (inside the allocation), checks that
 * tok_check_guards reports TOK_EGUARD, restores the band and checks that it
 * reports TOK_OK again. Returns TOK_OK when both checks behaved, TOK_ESTATE
 * when no arena is reserved, TOK_EGUARD otherwise. */
int tok_selftest_guards(tok_ctx* ctx);

/* Test hook: layer traces. While armed, every tok_encode / tok_decode (and
 * their batch forms, item 0) of this context copies, after the launch of the
 * named layer, that layer's tensors into the caller's device buffers with
 * device-to-device copies on the call's stream:
 *   conv layers ("enc.stem", "enc.l0.b0.c1", "enc.down0", "dec.up1", ...):
 *     d_in  <- its input activation (N,T,H,W,Cin) (for the BF16 path: the
 *              pixels for the stem where it forms its im2col rows on chip,
 *              the im2col matrix where the stem's frame needs edge extension,
 *              and the im2col matrix for the decoder input),
 *     d_res <- the residual it adds (same shape as the output), when it adds one,
 *     d_out <- its output: (N,T,H,W,Cout) bf16/fp32, after depth-to-space for
 *              the up convs and the pixel head, the latent z (fp32) for
 *              the last encoder conv;
 *   GroupNorm+SiLU layers ("enc.l0.b0.gn1", "dec.out_gn", ...):
 *     d_in <- its input, d_out <- its output;
 *   in tok_train_forward the same layers as above; in tok_backward
 *   "<conv>.wgrad" (d_in <- the conv's forward input, NULL for the stem and
 *     the decoder input, whose weight gradient runs on a rebuilt im2col
 *     matrix; d_res <- the gradient of its output as the weight gradient reads
 *     it: Cdy channels, the output channels padded to the adjoint's layout
 *     for narrow heads; before depth-to-space for the up convs and the pixel
 *     head) and "<conv>.dgrad" (d_in <- that output gradient as the adjoint
 *     conv reads it, zero-inserted onto the input grid for stride-2 convs;
 *     d_out <- the input gradient, its channels padded to the adjoint's
 *     rows).
 * A NULL buffer (or 0 bytes) skips that tensor. A buffer smaller than its
 * tensor makes the encode / decode return TOK_EINVAL. Several traces may be
 * armed at once; name == NULL disarms all. Returns TOK_EINVAL for an unknown
 * layer name. The buffers are the caller's and must stay valid while armed.
 * Not in the paper: it lets tests compare each layer of the full-size
 * network with the oracle on that layer's own input. */
int tok_trace_layer(tok_ctx* ctx, const char* name, void* d_in, size_t in_bytes, void* d_res, size_t res_bytes,
                    void* d_out, size_t out_bytes);

/* Number of kernels the library has launched since the context was created
 * (for launch accounting in benchmarks). */
int64_t tok_launch_count(const tok_ctx* ctx);

/* Opt-in timing of the context's kernels with CUDA events recorded on the
 * caller's stream around every launch, grouped by kernel class, with the
 * algorithmic work of each launch: convolutions count 2*M*N*K FLOPs
 * (M output voxels, N output channels, K = taps * input channels, padding
 * excluded); GroupNorm+SiLU counts one read and one write of the activation;
 * the gathers count their output bytes. tok_profile_enable allocates the
 * event pool (on = 1) or frees it (on = 0); tok_profile_read synchronises
 * the recorded events, fills `out` with the sums since the previous read and
 * resets them. */
typedef struct tok_profile_stats {
    int64_t conv_launches;
    double conv_ms;
    double conv_flop;
    int64_t gn_launches;
    double gn_ms;
    double gn_bytes;
    int64_t other_launches;
    double other_ms;
    double other_bytes;
} tok_profile_stats;
int tok_profile_enable(tok_ctx* ctx, int on);
int tok_profile_read(tok_ctx* ctx, tok_profile_stats* out);
/* The individual launches recorded since the last tok_profile_read, in launch
 * order (a trace): class (0 conv, 1 GroupNorm+SiLU, 2 other), device time,
 * algorithmic work as above, and the layer name (".dgrad" / ".wgrad" / ".bwd"
 * suffixes for the training backward) or a kernel label. Synchronises the
 * events; writes at most `cap` records; *count receives the number recorded.
 * Does not reset them (tok_profile_read does). */
typedef struct tok_profile_record {
    int cls;
    float ms;
    double work;
    char name[40];
} tok_profile_record;
int tok_profile_records(tok_ctx* ctx, tok_profile_record* out, int cap, int* count);

#ifdef __cplusplus
}
#endif
#endif /* MORPHE_TOK_H */
