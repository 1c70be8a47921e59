"""FP64 reference operations of the tokenizer hot path.

TEST INFRASTRUCTURE ONLY: the oracle. Only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product path never
does, and this package imports nothing from the product.

Every function is written from the definition it follows, cited beside it,
in float64, without blocking or fusion. Where the paper is silent the reading
used is stated in the docstring.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _conv_lib():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        lib.oracle_conv3d_fwd.argtypes = [dp, i, i, i, i, i, dp, dp, i, i, i, i, i, i, i, i, dp, i, i, i]
        lib.oracle_conv3d_dgrad.argtypes = [dp, i, i, i, i, i, dp, i, i, i, i, i, i, i, dp, i, i, i, i]
        lib.oracle_conv3d_wgrad.argtypes = [dp, i, i, i, i, i, dp, i, i, i, i, i, i, i, i, i, i, i, dp, dp]
        lib.oracle_num_threads.restype = i
        _lib = lib
    return _lib


def num_threads() -> int:
    """Number of OpenMP threads the oracle's convolution runs on."""
    return int(_conv_lib().oracle_num_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


PAD_REPLICATE = 0
PAD_ZERO = 1


def conv_out_shape(T, H, W, k, s):
    """Output extent of the causal conv: T_out = floor((T-1)/st) + 1 (causal
    left pad kt-1), H_out = floor((H + 2*((kh-1)//2) - kh)/sh) + 1."""
    kt, kh, kw = k
    st, sh, sw = s
    To = (T - 1) // st + 1
    Ho = (H + 2 * ((kh - 1) // 2) - kh) // sh + 1
    Wo = (W + 2 * ((kw - 1) // 2) - kw) // sw + 1
    return To, Ho, Wo


def conv3d(x, w, b, stride=(1, 1, 1), pad_mode=PAD_REPLICATE):
    """Causal 3D convolution (direct loops in C, FP64).

    x (N,T,H,W,Cin), w (Cout,kt,kh,kw,Cin), b (Cout,) or None.
    Follows the causal residual-block convolution of the tokenizer the paper
    builds on (Sec. 1, C2; encoder f_phi / decoder g_theta of Sec. 2.4):
    frames are padded only on the past side, so output frame t never reads a
    frame later than t*st.
    """
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N, T, H, W, Cin = x.shape
    Cout, kt, kh, kw, Cin2 = w.shape
    assert Cin == Cin2, (x.shape, w.shape)
    st, sh, sw = stride
    To, Ho, Wo = conv_out_shape(T, H, W, (kt, kh, kw), stride)
    y = np.empty((N, To, Ho, Wo, Cout), dtype=np.float64)
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    _conv_lib().oracle_conv3d_fwd(_p(x), N, T, H, W, Cin, _p(w), _p(bb) if bb is not None else None,
                                  Cout, kt, kh, kw, st, sh, sw, int(pad_mode), _p(y), To, Ho, Wo)
    return y


def conv3d_dgrad(dy, w, x_shape, stride=(1, 1, 1), pad_mode=PAD_REPLICATE):
    """Adjoint of :func:`conv3d` with respect to its input."""
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N, To, Ho, Wo, Cout = dy.shape
    _, kt, kh, kw, Cin = w.shape
    _, T, H, W, _ = x_shape
    dx = np.empty((N, T, H, W, Cin), dtype=np.float64)
    st, sh, sw = stride
    _conv_lib().oracle_conv3d_dgrad(_p(dy), N, To, Ho, Wo, Cout, _p(w), kt, kh, kw, st, sh, sw,
                                    int(pad_mode), _p(dx), T, H, W, Cin)
    return dx


def conv3d_wgrad(dy, x, k, stride=(1, 1, 1), pad_mode=PAD_REPLICATE):
    """Gradient of :func:`conv3d` with respect to its weights and bias."""
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, To, Ho, Wo, Cout = dy.shape
    _, T, H, W, Cin = x.shape
    kt, kh, kw = k
    dw = np.empty((Cout, kt, kh, kw, Cin), dtype=np.float64)
    db = np.empty((Cout,), dtype=np.float64)
    st, sh, sw = stride
    _conv_lib().oracle_conv3d_wgrad(_p(dy), N, To, Ho, Wo, Cout, _p(x), T, H, W, Cin,
                                    kt, kh, kw, st, sh, sw, int(pad_mode), _p(dw), _p(db))
    return dw, db


def _tap_frames(To, dt, st, kt, T, pad_mode):
    """Input frame read by every output frame at temporal tap dt (the causal rule of
    :func:`conv3d`): -1 where the tap reads zero padding."""
    ti = np.arange(To) * st + dt - (kt - 1)
    if pad_mode == PAD_REPLICATE:
        return np.where(ti < 0, 0, ti)
    return np.where(ti < 0, -1, ti)


def _tap_pos(O, d, s, k, extent):
    """Input row (column) read by every output row (column) at spatial tap d; -1 outside."""
    i = np.arange(O) * s + d - (k - 1) // 2
    return np.where((i < 0) | (i >= extent), -1, i)


def conv3d_wgrad_entries(dy, x, k, entries, stride=(1, 1, 1), pad_mode=PAD_REPLICATE):
    """Selected entries dW[co, dt, dh, dw, ci] of the weight gradient of :func:`conv3d`.

    Each entry is the sum over output voxels v of dy[v, co] * x[src(v, tap), ci],
    src being the forward's tap rule (causal frames, zero spatial padding); it
    lets a test check single entries of a gradient whose full computation would
    take too long (large clips). ``entries`` is a list of (co, dt, dh, dw, ci).
    Returns (values, magnitudes): the sums and the sums of |terms|."""
    kt, kh, kw = k
    st, sh, sw = stride
    N, To, Ho, Wo, _ = dy.shape
    _, T, H, W, _ = x.shape
    vals, mags = [], []
    for co, dt, dh, dw, ci in entries:
        ti = _tap_frames(To, dt, st, kt, T, pad_mode)
        hi = _tap_pos(Ho, dh, sh, kh, H)
        wi = _tap_pos(Wo, dw, sw, kw, W)
        xc = np.asarray(x[..., ci], dtype=np.float64)
        g = xc[:, np.maximum(ti, 0)][:, :, np.maximum(hi, 0)][:, :, :, np.maximum(wi, 0)]
        valid = (ti >= 0)[:, None, None] & (hi >= 0)[None, :, None] & (wi >= 0)[None, None, :]
        terms = np.asarray(dy[..., co], dtype=np.float64) * np.where(valid[None], g, 0.0)
        vals.append(terms.sum())
        mags.append(np.abs(terms).sum())
    return np.array(vals), np.array(mags)


def conv3d_dgrad_entries(dy, w, x_shape, points, stride=(1, 1, 1), pad_mode=PAD_REPLICATE):
    """dX[n, t, h, w, :] of :func:`conv3d` at the given points (n, t, h, w): the sum, over
    taps and the output voxels whose tap reads (t, h, w) under the forward's rule
    (with replicate padding, frame 0 is read by every tap that falls before it),
    of w[:, tap, :]^T dy[output voxel, :]. Returns (values (P, Cin), magnitudes
    (P, Cin): the sums of |terms|)."""
    Cout, kt, kh, kw, Cin = w.shape
    st, sh, sw = stride
    N, To, Ho, Wo, _ = dy.shape
    _, T, H, W, _ = x_shape
    w = np.asarray(w, dtype=np.float64)
    vals = np.zeros((len(points), Cin))
    mags = np.zeros((len(points), Cin))
    for p, (n, t, h, wv) in enumerate(points):
        for dt in range(kt):
            ots = np.nonzero(_tap_frames(To, dt, st, kt, T, pad_mode) == t)[0]
            for dh in range(kh):
                ohs = np.nonzero(_tap_pos(Ho, dh, sh, kh, H) == h)[0]
                for dw in range(kw):
                    ows = np.nonzero(_tap_pos(Wo, dw, sw, kw, W) == wv)[0]
                    for ot in ots:
                        for oh in ohs:
                            for ow in ows:
                                g = np.asarray(dy[n, ot, oh, ow], dtype=np.float64)
                                term = g[:, None] * w[:, dt, dh, dw, :]
                                vals[p] += term.sum(axis=0)
                                mags[p] += np.abs(term).sum(axis=0)
    return vals, mags


# --------------------------------------------------------------------------
# GroupNorm + SiLU
# --------------------------------------------------------------------------

def gn_groups(C: int, groups: int = 32) -> int:
    """Number of GroupNorm groups used for C channels: min(groups, C // 2).

    Reading: the architecture asks for GroupNorm(32); for narrow layers
    (C < 64) that would leave fewer than 2 channels per group, so the group
    count is capped at C/2."""
    return max(1, min(groups, C // 2))


def group_norm_frames(x, groups, eps=1e-6, gamma=None, beta=None):
    """GroupNorm with statistics per (sample, group, frame).

    Reading: the tokenizer is causal (Sec. 1, C2; streaming per GoP, Sec. 4.2),
    so a normalisation may not mix frames; statistics are taken over the
    group's channels and the frame's H x W positions only. Two-pass:
    mean, then the mean of squared deviations (biased variance).
    """
    x = np.asarray(x, dtype=np.float64)
    N, T, H, W, C = x.shape
    cg = C // groups
    xg = x.reshape(N, T, H * W, groups, cg)
    mean = xg.mean(axis=(2, 4), keepdims=True)
    var = ((xg - mean) ** 2).mean(axis=(2, 4), keepdims=True)
    y = ((xg - mean) / np.sqrt(var + eps)).reshape(N, T, H, W, C)
    if gamma is not None:
        y = y * np.asarray(gamma, dtype=np.float64)
    if beta is not None:
        y = y + np.asarray(beta, dtype=np.float64)
    return y


def silu(x):
    """SiLU(x) = x * sigmoid(x) = x / (1 + exp(-x))."""
    x = np.asarray(x, dtype=np.float64)
    return x / (1.0 + np.exp(-x))


# --------------------------------------------------------------------------
# Finite scalar quantisation (FSQ)
# --------------------------------------------------------------------------

FSQ_EPS = 1e-3


def fsq_constants(levels):
    """Per-channel FSQ constants, from the FSQ method (Mentzer et al., 2023):
    half-range h = (L-1)(1-eps)/2, offset o = 0.5 for even L else 0,
    shift s = atanh(o/h) (so that z = 0 maps to the code 0),
    half-width floor(L/2), and the mixed-radix basis B_i = prod_{j<i} L_j
    (channel 0 least significant)."""
    L = np.asarray(levels, dtype=np.float64)
    h = (L - 1.0) * (1.0 - FSQ_EPS) / 2.0
    o = np.where(np.asarray(levels) % 2 == 0, 0.5, 0.0)
    s = np.arctanh(o / h)
    hw = np.asarray(levels, dtype=np.int64) // 2
    basis = np.concatenate([[1], np.cumprod(np.asarray(levels, dtype=np.int64))[:-1]])
    return h, o, s, hw, basis


def fsq_bound(z, levels):
    """b_i = tanh(z_i + s_i) * h_i - o_i (FP64)."""
    h, o, s, _, _ = fsq_constants(levels)
    z = np.asarray(z, dtype=np.float64)
    return np.tanh(z + s) * h - o


def fsq_quantize(z, levels):
    """Quantise latent vectors z (..., len(levels)) to integer token indices.

    The token matrix the paper transmits (Sec. 4.3, Sec. 6.2) holds one index
    per latent position. Steps: bound, round half to even, digit
    d_i = q_i + floor(L_i/2) in [0, L_i), index = sum_i d_i * B_i,
    code_i = q_i / floor(L_i/2) in [-1, 1].
    Returns (idx int64, codes float64, bound float64).
    """
    _, _, _, hw, basis = fsq_constants(levels)
    b = fsq_bound(z, levels)
    q = np.rint(b)  # numpy rint rounds half to even
    d = (q + hw).astype(np.int64)
    idx = (d * basis).sum(axis=-1)
    codes = q / hw
    return idx, codes, b


def fsq_index_to_digits(idx, levels):
    """Mixed-radix decomposition of token indices into per-channel digits."""
    idx = np.asarray(idx, dtype=np.int64)
    L = np.asarray(levels, dtype=np.int64)
    _, _, _, _, basis = fsq_constants(levels)
    return (idx[..., None] // basis) % L


def fsq_dequantize(idx, levels):
    """Token indices back to code vectors: code_i = (d_i - floor(L_i/2)) / floor(L_i/2)."""
    _, _, _, hw, _ = fsq_constants(levels)
    d = fsq_index_to_digits(idx, levels)
    return (d - hw) / hw


def fsq_zero_index(levels) -> int:
    """Index of the all-zero code vector (digit floor(L_i/2) on every channel).

    The receiver fills dropped tokens and lost rows with zeros (Sec. 6.2;
    Appendix A.2); a zero code vector is this index."""
    _, _, _, hw, basis = fsq_constants(levels)
    return int((hw * basis).sum())


# --------------------------------------------------------------------------
# Counter-based random numbers and packet-drop token masking
# --------------------------------------------------------------------------

_M = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).

    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (32x32 -> 64-bit
    products), new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key
    is bumped by the Weyl constants (W0, W1) between rounds. Inputs are
    arrays (or scalars) of values < 2^32; returns four uint64 arrays of
    32-bit words."""
    c = [np.asarray(v, dtype=np.uint64) & _M for v in (c0, c1, c2, c3)]
    k = [np.asarray(v, dtype=np.uint64) & _M for v in (k0, k1)]
    for r in range(10):
        if r > 0:
            k = [(k[0] + PHILOX_W0) & _M, (k[1] + PHILOX_W1) & _M]
        p0 = PHILOX_M0 * c[0]
        p1 = PHILOX_M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M
        c = [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]
    return c


def drop_threshold(rate) -> int:
    """Integer threshold for a drop probability: floor(rate * 2^32) computed
    from the float32 rate (exact in float64), clipped to [0, 2^32]."""
    r = float(np.float32(rate))
    r = min(max(r, 0.0), 1.0)
    return int(np.floor(r * 4294967296.0))


def drop_mask(N, Tq, Hq, Wq, rate, seed, stream_id, chunk_id):
    """Per-token Bernoulli(rate) drop decisions (True = dropped).

    Models proactive token dropping / random token drop (Sec. 4.3;
    Appendix A.2 trains with drop rates U[0, 25%]). Counter-based so that the
    decision for a token depends only on (seed, stream, chunk, sample, token):
    token j = (t*Hq + h)*Wq + w of sample n uses Philox counter
    (j >> 2, n, chunk_id mod 2^32, stream_id mod 2^32), key
    (seed mod 2^32, seed >> 32), output word j & 3; it is dropped iff that
    word < floor(rate * 2^32)."""
    thr = drop_threshold(rate)
    ntok = Tq * Hq * Wq
    j = np.arange(ntok, dtype=np.uint64)
    out = np.zeros((N, ntok), dtype=bool)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    for n in range(N):
        words = philox4x32_10(j >> np.uint64(2), n, int(chunk_id) & 0xFFFFFFFF,
                              int(stream_id) & 0xFFFFFFFF, seed & 0xFFFFFFFF, seed >> 32)
        w = np.stack(words, axis=-1)  # (ntok, 4)
        r = w[np.arange(ntok), (j & np.uint64(3)).astype(np.int64)]
        out[n] = r < np.uint64(thr) if thr < (1 << 32) else np.ones(ntok, dtype=bool)
    return out.reshape(N, Tq, Hq, Wq)


def apply_drop(idx, dropped, levels):
    """Dropped tokens take the zero-code index (zero fill, Sec. 6.2)."""
    out = np.array(idx, dtype=np.int64, copy=True)
    out[dropped] = fsq_zero_index(levels)
    return out


# --------------------------------------------------------------------------
# Similarity-based token selection (Sec. 6.3, Eq. 3)
# --------------------------------------------------------------------------

def token_similarity(idx_p, idx_i, levels):
    """Per-position cosine similarity between P-frame and I-frame tokens (Eq. 3).

    S = <p, q> / (|p| |q|) for the code vectors p, q of the two indices at the
    same (sample, h, w); the I tokens (N, 1, H', W') are compared with every
    P latent frame. Reading: S = 0 where either code vector is zero (a zero
    vector has no direction; this is also the convention of a cosine with the
    norm product clamped from below). The selection is decided on these
    values, so they are computed in float32: dot product and both squared
    norms summed over channels in order, and the product of the squared norms
    (all exact: codes are multiples of 1/floor(L/2)), then one correctly
    rounded square root of that product and one correctly rounded division
    (so parallel codes give exactly +-1); -0 is returned as +0. The kernel
    computes the same float32 operations."""
    cp = fsq_dequantize(idx_p, levels).astype(np.float32)
    ci = fsq_dequantize(idx_i, levels).astype(np.float32)
    ci = np.broadcast_to(ci, cp.shape)
    dot = np.zeros(cp.shape[:-1], dtype=np.float32)
    sp = np.zeros_like(dot)
    si = np.zeros_like(dot)
    for c in range(cp.shape[-1]):
        dot = dot + cp[..., c] * ci[..., c]
        sp = sp + cp[..., c] * cp[..., c]
        si = si + ci[..., c] * ci[..., c]
    den = np.sqrt(sp * si)
    with np.errstate(divide="ignore", invalid="ignore"):
        S = np.where(den > 0, dot / np.where(den > 0, den, np.float32(1)), np.float32(0)).astype(np.float32)
    return S + np.float32(0.0)


def similarity_drop(idx_p, idx_i, levels, rate):
    """Drop decisions (True = dropped) of the similarity-based selection.

    Per sample and P latent frame of H' x W' tokens, the tokens with S > tau
    are dropped, tau chosen for the available bandwidth (Sec. 6.3). Reading:
    tau is the (1 - rate)-quantile of S over the frame, i.e. exactly
    k = floor(rate * H'W') tokens are dropped, those with the largest S, and
    among equal S the lower linear index (h * W' + w) goes first. rate is the
    float32 value, k computed in float64 and clipped to [0, H'W']."""
    S = token_similarity(idx_p, idx_i, levels)
    N, Tp, Hq, Wq = S.shape
    n = Hq * Wq
    k = int(np.floor(float(np.float32(rate)) * n))
    k = min(max(k, 0), n)
    out = np.zeros((N, Tp, n), dtype=bool)
    order_idx = np.arange(n)
    for b in range(N):
        for t in range(Tp):
            s = S[b, t].reshape(-1)
            order = np.lexsort((order_idx, -s))  # S descending, then index ascending
            out[b, t, order[:k]] = True
    return out.reshape(N, Tp, Hq, Wq)


# --------------------------------------------------------------------------
# Pixel residuals (Sec. 6.3, Eq. 4)
# --------------------------------------------------------------------------

def residual_windows(T, window):
    """Frame windows of a clip: [0, w), [w, 2w), ...; the last may be shorter."""
    return [(a, min(a + window, T)) for a in range(0, T, window)]


def residual_mean(x, xhat, window, theta):
    """Window-averaged, thresholded pixel residual (Sec. 6.3; Eq. 4).

    r = x - x_hat per pixel and channel, averaged over each window of
    consecutive frames: r_c(h,w,c) = (1/T) sum_t r(h,w,c,t), T the window's
    frame count; then elements with |r_c| < theta are zeroed. The zeroing is a
    decision on these values, so they are computed in float32 in the order of
    the definition: each difference rounded, summed over t in order, one
    division by T. x, x_hat: (N, T, H, W, C); returns (N, n_windows, H, W, C)."""
    x = np.asarray(x, dtype=np.float32)
    xh = np.asarray(xhat, dtype=np.float32)
    N, T = x.shape[:2]
    wins = residual_windows(T, window)
    out = np.zeros((N, len(wins)) + x.shape[2:], dtype=np.float32)
    th = np.float32(theta)
    for k, (a, b) in enumerate(wins):
        s = np.zeros((N,) + x.shape[2:], dtype=np.float32)
        for t in range(a, b):
            s = s + (x[:, t] - xh[:, t])
        r = s / np.float32(b - a)
        out[:, k] = np.where(np.abs(r) < th, np.float32(0), r)
    return out


def residual_sparse(r):
    """Sparse form of a thresholded residual: per (sample, window) segment, the
    nonzero elements in position order, position = (h*W + w)*C + c.
    Returns (positions int32, values float32, segment offsets int64 of length
    N*n_windows + 1)."""
    N, K = r.shape[:2]
    flat = r.reshape(N * K, -1)
    pos, val, offs = [], [], [0]
    for seg in flat:
        nz = np.nonzero(seg)[0]
        pos.append(nz.astype(np.int32))
        val.append(seg[nz])
        offs.append(offs[-1] + len(nz))
    return np.concatenate(pos), np.concatenate(val).astype(np.float32), np.asarray(offs, dtype=np.int64)


def residual_apply(xhat, pos, val, offs, window):
    """Receiver side (Sec. 6.3): every frame of a window gets that window's
    residual added (float32): x_hat[n, t] += r_c[n, window(t)]."""
    xh = np.array(xhat, dtype=np.float32, copy=True)
    N, T = xh.shape[:2]
    wins = residual_windows(T, window)
    flat = xh.reshape(N, T, -1)
    for n in range(N):
        for k, (a, b) in enumerate(wins):
            seg = n * len(wins) + k
            p = pos[offs[seg]:offs[seg + 1]]
            v = val[offs[seg]:offs[seg + 1]]
            for t in range(a, b):
                flat[n, t, p] = flat[n, t, p] + v
    return flat.reshape(xh.shape)


# --------------------------------------------------------------------------
# GoP boundary smoothing (Sec. 6.1, Eq. 1 and 2)
# --------------------------------------------------------------------------

def gop_blend(xhat_prev, xhat_curr, n):
    """Boundary blending (Eq. 2): for i = 1..n, frame i of the current GoP
    becomes a_i * prev[T-n+i] + (1 - a_i) * curr[i] with a_i = (n - i) / n
    (1-based frame numbers; T the previous GoP's frame count); the other
    frames are unchanged. Arrays (N, T, H, W, C), float64."""
    prev = np.asarray(xhat_prev, dtype=np.float64)
    out = np.array(xhat_curr, dtype=np.float64, copy=True)
    T = prev.shape[1]
    for i in range(1, n + 1):
        a = (n - i) / n
        out[:, i - 1] = a * prev[:, T - n + i - 1] + (1 - a) * out[:, i - 1]
    return out


def temporal_loss(xhat_curr, x_prev, n):
    """Boundary loss (Eq. 1): L = (1/n) sum_{i=1..n} || xhat_curr[i] - x_prev[T-n+i] ||,
    averaged over the batch. Reading (the norm is not specified): the
    Euclidean norm of the whole frame difference (all pixels and channels).
    Returns (L, dL/dxhat_curr) with the gradient (1/(N n)) d / ||d|| on the
    first n frames (0 where ||d|| = 0) and 0 elsewhere; float64."""
    xc = np.asarray(xhat_curr, dtype=np.float64)
    xp = np.asarray(x_prev, dtype=np.float64)
    N, T = xp.shape[:2]
    L = 0.0
    g = np.zeros_like(xc)
    for i in range(1, n + 1):
        d = xc[:, i - 1] - xp[:, T - n + i - 1]
        nrm = np.sqrt((d.reshape(N, -1) ** 2).sum(axis=1))
        L += nrm.sum() / (N * n)
        scale = np.where(nrm > 0, 1.0 / (N * n * np.where(nrm > 0, nrm, 1.0)), 0.0)
        g[:, i - 1] = d * scale.reshape((N,) + (1,) * (d.ndim - 1))
    return L, g


# --------------------------------------------------------------------------
# Resolution Scaling Accelerator: pre-encode downsampling (Sec. 5)
# --------------------------------------------------------------------------

def round_to_bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32 values.

    bfloat16 keeps the upper 16 bits of the IEEE binary32 pattern; rounding
    adds 0x7FFF plus the lowest kept bit to the pattern before truncation, so
    that a dropped half-way remainder goes to the even neighbour. NaNs stay
    NaN (quietened)."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_lsb) >> 16) << 16
    nan = np.isnan(f)
    r = np.where(nan, (u | 0x00400000) >> 16 << 16, r)
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).reshape(f.shape)


def box_downsample(x, s, out_bf16=False):
    """Downsampling by an integer factor s (the resolution control of Sec. 5,
    2x or 3x of 1080p in the paper's training and evaluation).

    Reading (the paper says the frames are "linearly" downsampled and gives no
    filter): every output pixel is the mean of the s x s block of input pixels
    it covers, blocks anchored at the top-left corner, output size floor(H/s)
    x floor(W/s) (trailing rows and columns dropped) -- the area filter, which
    for s = 2 coincides with bilinear sampling at the block centres.

    x: (F, H, W, C) frames, channels last, either uint8 (0..255) or float32
    values. The mean is computed in float32 in a fixed order, since the
    result is quantised to its output type: for float input, the s*s values
    summed row by row, left to right, each addition rounded, then one division
    by s*s; for uint8 input, the exact integer sum, one division by s*s, then
    the map to [-1, 1] as m / 127.5 - 1 (each step rounded to float32).
    out_bf16 rounds the float32 result to bfloat16 (ties to even).
    Returns float32 (F, H//s, W//s, C)."""
    x = np.asarray(x)
    F, H, W, C = x.shape
    Ho, Wo = H // s, W // s
    out = np.zeros((F, Ho, Wo, C), dtype=np.float32)
    ss = np.float32(s * s)
    if x.dtype == np.uint8:
        acc = np.zeros((F, Ho, Wo, C), dtype=np.int64)
        for i in range(s):
            for j in range(s):
                acc += x[:, i:Ho * s:s, j:Wo * s:s, :].astype(np.int64)
        m = acc.astype(np.float32) / ss
        out = m / np.float32(127.5) - np.float32(1.0)
    else:
        xf = x.astype(np.float32)
        acc = np.zeros((F, Ho, Wo, C), dtype=np.float32)
        for i in range(s):
            for j in range(s):
                acc = acc + xf[:, i:Ho * s:s, j:Wo * s:s, :]
        out = acc / ss
    out = out.astype(np.float32)
    return round_to_bf16(out) if out_bf16 else out


def keep_bits_from_mask(dropped):
    """Row masks of the packet header (Sec. 6.2): for every token row, a
    W-bit vector with bit w set when token w is kept, stored as
    ceil(W/32) little-endian 32-bit words per row."""
    dropped = np.asarray(dropped, dtype=bool)
    *lead, Wq = dropped.shape
    nw = (Wq + 31) // 32
    keep = ~dropped.reshape(-1, Wq)
    bits = np.zeros((keep.shape[0], nw), dtype=np.uint64)
    for w in range(Wq):
        bits[:, w // 32] |= keep[:, w].astype(np.uint64) << np.uint64(w % 32)
    return bits.astype(np.uint32).reshape(*lead, nw)


def pack_rows(idx, keep_bits, Wq):
    """Sender side of the row packetisation (Sec. 6.2): each token row
    becomes a packet whose payload is the kept tokens in column order.
    Returns (payload int32, row_offsets int64 of length rows+1)."""
    idx = np.asarray(idx).reshape(-1, Wq)
    kb = np.asarray(keep_bits).reshape(idx.shape[0], -1)
    payload, offs = [], [0]
    for r in range(idx.shape[0]):
        for w in range(Wq):
            if (int(kb[r, w // 32]) >> (w % 32)) & 1:
                payload.append(int(idx[r, w]))
        offs.append(len(payload))
    return np.asarray(payload, dtype=np.int32), np.asarray(offs, dtype=np.int64)


def unpack_rows(payload, row_offsets, keep_bits, row_received, Wq, zero_index):
    """Receiver side (Sec. 6.2): place kept tokens at their columns, fill
    masked positions with zeros (the zero-code index), and fill every
    token of a lost row (row_received == 0) with zeros."""
    kb = np.asarray(keep_bits).reshape(len(row_received), -1)
    out = np.full((len(row_received), Wq), zero_index, dtype=np.int64)
    for r in range(len(row_received)):
        if not row_received[r]:
            continue
        k = int(row_offsets[r])
        for w in range(Wq):
            if (int(kb[r, w // 32]) >> (w % 32)) & 1:
                out[r, w] = payload[k]
                k += 1
    return out


# --------------------------------------------------------------------------
# Depth-to-space and padding
# --------------------------------------------------------------------------

def depth_to_space(y, r, drop_first=None):
    """Rearrange channels into (time, height, width) sub-positions.

    y (N,T,H,W,C'*rt*rh*rw) -> (N, T*rt, H*rh, W*rw, C') with channel
    ((a*rh + b)*rw + c)*C' + ch going to (t*rt + a, h*rh + b, w*rw + c, ch);
    then the first ``drop_first`` frames (default rt - 1) are removed so that
    the causal decoder emits 1 + rt*(T-1) frames, mirroring the encoder's
    causal downsampling (Sec. 2.4: x_{0:T} <-> z_{0:T'})."""
    rt, rh, rw = r
    y = np.asarray(y)
    N, T, H, W, C = y.shape
    Co = C // (rt * rh * rw)
    o = y.reshape(N, T, H, W, rt, rh, rw, Co).transpose(0, 1, 4, 2, 5, 3, 6, 7)
    o = o.reshape(N, T * rt, H * rh, W * rw, Co)
    d = rt - 1 if drop_first is None else drop_first
    return o[:, d:]


def space_to_depth(x, r, pad_first=None):
    """Inverse of :func:`depth_to_space` (used only to pin it)."""
    rt, rh, rw = r
    x = np.asarray(x)
    d = rt - 1 if pad_first is None else pad_first
    N, T, H, W, Co = x.shape
    if d:
        x = np.concatenate([np.zeros((N, d, H, W, Co), x.dtype), x], axis=1)
        T += d
    o = x.reshape(N, T // rt, rt, H // rh, rh, W // rw, rw, Co).transpose(0, 1, 3, 5, 2, 4, 6, 7)
    return o.reshape(N, T // rt, H // rh, W // rw, rt * rh * rw * Co)


def edge_pad_to_multiple(x, m=8):
    """Pad H and W up to multiples of m by repeating the last row/column.

    Reading: the 8x spatial compression needs H and W divisible by 8
    (e.g. 854-wide 480p); the frame is edge-extended and the decoder output
    is cropped back."""
    x = np.asarray(x)
    N, T, H, W, C = x.shape
    Hp = -(-H // m) * m
    Wp = -(-W // m) * m
    if Hp == H and Wp == W:
        return x
    return np.pad(x, ((0, 0), (0, 0), (0, Hp - H), (0, Wp - W), (0, 0)), mode="edge")
