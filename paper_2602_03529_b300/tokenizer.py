"""Torch-tensor front end of the tokenizer library (thin marshalling layer).

PyTorch provides device memory and streams; every step of encode/decode runs
in the CUDA library through the C-ABI (see ``_lib``). Tensors must be CUDA,
contiguous, channels-last: clips (N, T, H, W, 3), latents (N, T', H', W', C),
token indices (N, T', H', W') int32.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

PRECISIONS = {"bf16": L.TOK_BF16, "fp32": L.TOK_FP32}


def make_arch(kind="full", ch=(128, 256, 512), blocks=2, levels=(8, 8, 8, 5, 5, 5), gn_groups=32,
              gn_eps=1e-6, time_pad="replicate", t_stem=1) -> L.tok_arch:
    """Architecture descriptor; ``t_stem`` = 2 gives the 8x temporal / 8x8 spatial setting
    (Sec. 4.1) with three levels, 1 the 4x / 8x8 one."""
    a = L.tok_arch_default()
    a.kind = L.TOK_ARCH_FULL if kind == "full" else L.TOK_ARCH_STAGE
    a.nlevels = len(ch)
    for i in range(4):
        a.ch[i] = ch[i] if i < len(ch) else 0
    a.blocks = blocks
    a.nlev = len(levels)
    for i in range(8):
        a.levels[i] = levels[i] if i < len(levels) else 0
    a.gn_groups = gn_groups
    a.gn_eps = gn_eps
    a.time_pad = L.TOK_PAD_REPLICATE if time_pad == "replicate" else L.TOK_PAD_ZERO
    a.t_stem = t_stem
    return a


def arch_kwargs(a: L.tok_arch) -> dict:
    """The make_arch keywords of a descriptor."""
    n = 2 if a.kind == L.TOK_ARCH_STAGE else a.nlevels
    return dict(kind="stage" if a.kind == L.TOK_ARCH_STAGE else "full", ch=tuple(a.ch[:n]), blocks=a.blocks,
                levels=tuple(a.levels[:a.nlev]), gn_groups=a.gn_groups, gn_eps=a.gn_eps,
                time_pad="replicate" if a.time_pad == L.TOK_PAD_REPLICATE else "zero", t_stem=a.t_stem)


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class Tokenizer:
    """One tokenizer context (weights resident on the device)."""

    def __init__(self, precision: str = "bf16", **arch):
        self.precision = precision
        self.arch_kw = arch
        self.arch = make_arch(**arch)
        self.levels = tuple(arch.get("levels", (8, 8, 8, 5, 5, 5)))
        self.ctx = L.tok_create(self.arch, PRECISIONS[precision])
        self.dtype = torch.bfloat16 if precision == "bf16" else torch.float32

    @classmethod
    def from_file(cls, path: str, precision: str = "bf16"):
        """A context whose descriptor and weights come from a file written by save()."""
        arch, _ = L.tok_read_weights_header(path)
        self = cls.__new__(cls)
        self.precision = precision
        self.arch = arch
        self.arch_kw = arch_kwargs(arch)
        self.levels = tuple(arch.levels[:arch.nlev])
        self.ctx = L.tok_create_from_file(path, PRECISIONS[precision])
        self.dtype = torch.bfloat16 if precision == "bf16" else torch.float32
        return self

    def save(self, path: str):
        """Write the descriptor and the flat FP32 parameters (synchronous)."""
        L.tok_save_params(self.ctx, path)

    # -- parameters -------------------------------------------------------
    def param_list(self):
        """[(name, shape)] in the architecture's order."""
        return [L.tok_param_info(self.ctx, i) for i in range(L.tok_param_count(self.ctx))]

    def param_spec(self):
        """[(name, shape, kind)] with kind conv / bias / gn_gamma / gn_beta."""
        out = []
        for name, shape in self.param_list():
            if len(shape) == 5:
                kind = "conv"
            elif name.endswith(".g"):
                kind = "gn_gamma"
            elif ".gn" in name or name.endswith("_gn.b"):
                kind = "gn_beta"
            else:
                kind = "bias"
            out.append((name, shape, kind))
        return out

    def set_params(self, params: dict):
        for name, shape in self.param_list():
            a = np.ascontiguousarray(params[name], dtype=np.float32)
            if tuple(a.shape) != tuple(shape):
                raise ValueError(f"{name}: shape {a.shape} != {shape}")
            L.tok_set_param(self.ctx, name, a.ctypes.data_as(C.c_void_p).value, a.size)

    # -- shapes / workspace ----------------------------------------------
    def latent_shape(self, T, H, W):
        return L.tok_latent_shape(self.ctx, T, H, W)

    def reserve(self, N, T, H, W):
        L.tok_reserve(self.ctx, N, T, H, W)

    def workspace_bytes(self, N, T, H, W):
        return L.tok_workspace_bytes(self.ctx, N, T, H, W)

    # -- encode / decode --------------------------------------------------
    def encode(self, x: torch.Tensor, z: torch.Tensor | None = None, idx: torch.Tensor | None = None,
               stream=None, want_z=True, video=None):
        """Encode a clip, or (``video`` = a handle from stream_open) the next chunk of a video:
        1 frame for its first chunk, s_T frames after that, giving one latent frame."""
        N, T, H, W, c = x.shape
        if x.dtype != self.dtype:
            raise ValueError(f"x must be {self.dtype}")
        if video is not None:
            Tq, Hq, Wq = (1,) + self.latent_shape(1, H, W)[1:]
        else:
            Tq, Hq, Wq = self.latent_shape(T, H, W)
        if z is None and want_z:
            z = torch.empty((N, Tq, Hq, Wq, len(self.levels)), device=x.device, dtype=torch.float32)
        if idx is None:
            idx = torch.empty((N, Tq, Hq, Wq), device=x.device, dtype=torch.int32)
        L.tok_encode(self.ctx, _ptr(x), N, T, H, W, _ptr(z), _ptr(idx), video, _stream_ptr(stream))
        return z, idx

    def decode(self, idx: torch.Tensor, H: int, W: int, out: torch.Tensor | None = None, stream=None,
               video=None, first_chunk=None):
        """Decode token indices; with ``video`` one latent frame of a stream (``first_chunk``
        tells whether it is the stream's first, which yields 1 frame instead of s_T)."""
        N, Tq, Hq, Wq = idx.shape
        if video is not None:
            T = 1 if first_chunk else self.s_t
        else:
            T = 1 + (Tq - 1) * self.s_t
        if out is None:
            out = torch.empty((N, T, H, W, 3), device=idx.device, dtype=torch.float32)
        L.tok_decode(self.ctx, _ptr(idx), N, Tq, Hq, Wq, H, W, _ptr(out), video, _stream_ptr(stream))
        return out

    def decode_gop(self, idx: torch.Tensor, H: int, W: int, prev: torch.Tensor, n: int,
                   out: torch.Tensor | None = None, stream=None):
        """Decode a GoP's tokens (a whole clip) with its first n frames blended with the
        last n frames of the previous GoP's reconstruction `prev` (N, T_prev, H, W, 3)
        fp32 (Eq. 2, fused into the pixel head)."""
        N, Tq, Hq, Wq = idx.shape
        T = 1 + (Tq - 1) * self.s_t
        if out is None:
            out = torch.empty((N, T, H, W, 3), device=idx.device, dtype=torch.float32)
        L.tok_decode_gop(self.ctx, _ptr(idx), N, Tq, Hq, Wq, H, W, _ptr(prev), prev.shape[1], n, _ptr(out),
                         _stream_ptr(stream))
        return out

    def set_cta_tiles(self, tiles: int):
        """0: persistent conv CTAs; n > 0: at most n tiles per CTA (yields SMs quickly to
        work on higher-priority CUDA streams; results are unchanged)."""
        L.tok_set_cta_tiles(self.ctx, tiles)

    def trace_layer(self, name, inp=None, res=None, out=None):
        """Arm a layer trace (a test hook): the next encodes / decodes copy the named
        layer's input, residual and output into the given device tensors (None skips
        one). trace_layer(None) disarms all traces."""
        def pb(t):
            return (None, 0) if t is None else (t.data_ptr(), t.numel() * t.element_size())
        if name is None:
            L.tok_trace_layer(self.ctx, None, None, 0, None, 0, None, 0)
            return
        L.tok_trace_layer(self.ctx, name, *pb(inp), *pb(res), *pb(out))

    # -- grouped (one launch per layer over several inputs) --------------------
    def reserve_batch(self, shapes):
        """shapes: list of (N, T, H, W); a stream chunk counts as (1, s_T, H, W)."""
        L.tok_reserve_batch(self.ctx, list(shapes))

    def batch_workspace_bytes(self, shapes) -> int:
        return L.tok_batch_workspace_bytes(self.ctx, list(shapes))

    def encode_batch(self, xs, videos=None, stream=None, want_z=True):
        """Encode several clips (or stream chunks, ``videos[i]`` a handle or None) of
        any sizes in one grouped pass; returns lists of z (or None) and idx."""
        videos = videos or [None] * len(xs)
        zs, idxs, items = [], [], []
        for x, v in zip(xs, videos):
            N, T, H, W, _ = x.shape
            if x.dtype != self.dtype:
                raise ValueError(f"x must be {self.dtype}")
            Tq, Hq, Wq = (1,) + self.latent_shape(1, H, W)[1:] if v is not None else self.latent_shape(T, H, W)
            z = torch.empty((N, Tq, Hq, Wq, len(self.levels)), device=x.device, dtype=torch.float32) \
                if want_z else None
            idx = torch.empty((N, Tq, Hq, Wq), device=x.device, dtype=torch.int32)
            zs.append(z)
            idxs.append(idx)
            items.append((_ptr(x), N, T, H, W, _ptr(z), _ptr(idx), v))
        L.tok_encode_batch(self.ctx, items, _stream_ptr(stream))
        return zs, idxs

    def decode_batch(self, idxs, sizes, videos=None, first_chunks=None, stream=None):
        """Decode several token tensors in one grouped pass; ``sizes[i]`` = (H, W)."""
        videos = videos or [None] * len(idxs)
        first_chunks = first_chunks or [None] * len(idxs)
        outs, items = [], []
        for idx, (H, W), v, f in zip(idxs, sizes, videos, first_chunks):
            N, Tq, Hq, Wq = idx.shape
            T = (1 if f else self.s_t) if v is not None else 1 + (Tq - 1) * self.s_t
            out = torch.empty((N, T, H, W, 3), device=idx.device, dtype=torch.float32)
            outs.append(out)
            items.append((_ptr(idx), N, Tq, Hq, Wq, H, W, _ptr(out), v))
        L.tok_decode_batch(self.ctx, items, _stream_ptr(stream))
        return outs

    # -- streaming -----------------------------------------------------------
    def stream_bytes(self, H, W) -> int:
        return L.tok_stream_bytes(self.ctx, H, W)

    def stream_open(self, H, W) -> int:
        """Per-video causal state on the device (the conv caches); reserves the chunk workspace."""
        self.reserve(1, self.s_t, H, W)
        return L.tok_stream_open(self.ctx, H, W)

    def stream_close(self, handle) -> None:
        L.tok_stream_close(handle)

    def stream_reset(self, handle) -> None:
        L.tok_stream_reset(handle)

    @property
    def s_t(self):
        return 1 if self.arch.kind == L.TOK_ARCH_STAGE else self.arch.t_stem * 2 ** (self.arch.nlevels - 1)

    def status(self) -> int:
        return L.tok_status(self.ctx)

    def check_guards(self) -> int:
        """TOK_OK, or TOK_EGUARD if a kernel wrote outside the context's workspaces."""
        return L.tok_check_guards(self.ctx)

    def launch_count(self) -> int:
        return L.tok_launch_count(self.ctx)

    def profile(self, on: bool = True):
        L.tok_profile_enable(self.ctx, on)

    def profile_read(self) -> dict:
        return L.tok_profile_read(self.ctx)

    def profile_records(self) -> list:
        """Per-launch trace since the last profile_read: [{cls, ms, work, name}] in launch order."""
        return L.tok_profile_records(self.ctx)

    def close(self):
        if self.ctx:
            L.tok_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -- stand-alone token ops ----------------------------------------------------

def quantize(z: torch.Tensor, levels=(8, 8, 8, 5, 5, 5), codes=False, stream=None):
    ntok = z.numel() // len(levels)
    idx = torch.empty(z.shape[:-1], device=z.device, dtype=torch.int32)
    cd = torch.empty_like(z) if codes else None
    L.tok_quantize(_ptr(z), ntok, list(levels), _ptr(idx), _ptr(cd), _stream_ptr(stream))
    return (idx, cd) if codes else idx


def dequantize(idx: torch.Tensor, levels=(8, 8, 8, 5, 5, 5), stream=None):
    out = torch.empty((*idx.shape, len(levels)), device=idx.device, dtype=torch.float32)
    L.tok_dequantize(_ptr(idx), idx.numel(), list(levels), _ptr(out), _stream_ptr(stream))
    return out


def zero_index(levels=(8, 8, 8, 5, 5, 5)) -> int:
    return L.tok_zero_index(list(levels))


def drop_mask(idx: torch.Tensor, rate: float, seed: int, stream_id: int = 0, chunk_id: int = 0,
              levels=(8, 8, 8, 5, 5, 5), keep_bits=True, out=None, stream=None):
    N, Tq, Hq, Wq = idx.shape
    if out is None:
        out = torch.empty_like(idx)
    if isinstance(keep_bits, torch.Tensor):
        kb = keep_bits
    elif keep_bits:
        kb = torch.empty((N, Tq, Hq, (Wq + 31) // 32), device=idx.device, dtype=torch.int32)
    else:
        kb = None
    L.tok_drop_mask(_ptr(idx), N, Tq, Hq, Wq, float(rate), int(seed), int(stream_id), int(chunk_id),
                    zero_index(levels), _ptr(out), _ptr(kb), _stream_ptr(stream))
    return out, kb


def similarity_mask(idx_p: torch.Tensor, idx_i: torch.Tensor, rate: float, levels=(8, 8, 8, 5, 5, 5),
                    keep_bits=True, want_sim=False, out=None, workspace=None, stream=None):
    """Similarity-based token selection (Eq. 3): drop the floor(rate * Hq*Wq) P tokens of
    every latent frame most similar (cosine of code vectors) to the I token at the same
    position. idx_p (N, Tp, Hq, Wq), idx_i (N, 1, Hq, Wq). Returns (out, keep_bits, sim)."""
    N, Tp, Hq, Wq = idx_p.shape
    if tuple(idx_i.shape) != (N, 1, Hq, Wq):
        raise ValueError("idx_i must be (N, 1, Hq, Wq)")
    if out is None:
        out = torch.empty_like(idx_p)
    kb = torch.empty((N, Tp, Hq, (Wq + 31) // 32), device=idx_p.device, dtype=torch.int32) if keep_bits else None
    sim = torch.empty((N, Tp, Hq, Wq), device=idx_p.device, dtype=torch.float32) if want_sim else None
    need = L.tok_similarity_workspace_bytes(N, Tp, Hq, Wq)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, device=idx_p.device, dtype=torch.uint8)
    L.tok_similarity_mask(_ptr(idx_p), _ptr(idx_i), N, Tp, Hq, Wq, list(levels), rate, _ptr(out), _ptr(kb),
                          _ptr(sim), _ptr(workspace), workspace.numel(), _stream_ptr(stream))
    return out, kb, sim


def residual(x: torch.Tensor, xhat: torch.Tensor, window: int, theta: float, stream=None):
    """Window-averaged, thresholded pixel residual (Eq. 4): x (N,T,H,W,C) bf16 or fp32,
    xhat fp32 of the same shape -> (N, ceil(T/window), H, W, C) fp32."""
    N, T, H, W, C = x.shape
    prec = L.TOK_BF16 if x.dtype == torch.bfloat16 else L.TOK_FP32
    r = torch.empty((N, (T + window - 1) // window, H, W, C), device=x.device, dtype=torch.float32)
    L.tok_residual(prec, _ptr(x), _ptr(xhat), N, T, H, W, C, window, theta, _ptr(r), _stream_ptr(stream))
    return r


def residual_sparse(r: torch.Tensor, stream=None):
    """Sparse form of a thresholded residual: (positions int32, values fp32, segment
    offsets int64 (N*n_windows + 1)); the arrays hold the worst case, the first
    offsets[-1] entries are used."""
    N, K, H, W, C = r.shape
    cap = r.numel()
    pos = torch.empty(cap, device=r.device, dtype=torch.int32)
    val = torch.empty(cap, device=r.device, dtype=torch.float32)
    offs = torch.empty(N * K + 1, device=r.device, dtype=torch.int64)
    need = L.tok_residual_sparse_workspace_bytes(N, K, H, W, C)
    ws = torch.empty(max(need, 1), device=r.device, dtype=torch.uint8)
    L.tok_residual_sparse(_ptr(r), N, K, H, W, C, _ptr(pos), _ptr(val), _ptr(offs), _ptr(ws), need,
                          _stream_ptr(stream))
    return pos, val, offs


def residual_apply(xhat: torch.Tensor, window: int, pos, val, offs, stream=None):
    """Receiver side: adds each window's residual to every frame of the window (in place)."""
    N, T, H, W, C = xhat.shape
    L.tok_residual_apply(_ptr(xhat), N, T, H, W, C, window, _ptr(pos), _ptr(val), _ptr(offs), pos.numel(),
                         _stream_ptr(stream))
    return xhat


_PIX = {torch.uint8: L.TOK_PIX_U8, torch.bfloat16: L.TOK_PIX_BF16, torch.float32: L.TOK_PIX_FP32}


def downsample(x: torch.Tensor, s: int, out_dtype=torch.bfloat16, out=None, stream=None):
    """Sec. 5 resolution control: s x s area-mean downsampling of frames (..., H, W, C);
    uint8 input is mapped to [-1, 1]. Returns (..., H//s, W//s, C) of out_dtype."""
    if x.dtype not in _PIX:
        raise ValueError("x must be uint8, bfloat16 or float32")
    if out_dtype not in (torch.bfloat16, torch.float32):
        raise ValueError("out_dtype must be bfloat16 or float32")
    *lead, H, W, C = x.shape
    F = 1
    for d in lead:
        F *= d
    if out is None:
        out = torch.empty((*lead, H // s, W // s, C), device=x.device, dtype=out_dtype)
    L.tok_downsample(_PIX[x.dtype], _ptr(x), F, H, W, C, s, PRECISIONS["bf16" if out_dtype == torch.bfloat16
                                                                      else "fp32"], _ptr(out), _stream_ptr(stream))
    return out


def gop_blend(xhat_prev: torch.Tensor, xhat_curr: torch.Tensor, n: int, out=None, stream=None):
    """Eq. 2: blend the first n frames of the current GoP with the last n of the previous one."""
    N, T, H, W, C = xhat_curr.shape
    if out is None:
        out = torch.empty_like(xhat_curr)
    L.tok_gop_blend(_ptr(xhat_prev), xhat_prev.shape[1], _ptr(xhat_curr), _ptr(out), N, T, H, W, C, n,
                    _stream_ptr(stream))
    return out


def temporal_loss(xhat_curr: torch.Tensor, x_prev: torch.Tensor, n: int, grad=True, stream=None):
    """Eq. 1: (loss (1-element fp32 tensor), dL/dxhat_curr or None)."""
    N, Tc, H, W, C = xhat_curr.shape
    loss = torch.empty(1, device=xhat_curr.device, dtype=torch.float32)
    g = torch.empty_like(xhat_curr) if grad else None
    need = L.tok_temporal_loss_workspace_bytes(N, n, H, W, C)
    ws = torch.empty(need, device=xhat_curr.device, dtype=torch.uint8)
    L.tok_temporal_loss(_ptr(xhat_curr), _ptr(x_prev), N, Tc, x_prev.shape[1], H, W, C, n, _ptr(loss), _ptr(g),
                        _ptr(ws), need, _stream_ptr(stream))
    return loss, g


def pack_rows(idx: torch.Tensor, keep_bits: torch.Tensor, stream=None):
    Wq = idx.shape[-1]
    rows = idx.numel() // Wq
    payload = torch.empty(idx.numel(), device=idx.device, dtype=torch.int32)
    offs = torch.empty(rows + 1, device=idx.device, dtype=torch.int64)
    L.tok_pack_rows(_ptr(idx), _ptr(keep_bits), rows, Wq, _ptr(payload), _ptr(offs), _stream_ptr(stream))
    return payload, offs


def unpack_rows(payload, offs, keep_bits, received, shape, levels=(8, 8, 8, 5, 5, 5), stream=None):
    Wq = shape[-1]
    rows = int(np.prod(shape)) // Wq
    out = torch.empty(shape, device=payload.device, dtype=torch.int32)
    L.tok_unpack_rows(_ptr(payload), _ptr(offs), _ptr(keep_bits), _ptr(received), rows, Wq, zero_index(levels),
                      _ptr(out), _stream_ptr(stream))
    return out


def conv3d(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor | None = None, stride=(1, 1, 1),
           time_pad="replicate", residual: torch.Tensor | None = None, stream=None):
    """One causal conv through tok_conv3d. x (N,T,H,W,Cin) bf16 -> BF16 tensor-core path,
    fp32 -> FP32 CUDA-core path; w (Cout,k,k,k,Cin) fp32, bias (Cout) fp32."""
    prec = L.TOK_BF16 if x.dtype == torch.bfloat16 else L.TOK_FP32
    N, T, H, W, Cin = x.shape
    Cout, k = w.shape[0], w.shape[1]
    st, sh, sw = stride
    To = (T - 1) // st + 1
    Ho = (H + 2 * ((k - 1) // 2) - k) // sh + 1
    Wo = (W + 2 * ((k - 1) // 2) - k) // sw + 1
    y = torch.empty((N, To, Ho, Wo, Cout), device=x.device, dtype=x.dtype)
    nb = L.tok_conv3d_workspace_bytes(prec, Cin, Cout, k)
    ws = torch.empty(nb, device=x.device, dtype=torch.uint8)
    L.tok_conv3d(prec, _ptr(x), N, T, H, W, Cin, _ptr(w), _ptr(bias), Cout, k, st, sh, sw,
                 L.TOK_PAD_REPLICATE if time_pad == "replicate" else L.TOK_PAD_ZERO, _ptr(residual), _ptr(y),
                 _ptr(ws), nb, _stream_ptr(stream))
    return y


def groupnorm_silu(x: torch.Tensor, groups: int, gamma=None, beta=None, eps=1e-6, out=None, stream=None):
    """GroupNorm (statistics per sample, group and frame) + SiLU of x (N,T,H,W,C)."""
    prec = L.TOK_BF16 if x.dtype == torch.bfloat16 else L.TOK_FP32
    N, T, H, W, Cc = x.shape
    y = torch.empty_like(x) if out is None else out
    nb = L.tok_groupnorm_workspace_bytes(prec, N * T, H * W, Cc, groups)
    ws = torch.empty(nb, device=x.device, dtype=torch.uint8)
    L.tok_groupnorm_silu(prec, _ptr(x), N * T, H * W, Cc, groups, _ptr(gamma), _ptr(beta), eps, _ptr(y), _ptr(ws),
                         nb, _stream_ptr(stream))
    return y
