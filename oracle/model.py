"""FP64 reference tokenizer: encoder f_phi, FSQ, masking, decoder g_theta.

TEST INFRASTRUCTURE ONLY (the oracle). Imported only by tests, the smoke
check and the benchmark's CPU-baseline leg.

The paper defines the codec as an encoder f_phi mapping x_{0:T} in
R^{(1+T) x H x W x 3} to latents z_{0:T'} in R^{(1+T') x H' x W' x C} with
spatial factor s_HW and temporal factor s_T, and a decoder g_theta back to
pixels (Sec. 2.4); it uses the 4x temporal / 8x8 spatial setting as one of the
two standard settings (Sec. 4.1) built from causal residual blocks (Sec. 1,
C2). The paper gives no layer list; the one here follows the workload
description the implementation is measured on:

  encoder: stem conv k3 stride (t_stem,2,2) -> per level l: ``blocks`` causal
  residual blocks (GN -> SiLU -> conv -> GN -> SiLU -> conv, plus a skip that is
  a 1x1x1 conv when channels change) -> between levels a k3 conv with stride
  (2,2,2) -> GN -> SiLU -> conv to the latent dim -> FSQ.
  decoder (mirror): conv from the code vectors -> per level (deepest first)
  ``blocks`` residual blocks -> a k3 conv to C_{l-1} * 8 channels followed by
  depth-to-space (2,2,2) -> ... -> GN -> SiLU -> conv to 3*4*t_stem channels ->
  depth-to-space (t_stem,2,2) -> crop.

t_stem = 1 gives the 4x temporal / 8x8 spatial setting; t_stem = 2 adds a
third temporal halving in the stem: the paper's own asymmetric 8x temporal,
8x8 spatial setting (Sec. 4.1), whose 9-frame GoP is one I frame coded only
spatially plus 8 P frames coded jointly (Sec. 6.3).

The single-stage variant ("stage") is: conv k3 in->c0 (no activation) ->
conv k3 stride (1,2,2) c0->c1 -> GN -> SiLU -> 1x1x1 conv c1->zdim -> FSQ.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ops


@dataclass(frozen=True)
class Arch:
    kind: str = "full"                 # "full" tokenizer or single encoder "stage"
    in_ch: int = 3
    ch: tuple = (128, 256, 512)        # channels per level (full) / (c0, c1) (stage)
    blocks: int = 2                    # residual blocks per level
    levels: tuple = (8, 8, 8, 5, 5, 5) # FSQ levels; zdim = len(levels)
    gn_groups: int = 32
    gn_eps: float = 1e-6
    time_pad: int = ops.PAD_REPLICATE
    t_stem: int = 1                    # temporal stride of the stem: 1 (4x8x8) or 2 (8x8x8)

    @property
    def zdim(self) -> int:
        return len(self.levels)

    @property
    def nlevels(self) -> int:
        return len(self.ch)

    @property
    def s_t(self) -> int:
        """Temporal compression: the stem's temporal stride times one stride-2 per level transition."""
        return 1 if self.kind == "stage" else self.t_stem * 2 ** (self.nlevels - 1)

    @property
    def s_hw(self) -> int:
        """Spatial compression: the stride-2 stem times one stride-2 per level transition."""
        return 2 if self.kind == "stage" else 2 ** self.nlevels


def _conv_spec(name, cout, cin, k=3, kind="conv"):
    return [(name + ".w", (cout, k, k, k, cin), kind), (name + ".b", (cout,), "bias")]


def _gn_spec(name, c):
    return [(name + ".g", (c,), "gn_gamma"), (name + ".b", (c,), "gn_beta")]


def _block_spec(name, cin, cout):
    s = _gn_spec(name + ".gn1", cin) + _conv_spec(name + ".c1", cout, cin)
    s += _gn_spec(name + ".gn2", cout) + _conv_spec(name + ".c2", cout, cout)
    if cin != cout:
        s += _conv_spec(name + ".sc", cout, cin, k=1)
    return s


def param_spec(arch: Arch):
    """Ordered list of (name, shape, kind) for every parameter."""
    c = arch.ch
    if arch.kind == "stage":
        s = _conv_spec("stage.c0", c[0], arch.in_ch) + _conv_spec("stage.c1", c[1], c[0])
        s += _gn_spec("stage.gn", c[1]) + _conv_spec("stage.out", arch.zdim, c[1], k=1)
        return s
    s = _conv_spec("enc.stem", c[0], arch.in_ch)
    for l in range(arch.nlevels):
        cin = c[l - 1] if l > 0 else c[0]
        for b in range(arch.blocks):
            s += _block_spec(f"enc.l{l}.b{b}", cin if b == 0 else c[l], c[l])
        if l < arch.nlevels - 1:
            s += _conv_spec(f"enc.down{l}", c[l], c[l])
    s += _gn_spec("enc.out_gn", c[-1]) + _conv_spec("enc.out", arch.zdim, c[-1])
    s += _conv_spec("dec.in", c[-1], arch.zdim)
    for l in reversed(range(arch.nlevels)):
        for b in range(arch.blocks):
            s += _block_spec(f"dec.l{l}.b{b}", c[l], c[l])
        if l > 0:
            s += _conv_spec(f"dec.up{l - 1}", c[l - 1] * 8, c[l])
    s += _gn_spec("dec.out_gn", c[0]) + _conv_spec("dec.out", arch.in_ch * 4 * arch.t_stem, c[0])
    return s


class Oracle:
    """The reference tokenizer over a dict of named float parameters.

    act_bf16: model BF16 activations ("BF16 weights/activations with FP32
    accumulation" of the workload description): every tensor a layer stores
    between layers -- the stem, residual-block and down-conv outputs, every
    GroupNorm+SiLU output, the up-conv outputs and the decoder input conv's
    output -- is the exact value rounded to float32 and then to the nearest
    bfloat16 (ties to even), as an FP32 accumulator is stored in bf16. A
    residual block's output is rounded once, after its skip is added. The
    latent z and the decoded pixels stay unrounded. Default: exact FP64."""

    def __init__(self, arch: Arch, params: dict, act_bf16: bool = False):
        self.arch = arch
        self.act_bf16 = act_bf16
        self.p = {k: np.asarray(v, dtype=np.float64) for k, v in params.items()}
        names = [n for n, _, _ in param_spec(arch)]
        missing = [n for n in names if n not in self.p]
        if missing:
            raise KeyError(f"missing parameters: {missing[:5]}")

    # -- building blocks -------------------------------------------------
    def store(self, x):
        """The value of a stored activation (see act_bf16)."""
        if not self.act_bf16:
            return x
        return ops.round_to_bf16(np.asarray(x, dtype=np.float32)).astype(np.float64)

    def conv(self, name, x, stride=(1, 1, 1)):
        return ops.conv3d(x, self.p[name + ".w"], self.p[name + ".b"], stride, self.arch.time_pad)

    def gn_silu(self, name, x):
        C = x.shape[-1]
        g = ops.gn_groups(C, self.arch.gn_groups)
        return self.store(ops.silu(ops.group_norm_frames(x, g, self.arch.gn_eps,
                                                         self.p[name + ".g"], self.p[name + ".b"])))

    def block(self, name, x):
        """Causal residual block: skip(x) + conv2(SiLU(GN2(conv1(SiLU(GN1(x))))))."""
        h = self.store(self.conv(name + ".c1", self.gn_silu(name + ".gn1", x)))
        h = self.conv(name + ".c2", self.gn_silu(name + ".gn2", h))
        skip = self.store(self.conv(name + ".sc", x)) if (name + ".sc.w") in self.p else x
        return self.store(skip + h)

    # -- encoder ---------------------------------------------------------
    def encode_latent(self, x):
        """x (N,T,H,W,3) in [-1,1] -> pre-quantisation latent z (N,T',H',W',zdim)."""
        a = self.arch
        x = ops.edge_pad_to_multiple(np.asarray(x, dtype=np.float64), a.s_hw)
        if a.kind == "stage":
            h = self.store(self.conv("stage.c0", x))
            h = self.store(self.conv("stage.c1", h, (1, 2, 2)))
            return self.conv("stage.out", self.gn_silu("stage.gn", h))
        h = self.store(self.conv("enc.stem", x, (a.t_stem, 2, 2)))
        for l in range(a.nlevels):
            for b in range(a.blocks):
                h = self.block(f"enc.l{l}.b{b}", h)
            if l < a.nlevels - 1:
                h = self.store(self.conv(f"enc.down{l}", h, (2, 2, 2)))
        return self.conv("enc.out", self.gn_silu("enc.out_gn", h))

    def encode(self, x):
        """Returns (idx int64 (N,T',H',W'), z float64, bound float64)."""
        z = self.encode_latent(x)
        idx, _, b = ops.fsq_quantize(z, self.arch.levels)
        return idx, z, b

    # -- decoder ---------------------------------------------------------
    def decode_codes(self, codes, H, W):
        """Code vectors (N,T',H',W',zdim) -> pixels (N,T,H,W,3), cropped to H x W."""
        a = self.arch
        h = self.store(self.conv("dec.in", codes))
        for l in reversed(range(a.nlevels)):
            for b in range(a.blocks):
                h = self.block(f"dec.l{l}.b{b}", h)
            if l > 0:
                h = self.store(ops.depth_to_space(self.conv(f"dec.up{l - 1}", h), (2, 2, 2)))
        y = self.conv("dec.out", self.gn_silu("dec.out_gn", h))
        y = ops.depth_to_space(y, (a.t_stem, 2, 2))
        return y[:, :, :H, :W, :]

    def decode(self, idx, H, W):
        return self.decode_codes(ops.fsq_dequantize(idx, self.arch.levels), H, W)


def latent_shape(arch: Arch, N, T, H, W):
    """(N, T', H', W') of the token matrix for an N x T x H x W clip:
    T' = 1 + (T-1)/s_T (needs T = 1 mod s_T), H' = ceil(H/s_HW), W' = ceil(W/s_HW)."""
    st, s = arch.s_t, arch.s_hw
    return N, (T - 1) // st + 1, -(-H // s), -(-W // s)
