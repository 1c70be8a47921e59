"""FP64 gradient of the tokenizer's training objective (straight-through FSQ).

TEST INFRASTRUCTURE ONLY (the oracle). Imported only by tests and the
benchmark's CPU-baseline leg.

The paper trains encoder and decoder jointly on reconstructions from token
matrices with randomly dropped, zero-filled tokens, and the gradient reaches
the encoder through the masked decode (Sec. 7, codec training; Appendix A.2,
Eq. 7). Its losses (L1 + optical flow + adversarial, Eq. 5-6) need networks
and data that are not available; the objective here is the mean squared
reconstruction error L = mean((x_hat - x)^2), with x_hat = g(drop(FSQ(f(x)))).

FSQ's rounding has zero derivative almost everywhere; the straight-through
estimator replaces d round(b)/db by 1. Its gradient is exactly the gradient of
the "surrogate" network in which round is the identity, which is what the
finite-difference pin (tests/test_oracle_grad.py) differentiates.

The backward here is written layer by layer as the adjoint of each forward
step of model.Oracle (conv: conv3d_dgrad / conv3d_wgrad in C; GroupNorm per
frame; SiLU; depth-to-space; crop; edge padding), with every saved forward
value recomputed or kept explicitly.
"""
from __future__ import annotations

import numpy as np

from . import ops
from .model import Arch, Oracle


def gn_silu_fwd(x, groups, eps, gamma, beta):
    """y = SiLU(GN(x)) with per-(sample, frame, group) statistics; returns y and
    the values the backward needs."""
    N, T, H, W, C = x.shape
    cg = C // groups
    xg = x.reshape(N, T, H * W, groups, cg)
    mu = xg.mean(axis=(2, 4), keepdims=True)
    var = ((xg - mu) ** 2).mean(axis=(2, 4), keepdims=True)
    r = 1.0 / np.sqrt(var + eps)
    xh = ((xg - mu) * r).reshape(x.shape)
    h = xh * gamma + beta
    s = 1.0 / (1.0 + np.exp(-h))
    return h * s, (xh, r, h, s)


def gn_silu_bwd(dy, saved, groups, gamma):
    """Adjoint of gn_silu_fwd: dx, dgamma, dbeta.

    SiLU'(h) = s (1 + h (1 - s)); with g = dh * gamma and n = C/G * H * W
    elements per group, dx = r (g - mean(g) - xh * mean(g * xh))."""
    xh, r, h, s = saved
    N, T, H, W, C = dy.shape
    dh = dy * s * (1.0 + h * (1.0 - s))
    dgamma = (dh * xh).sum(axis=(0, 1, 2, 3))
    dbeta = dh.sum(axis=(0, 1, 2, 3))
    cg = C // groups
    g = (dh * gamma).reshape(N, T, H * W, groups, cg)
    xhg = xh.reshape(N, T, H * W, groups, cg)
    m1 = g.mean(axis=(2, 4), keepdims=True)
    m2 = (g * xhg).mean(axis=(2, 4), keepdims=True)
    dx = (r * (g - m1 - xhg * m2)).reshape(dy.shape)
    return dx, dgamma, dbeta


def d2s_bwd(dout, r):
    """Adjoint of ops.depth_to_space (with its causal trim): space-to-depth with
    zeros for the trimmed frames."""
    return ops.space_to_depth(dout, r)


def fsq_ste_fwd(z, levels):
    """Codes of the surrogate (round -> identity) and of the true quantiser."""
    h, o, s, hw, _ = ops.fsq_constants(levels)
    t = np.tanh(z + s)
    b = t * h - o
    return b / hw, np.rint(b) / hw, (t, h, hw)


def fsq_ste_bwd(dcodes, saved):
    """d code_i / d z_i = h_i (1 - tanh^2(z_i + s_i)) / floor(L_i/2) (rounding passed straight through)."""
    t, h, hw = saved
    return dcodes * h * (1.0 - t * t) / hw


class OracleTrain(Oracle):
    """Forward (keeping every value the backward needs) and exact backward of
    L = mean((x_hat - x)^2) with FSQ straight-through and a fixed drop mask.

    `surrogate=True` replaces rounding by the identity in the forward as well,
    which makes L differentiable and lets finite differences check the
    gradient; `surrogate=False` is the training forward (rounded codes, same
    gradient)."""

    def __init__(self, arch: Arch, params: dict, surrogate: bool = False):
        super().__init__(arch, params)
        self.surrogate = surrogate

    # -- pieces with tapes ------------------------------------------------
    def _conv(self, tape, name, x, stride=(1, 1, 1)):
        y = ops.conv3d(x, self.p[name + ".w"], self.p[name + ".b"], stride, self.arch.time_pad)
        tape.append(("conv", name, x, stride))
        return y

    def _gn(self, tape, name, x):
        G = ops.gn_groups(x.shape[-1], self.arch.gn_groups)
        y, saved = gn_silu_fwd(x, G, self.arch.gn_eps, self.p[name + ".g"], self.p[name + ".b"])
        tape.append(("gn", name, saved, G))
        return y

    def _block(self, tape, name, x):
        tape.append(("block_begin", name, x))
        h = self._conv(tape, name + ".c1", self._gn(tape, name + ".gn1", x))
        h = self._conv(tape, name + ".c2", self._gn(tape, name + ".gn2", h))
        if (name + ".sc.w") in self.p:
            skip = self._conv(tape, name + ".sc", x)
        else:
            skip = x
        tape.append(("block_end", name))
        return skip + h

    def forward_train(self, x, dropped):
        """x (N,T,H,W,3) with H, W multiples of 8; dropped (N,T',H',W') bool.
        Returns (loss, x_hat, tape)."""
        a = self.arch
        assert a.kind == "full"
        x = np.asarray(x, dtype=np.float64)
        assert x.shape[2] % a.s_hw == 0 and x.shape[3] % a.s_hw == 0, "training needs H, W multiples of 8"
        tape = []
        h = self._conv(tape, "enc.stem", x, (a.t_stem, 2, 2))
        for l in range(a.nlevels):
            for b in range(a.blocks):
                h = self._block(tape, f"enc.l{l}.b{b}", h)
            if l < a.nlevels - 1:
                h = self._conv(tape, f"enc.down{l}", h, (2, 2, 2))
        z = self._conv(tape, "enc.out", self._gn(tape, "enc.out_gn", h))
        c_sur, c_round, saved = fsq_ste_fwd(z, a.levels)
        codes = c_sur if self.surrogate else c_round
        keep = ~np.asarray(dropped, dtype=bool)
        codes = codes * keep[..., None]
        tape.append(("fsq", saved, keep))
        h = self._conv(tape, "dec.in", codes)
        for l in reversed(range(a.nlevels)):
            for b in range(a.blocks):
                h = self._block(tape, f"dec.l{l}.b{b}", h)
            if l > 0:
                h = ops.depth_to_space(self._conv(tape, f"dec.up{l - 1}", h), (2, 2, 2))
                tape.append(("d2s", (2, 2, 2)))
        y = self._conv(tape, "dec.out", self._gn(tape, "dec.out_gn", h))
        xh = ops.depth_to_space(y, (a.t_stem, 2, 2))
        tape.append(("d2s", (a.t_stem, 2, 2)))
        loss = float(np.mean((xh - x) ** 2))
        return loss, xh, (tape, x, xh, z)

    def backward(self, saved):
        """Gradients of the loss with respect to every parameter and to x.

        Walks the tape backwards. A residual block y = skip(x) + h(x) is seen
        as: block_end (g flows to both branches), [shortcut conv], the h
        branch, block_begin (the two input gradients are summed)."""
        tape, x, xh, z = saved
        grads = {k: np.zeros_like(v) for k, v in self.p.items()}
        g = 2.0 * (xh - x) / xh.size
        dx_in = -g.copy()  # the loss's direct dependence on its target x
        blocks = []  # per open block: {"skip": grad of x via the skip, "h": grad entering the h branch}
        for item in reversed(tape):
            kind = item[0]
            if kind == "d2s":
                g = d2s_bwd(g, item[1])
            elif kind == "conv":
                _, name, xin, stride = item
                w = self.p[name + ".w"]
                dw, db = ops.conv3d_wgrad(g, xin, w.shape[1:4], stride, self.arch.time_pad)
                grads[name + ".w"] += dw
                grads[name + ".b"] += db
                g = ops.conv3d_dgrad(g, w, xin.shape, stride, self.arch.time_pad)
                if name.endswith(".sc"):
                    blocks[-1]["skip"] = g
                    g = blocks[-1]["h"]
            elif kind == "gn":
                _, name, sv, G = item
                g, dga, dbe = gn_silu_bwd(g, sv, G, self.p[name + ".g"])
                grads[name + ".g"] += dga
                grads[name + ".b"] += dbe
            elif kind == "block_end":
                name = item[1]
                has_sc = (name + ".sc.w") in self.p
                # identity skip: x receives g directly; shortcut conv: replayed next
                blocks.append({"skip": None if has_sc else g.copy(), "h": g.copy()})
            elif kind == "block_begin":
                b = blocks.pop()
                g = g + b["skip"]
            elif kind == "fsq":
                _, sv, keep = item
                g = fsq_ste_bwd(g * keep[..., None], sv)
        dx_in += g
        return grads, dx_in
