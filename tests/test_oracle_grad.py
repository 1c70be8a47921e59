"""Pins of the oracle's training gradient (straight-through FSQ, MSE, fixed drop mask).

* Central finite differences in FP64 on the surrogate network (rounding
  replaced by the identity, whose exact gradient is the straight-through
  gradient), on the 1x3x5x32x32 copy with channels 16/32/64.
* The GroupNorm+SiLU adjoint against torch autograd in FP64 (library).
* The straight-through FSQ derivative against its closed form h(1-tanh^2)/floor(L/2).
"""
import numpy as np
import torch
import torch.nn.functional as F

import synthetic as S
from oracle import Arch, ops, param_spec
from oracle.grad import OracleTrain, fsq_ste_bwd, fsq_ste_fwd, gn_silu_bwd, gn_silu_fwd

ARCH = Arch(ch=(16, 32, 64), blocks=1)


def _params(seed=0):
    rng = np.random.default_rng(seed)
    p = S.weights_for(param_spec(ARCH), seed=seed)
    for n, shape, kind in param_spec(ARCH):
        if kind == "bias" or kind == "gn_beta":
            p[n] = (0.1 * rng.standard_normal(shape)).astype(np.float64)
        elif kind == "gn_gamma":
            p[n] = (1 + 0.1 * rng.standard_normal(shape)).astype(np.float64)
        else:
            p[n] = p[n].astype(np.float64)
    return p


def test_gn_silu_bwd_matches_torch():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5, 16)) * 2 + 0.5
    ga, be = 1 + 0.2 * rng.standard_normal(16), 0.2 * rng.standard_normal(16)
    dy = rng.standard_normal(x.shape)
    y, sv = gn_silu_fwd(x, 8, 1e-6, ga, be)
    dx, dga, dbe = gn_silu_bwd(dy, sv, 8, ga)
    xt = torch.from_numpy(x).requires_grad_(True)
    gt = torch.from_numpy(ga).requires_grad_(True)
    bt = torch.from_numpy(be).requires_grad_(True)
    xf = xt.reshape(6, 4, 5, 16).permute(0, 3, 1, 2)
    yt = F.silu(F.group_norm(xf, 8, gt, bt, eps=1e-6)).permute(0, 2, 3, 1).reshape(x.shape)
    np.testing.assert_allclose(y, yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    (yt * torch.from_numpy(dy)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dga, gt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dbe, bt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_fsq_ste_derivative_closed_form():
    lv = (8, 8, 8, 5, 5, 5)
    z = np.linspace(-3, 3, 61)[:, None] * np.ones((1, 6))
    c, _, sv = fsq_ste_fwd(z, lv)
    d = fsq_ste_bwd(np.ones_like(z), sv)
    h, o, s, hw, _ = ops.fsq_constants(lv)
    eps = 1e-6
    fd = (fsq_ste_fwd(z + eps, lv)[0] - fsq_ste_fwd(z - eps, lv)[0]) / (2 * eps)
    np.testing.assert_allclose(d, fd, rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(d, h * (1 - np.tanh(z + s) ** 2) / hw, rtol=1e-14)


def test_full_gradient_finite_differences():
    p = _params(0)
    x = S.blurred_noise_clip(0, 1, 5, 32, 32).astype(np.float64)
    dropped = np.random.default_rng(2).random((1, 2, 4, 4)) < 0.2
    o = OracleTrain(ARCH, p, surrogate=True)
    loss, _, saved = o.forward_train(x, dropped)
    grads, dx = o.backward(saved)

    def L(pp=None, xx=None):
        oo = OracleTrain(ARCH, pp if pp is not None else p, surrogate=True)
        return oo.forward_train(x if xx is None else xx, dropped)[0]

    rng = np.random.default_rng(3)
    checked = 0
    for name in ["enc.stem.w", "enc.l0.b0.c1.w", "enc.l1.b0.sc.w", "enc.l2.b0.gn2.g", "enc.down1.b",
                 "enc.out.w", "dec.in.w", "dec.l2.b0.c2.w", "dec.up1.w", "dec.l0.b0.gn1.b", "dec.out.w",
                 "dec.out.b"]:
        g = grads[name]
        scale = np.abs(g).max()
        for _ in range(3):
            i = tuple(int(rng.integers(0, s)) for s in g.shape)
            h = 1e-6 * max(1.0, abs(p[name][i]))
            pp = dict(p)
            pp[name] = p[name].copy()
            pp[name][i] += h
            lp = L(pp)
            pp[name][i] -= 2 * h
            lm = L(pp)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i]) <= 1e-5 * max(abs(g[i]), 1e-3 * scale), (name, i, fd, g[i])
            checked += 1
    for _ in range(4):
        i = tuple(int(rng.integers(0, s)) for s in x.shape)
        xp = x.copy()
        xp[i] += 1e-6
        lp = L(xx=xp)
        xp[i] -= 2e-6
        lm = L(xx=xp)
        fd = (lp - lm) / 2e-6
        assert abs(fd - dx[i]) <= 1e-5 * max(abs(dx[i]), 1e-3 * np.abs(dx).max()), (i, fd, dx[i])
    assert checked == 36


def test_rounded_forward_has_same_gradient_structure():
    """The training forward (rounded codes) and the surrogate share the
    backward; with rounding the loss differs but the gradient of a weight
    that feeds only the decoder output bias is the same closed form."""
    p = _params(4)
    x = S.blurred_noise_clip(1, 1, 5, 16, 16).astype(np.float64)
    dropped = np.zeros((1, 2, 2, 2), bool)
    o = OracleTrain(ARCH, p, surrogate=False)
    loss, xh, saved = o.forward_train(x, dropped)
    grads, _ = o.backward(saved)
    # d loss / d dec.out.b[c] = sum over positions of 2 (xh - x)/n of the channels fed by c
    gb = grads["dec.out.b"]
    r = 2 * (xh - x) / xh.size
    ref = ops.space_to_depth(r, (1, 2, 2)).sum(axis=(0, 1, 2, 3))
    np.testing.assert_allclose(gb, ref, rtol=1e-10, atol=1e-14)


def test_888_gradient_finite_differences():
    """The 8x8x8 setting (stem with temporal stride 2, (2,2,2) pixel head)."""
    a = Arch(ch=(16, 32, 64), blocks=1, t_stem=2)
    rng = np.random.default_rng(7)
    p = {k: np.asarray(v, dtype=np.float64) for k, v in S.weights_for(param_spec(a), seed=5).items()}
    for n, shape, kind in param_spec(a):
        if kind in ("bias", "gn_beta"):
            p[n] = 0.1 * rng.standard_normal(shape)
    x = S.blurred_noise_clip(4, 1, 9, 32, 32).astype(np.float64)
    dropped = rng.random((1, 2, 4, 4)) < 0.2
    o = OracleTrain(a, p, surrogate=True)
    loss, _, saved = o.forward_train(x, dropped)
    grads, dx = o.backward(saved)
    for name in ["enc.stem.w", "enc.l0.b0.c1.w", "dec.out.w", "dec.out.b", "dec.up0.w"]:
        g = grads[name]
        for _ in range(2):
            i = tuple(int(rng.integers(0, s)) for s in g.shape)
            h = 1e-6 * max(1.0, abs(p[name][i]))
            pp = dict(p)
            pp[name] = p[name].copy()
            pp[name][i] += h
            lp = OracleTrain(a, pp, surrogate=True).forward_train(x, dropped)[0]
            pp[name][i] -= 2 * h
            lm = OracleTrain(a, pp, surrogate=True).forward_train(x, dropped)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i]) <= 1e-5 * max(abs(g[i]), 1e-3 * np.abs(g).max()), (name, i, fd, g[i])
