"""The hand-written backward on the GPU against the FP64 oracle's gradient.

Same weights, same input, same drop mask (Philox, so identical on both
sides); the oracle runs the rounded (training) forward. Tolerances on the
relative Frobenius error per parameter tensor:
  FP32 path: 1e-4 (FP32 accumulation through ~40 convs, forward and backward)
  BF16 path: 5e-2 (bf16 activations and activation gradients)
plus the loss itself (FP32: 1e-5 relative; BF16: 2e-2).
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import Arch, ops, param_spec
from oracle.grad import OracleTrain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _params(arch, seed):
    rng = np.random.default_rng(seed)
    p = S.weights_for(param_spec(arch), seed=seed)
    for n, shape, kind in param_spec(arch):
        if kind in ("bias", "gn_beta"):
            p[n] = (0.1 * rng.standard_normal(shape)).astype(np.float32)
        elif kind == "gn_gamma":
            p[n] = (1 + 0.1 * rng.standard_normal(shape)).astype(np.float32)
    return p


def _run(P, prec, ch, shape, rate=0.2, seed=7, step=3, margin_keep=None, blocks=1, t_stem=1):
    from paper_2602_03529_b300.train import Trainer
    arch = Arch(ch=ch, blocks=blocks, t_stem=t_stem)
    p = _params(arch, 11)
    if prec == "bf16":
        p = {k: S.to_bf16_f32(v) for k, v in p.items()}
    N, T, H, W = shape
    x = S.blurred_noise_clip(5, N, T, H, W)
    if prec == "bf16":
        x = S.to_bf16_f32(x)
    tk = P.Tokenizer(prec, ch=ch, blocks=blocks, t_stem=t_stem)
    tk.set_params(p)
    tr = Trainer(tk, N, T, H, W)
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    xd = torch.from_numpy(x).to("cuda", dt)
    Tq, Hq, Wq = tk.latent_shape(T, H, W)
    o = OracleTrain(arch, p, surrogate=False)
    kb = None
    if margin_keep is not None:
        # keep only tokens whose every channel is at least `margin_keep` away from a
        # rounding boundary in the oracle, so that both sides quantise them alike
        _, _, b = o.encode(x)
        margin = np.abs((b - np.floor(b)) - 0.5).min(axis=-1)
        dropped = margin < margin_keep
        kb = torch.from_numpy(ops.keep_bits_from_mask(dropped).view(np.int32)).cuda()
    else:
        dropped = ops.drop_mask(N, Tq, Hq, Wq, rate, seed, 0, step)
    loss = float(tr.forward(xd, rate, seed, step, keep_bits=kb).item())
    g = tr.backward().cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert tk.status() == 0
    loss_ref, _, saved = o.forward_train(x, dropped)
    gref, _ = o.backward(saved)
    off, rel = 0, {}
    for name, shp in tk.param_list():
        n = int(np.prod(shp))
        gg = g[off:off + n].reshape(shp)
        off += n
        ref = gref[name]
        rel[name] = float(np.linalg.norm(gg - ref) / max(np.linalg.norm(ref), 1e-30))
    assert tk.check_guards() == 0
    tk.close()
    return loss, loss_ref, rel


def test_fp32_gradient_matches_oracle(P):
    loss, loss_ref, rel = _run(P, "fp32", (16, 32, 64), (1, 5, 32, 32))
    worst = max(rel.items(), key=lambda kv: kv[1])
    print("fp32 loss", loss, loss_ref, "worst", worst)
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    assert worst[1] <= 1e-4, worst


def test_bf16_gradient_matches_oracle(P):
    """Tokens near a rounding tie are dropped on both sides (a caller mask), so
    the BF16 forward quantises every kept token like the FP64 oracle."""
    loss, loss_ref, rel = _run(P, "bf16", (64, 128, 256), (1, 5, 64, 64), margin_keep=0.12, blocks=2)
    worst = max(rel.items(), key=lambda kv: kv[1])
    print("bf16 loss", loss, loss_ref, "worst", worst, "median", float(np.median(list(rel.values()))))
    # every BF16 weight gradient runs on the tensor cores; these are the layer kinds
    # with their own operand handling: im2col (stem, dec.in), stride 2 (down),
    # narrow output (enc.out, dec.out), 64 input channels
    kinds = ["enc.stem.w", "enc.down0.w", "enc.down1.w", "enc.out.w", "dec.in.w", "dec.out.w",
             "enc.l0.b0.c1.w", "dec.up0.w"]
    print("per-kind weight gradient error", {k: round(rel[k], 5) for k in kinds if k in rel})
    for k in kinds:
        assert rel[k] <= 5e-2, (k, rel[k])
    assert abs(loss - loss_ref) <= 2e-2 * abs(loss_ref)
    assert worst[1] <= 5e-2, worst


def test_fp32_gradient_8x8x8(P):
    """Temporal-stride-2 stem and (2,2,2) pixel head: the stem's weight gradient over the
    strided taps and the depth-to-space adjoint with its trimmed first frame."""
    loss, loss_ref, rel = _run(P, "fp32", (16, 32, 64), (1, 9, 32, 32), t_stem=2)
    worst = max(rel.items(), key=lambda kv: kv[1])
    print("fp32 8x8x8 loss", loss, loss_ref, "worst", worst)
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    assert worst[1] <= 1e-4, worst


def test_bf16_gradient_8x8x8(P):
    loss, loss_ref, rel = _run(P, "bf16", (64, 128, 256), (1, 9, 64, 64), margin_keep=0.12, t_stem=2)
    worst = max(rel.items(), key=lambda kv: kv[1])
    print("bf16 8x8x8 loss", loss, loss_ref, "worst", worst, {k: round(rel[k], 5) for k in ("enc.stem.w", "dec.out.w")})
    assert abs(loss - loss_ref) <= 2e-2 * abs(loss_ref)
    assert worst[1] <= 5e-2, worst


def test_bf16_decoder_gradient_all_dropped(P):
    """With every token dropped the decoder sees only zero codes on both sides:
    decoder gradients match, encoder gradients are exactly zero."""
    loss, loss_ref, rel = _run(P, "bf16", (64, 128, 256), (1, 5, 32, 32), rate=1.0)
    dec = {k: v for k, v in rel.items() if k.startswith("dec.")}
    worst = max(dec.items(), key=lambda kv: kv[1])
    print("bf16 all-dropped loss", loss, loss_ref, "worst decoder", worst)
    assert abs(loss - loss_ref) <= 2e-2 * abs(loss_ref)
    assert worst[1] <= 5e-2, worst


def test_sgd_reduces_loss_and_autograd_node(P):
    from paper_2602_03529_b300.train import Trainer, TokenizerLoss
    tk = P.Tokenizer("bf16", ch=(64, 128, 256), blocks=1)
    tk.set_params(S.weights_for(tk.param_spec(), seed=3))
    N, T, H, W = 1, 5, 32, 32
    tr = Trainer(tk, N, T, H, W)
    x = torch.from_numpy(S.blurred_noise_clip(9, N, T, H, W)).to("cuda", torch.bfloat16)
    losses = [float(tr.step(x, 0.0, 1, i, lr=0.05).item()) for i in range(6)]
    assert losses[-1] < losses[0], losses
    params = tr.params.clone().requires_grad_(True)
    loss = TokenizerLoss.apply(params, x, tr, 0.1, 1, 99)
    loss.backward()
    g2 = tr.backward().clone()
    torch.cuda.synchronize()
    assert torch.equal(params.grad, g2)
    assert tk.status() == 0
    assert tk.check_guards() == 0
    tk.close()


def test_repacked_weights_equal_fresh_context(P):
    """After an SGD step the context re-packs the forward rows and both adjoint layouts of
    every 3x3x3 conv in one pass; the next gradient must equal, bit for bit, the one of a
    fresh context given the same parameters (which packs each layout separately)."""
    from paper_2602_03529_b300.train import Trainer
    N, T, H, W = 1, 5, 32, 32
    kw = dict(ch=(64, 128, 256), blocks=1)
    tk = P.Tokenizer("bf16", **kw)
    tk.set_params(S.weights_for(tk.param_spec(), seed=4))
    tr = Trainer(tk, N, T, H, W)
    x = torch.from_numpy(S.blurred_noise_clip(3, N, T, H, W)).to("cuda", torch.bfloat16)
    tr.step(x, 0.1, 1, 0, lr=0.05)
    l1 = tr.forward(x, 0.1, 1, 1).clone()
    g1 = tr.backward().clone()
    tk2 = P.Tokenizer("bf16", **kw)
    tr2 = Trainer(tk2, N, T, H, W)
    tr2.load(tr.params.clone())
    l2 = tr2.forward(x, 0.1, 1, 1).clone()
    g2 = tr2.backward().clone()
    torch.cuda.synchronize()
    assert tk.status() == 0 and tk2.status() == 0
    assert torch.equal(l1, l2)
    assert torch.equal(g1, g2)
    assert tk.check_guards() == 0
    tk.close()
    assert tk2.check_guards() == 0
    tk2.close()


# ------------------------------------------------------------ memory modes

@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_recompute_and_keep_modes_give_equal_gradients(P, prec):
    """Per-residual-block recomputation (the default: block interiors rebuilt in the
    backward from the kept block input and GroupNorm statistics) and the keep mode
    (interiors kept from the forward) give bitwise the same loss and gradient; the
    recomputing workspace is the smaller one. A backward whose forward ran in the other
    mode is refused."""
    from paper_2602_03529_b300 import _lib as L
    from paper_2602_03529_b300.train import Trainer
    kw = dict(ch=(64, 128, 256), blocks=2)
    p = _params(Arch(**kw), 11)
    if prec == "bf16":
        p = {k: S.to_bf16_f32(v) for k, v in p.items()}
    N, T, H, W = 1, 9, 32, 32
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    xd = torch.from_numpy(S.blurred_noise_clip(5, N, T, H, W)).to("cuda", dt)
    out = {}
    for rc in (True, False):
        tk = P.Tokenizer(prec, **kw)
        tk.set_params(p)
        tr = Trainer(tk, N, T, H, W, recompute=rc)
        loss = tr.forward(xd, 0.2, 7, 3).clone()
        g = tr.backward().clone()
        torch.cuda.synchronize()
        assert tk.status() == 0
        out[rc] = (loss, g, tr.workspace_bytes)
        if rc:
            L.tok_set_train_mode(tk.ctx, L.TOK_TRAIN_KEEP)
            with pytest.raises(L.TokError) as e:
                tr.backward()
            assert e.value.code == L.TOK_ESTATE
        assert tk.check_guards() == 0
        tk.close()
    assert torch.equal(out[True][0], out[False][0])
    assert torch.equal(out[True][1], out[False][1])
    assert out[True][2] < out[False][2], (out[True][2], out[False][2])


def test_fp32_gradient_elementwise(P):
    """FP32 path, every gradient element against the FP64 oracle:
    |g - g_ref| <= 1e-4 * max|g_ref| (of its tensor) + 1e-3 * |g_ref|."""
    from paper_2602_03529_b300.train import Trainer
    arch = Arch(ch=(16, 32, 64), blocks=1)
    p = _params(arch, 11)
    N, T, H, W = 1, 5, 32, 32
    x = S.blurred_noise_clip(5, N, T, H, W)
    tk = P.Tokenizer("fp32", ch=(16, 32, 64), blocks=1)
    tk.set_params(p)
    tr = Trainer(tk, N, T, H, W)
    Tq, Hq, Wq = tk.latent_shape(T, H, W)
    dropped = ops.drop_mask(N, Tq, Hq, Wq, 0.2, 7, 0, 3)
    tr.forward(torch.from_numpy(x).cuda(), 0.2, 7, 3)
    g = tr.backward().cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert tk.status() == 0
    o = OracleTrain(arch, p, surrogate=False)
    _, _, saved = o.forward_train(x, dropped)
    gref, _ = o.backward(saved)
    off, worst = 0, (None, 0.0)
    for name, shp in tk.param_list():
        n = int(np.prod(shp))
        gg, ref = g[off:off + n].reshape(shp), gref[name]
        off += n
        tol = 1e-4 * np.abs(ref).max() + 1e-3 * np.abs(ref) + 1e-30
        r = float((np.abs(gg - ref) / tol).max())
        worst = max(worst, (name, r), key=lambda t: t[1])
    assert tk.check_guards() == 0
    tk.close()
    print("fp32 elementwise worst (error / tolerance)", worst)
    assert worst[1] <= 1.0, worst


# --------------------------------------- sampled gradients at the training shape

# conv -> (kernel size, forward stride, shapes at 2 x 3 x 17 x 256 x 256: forward input,
# output gradient as the weight gradient reads it, input gradient of the adjoint conv)
_L0, _L1 = (2, 17, 128, 128), (2, 9, 64, 64)
SAMPLED = {
    "enc.stem": (3, (1, 2, 2), None, _L0 + (128,), None),
    "enc.l0.b0.c1": (3, (1, 1, 1), _L0 + (128,), _L0 + (128,), _L0 + (128,)),
    "enc.down0": (3, (2, 2, 2), _L0 + (128,), _L1 + (128,), _L0 + (128,)),
    "enc.l1.b0.sc": (1, (1, 1, 1), _L1 + (128,), _L1 + (256,), _L1 + (128,)),
    "dec.up0": (3, (1, 1, 1), _L1 + (256,), _L1 + (1024,), _L1 + (256,)),
    "dec.out": (3, (1, 1, 1), _L0 + (128,), _L0 + (64,), _L0 + (128,)),
}


def test_bf16_sampled_gradients_at_training_shape(P):
    """The weight and input gradients of the BF16 training step at its benchmark shape
    (2 x 3 x 17 x 256 x 256, default tokenizer, recomputing backward, full split-K),
    checked on sampled entries against the oracle's single-entry gradients, computed
    from the traced forward input and output gradient of each layer: the stem (im2col),
    a level-0 3x3x3 conv, the stride-2 down conv, a 1x1x1 shortcut, the up conv before
    its depth-to-space, the 12-channel pixel head. Weight gradients (fp32 sums of exact
    bf16 products over up to ~560k voxels): |g - ref| <= 2e-5 * sum|terms| + 5e-4 |ref|,
    the second term for the tensor cores' FP32 accumulation, which truncates toward zero
    over a long split (measured on the 1024-channel up conv: every entry 0.3 - 2.3e-4
    closer to zero than the exact sum; a wrong tap, channel or padding rule is off by
    the order of |ref| itself); input gradients
    (bf16): |g - ref| <= 2^-8 |ref| + 2e-5 * sum|terms|, and at input frame 0 of a
    replicate-padded 3x3x3 conv 2^-8 (|ref| + sum|terms|): there the adjoint reads the
    summed taps of the padded frames (W0 + W1 + W2, W0 + W1) as one bf16 weight map,
    each sum rounded to bf16. Also: the keep mode gives bitwise the same gradient at
    this shape."""
    from paper_2602_03529_b300.train import Trainer
    arch = Arch()
    p = {k: S.to_bf16_f32(v) for k, v in _params(arch, 11).items()}
    N, T, H, W = 2, 17, 256, 256
    x = S.to_bf16_f32(S.blurred_noise_clip(5, N, T, H, W))
    xd = torch.from_numpy(x).to("cuda", torch.bfloat16)
    tk = P.Tokenizer("bf16")
    tk.set_params(p)
    tr = Trainer(tk, N, T, H, W)
    bufs = {}
    for name, (k, st, xs, ys, dxs) in SAMPLED.items():
        b = {"x": None if xs is None else torch.empty(xs, device="cuda", dtype=torch.bfloat16),
             "dy": torch.empty(ys, device="cuda", dtype=torch.bfloat16),
             "dx": None if dxs is None else torch.empty(dxs, device="cuda", dtype=torch.bfloat16)}
        tk.trace_layer(name + ".wgrad", b["x"], b["dy"], None)
        if b["dx"] is not None:
            tk.trace_layer(name + ".dgrad", None, None, b["dx"])
        bufs[name] = b
    tr.forward(xd, 0.1, 3, 1)
    g = tr.backward().clone()
    torch.cuda.synchronize()
    assert tk.status() == 0
    tk.trace_layer(None)
    offs, o = {}, 0
    for name, shp in tk.param_list():
        offs[name] = (o, tuple(shp))
        o += int(np.prod(shp))
    gh = g.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(17)
    worst = {}
    for name, (k, st, xs, ys, dxs) in SAMPLED.items():
        b = bufs[name]
        w = p[name + ".w"]
        Cout, Cin = w.shape[0], w.shape[-1]
        xin = x if name == "enc.stem" else b["x"].float().cpu().numpy()
        dy = b["dy"][..., :Cout].float().cpu().numpy()
        ent = [(int(rng.integers(Cout)), int(rng.integers(k)), int(rng.integers(k)), int(rng.integers(k)),
                int(rng.integers(Cin))) for _ in range(12)]
        ent += [(0, 0, 0, 0, 0), (Cout - 1, k - 1, k - 1, k - 1, Cin - 1)]
        ref, mag = ops.conv3d_wgrad_entries(dy, xin, (k, k, k), ent, st)
        o0, shp = offs[name + ".w"]
        got = np.array([gh[o0 + np.ravel_multi_index(e, shp)] for e in ent])
        r = np.abs(got - ref) / (2e-5 * mag + 5e-4 * np.abs(ref) + 1e-30)
        worst[name + " dW"] = float(r.max())
        if r.max() > 0.5:
            for e, gv, rv, mv in zip(ent, got, ref, mag):
                print(f"  {name} dW{e}: got {gv:.6e} ref {rv:.6e} sum|terms| {mv:.6e} "
                      f"err/|ref| {abs(gv - rv) / max(abs(rv), 1e-30):.2e} err/sum {abs(gv - rv) / mv:.2e}")
        if b["dx"] is None:
            continue
        Nn, Tn, Hn, Wn = xs[:4]
        pts = [(0, 0, 0, 0), (Nn - 1, Tn - 1, Hn - 1, Wn - 1), (1, 1, Hn - 1, 0)]
        pts += [(int(rng.integers(Nn)), int(rng.integers(Tn)), int(rng.integers(Hn)), int(rng.integers(Wn)))
                for _ in range(9)]
        ref, mag = ops.conv3d_dgrad_entries(dy, w, xs, pts, st)
        got = np.stack([b["dx"][n, t, h, wv, :Cin].double().cpu().numpy() for n, t, h, wv in pts])
        fold = np.array([t == 0 and k == 3 for _, t, _, _ in pts])[:, None]
        tol = 2.0 ** -8 * np.abs(ref) + np.where(fold, 2.0 ** -8, 2e-5) * mag + 1e-30
        r = np.abs(got - ref) / tol
        worst[name + " dX"] = float(r.max())
    print("sampled gradients, worst error / tolerance:", worst)
    assert max(worst.values()) <= 1.0, worst
    assert tk.check_guards() == 0
    tk.close()
    tk2 = P.Tokenizer("bf16")
    tk2.set_params(p)
    tr2 = Trainer(tk2, N, T, H, W, recompute=False)
    tr2.forward(xd, 0.1, 3, 1)
    g2 = tr2.backward().clone()
    torch.cuda.synchronize()
    assert tk2.status() == 0
    assert torch.equal(g, g2)
    assert tk2.check_guards() == 0
    tk2.close()
