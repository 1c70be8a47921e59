"""Pins of the oracle tokenizer as a whole: layer list and FLOP count of the
reading of the architecture, causality of encoder and decoder, and the
composition checked against an independent PyTorch FP64 build from library
primitives (conv3d, group_norm, silu)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import synthetic as S
from oracle import Arch, Oracle, latent_shape, ops, param_spec


def _walk_flops(arch, shape):
    """Run the oracle with a shape-only conv to list every conv it performs."""
    calls = []
    real = ops.conv3d

    def fake(x, w, b, stride=(1, 1, 1), pad_mode=0):
        N, T, H, W, Cin = x.shape
        Cout, kt, kh, kw, _ = w.shape
        To, Ho, Wo = ops.conv_out_shape(T, H, W, (kt, kh, kw), stride)
        calls.append((N * To * Ho * Wo, Cout, kt * kh * kw * Cin))
        return np.zeros((N, To, Ho, Wo, Cout))

    ops.conv3d = fake
    try:
        p = {n: np.zeros(s) for n, s, _ in param_spec(arch)}
        o = Oracle(arch, p)
        N, T, H, W = shape
        z = o.encode_latent(np.zeros((N, T, H, W, 3)))
        n_enc = len(calls)
        o.decode_codes(np.zeros(z.shape), H, W)
    finally:
        ops.conv3d = real
    fl = [2 * m * n * k for m, n, k in calls]
    return calls, sum(fl[:n_enc]), sum(fl[n_enc:])


def test_layer_list_and_flops_cfg1():
    """Reading B of the architecture (stride-2 stem, levels at /2, /4, /8):
    1x3x17x256x256 costs enc ~1757 + dec ~2633 GFLOP, 4.39 TFLOP per clip."""
    a = Arch()
    calls, fe, fd = _walk_flops(a, (1, 17, 256, 256))
    assert calls[0] == (17 * 128 * 128, 128, 81)               # enc.stem
    assert (36864, 256, 3456) in calls                          # enc.l1.b0.c1
    assert (5120, 2048, 13824) in calls                         # dec.up1
    assert (278528, 12, 3456) == calls[-1]                      # dec.out
    assert abs(fe / 1e9 - 1757) < 2 and abs(fd / 1e9 - 2633) < 2
    assert abs((fe + fd) / 1e12 - 4.39) < 0.01


def test_param_spec_shapes():
    spec = {n: s for n, s, _ in param_spec(Arch())}
    assert spec["enc.stem.w"] == (128, 3, 3, 3, 3)
    assert spec["enc.l1.b0.sc.w"] == (256, 1, 1, 1, 128)
    assert spec["enc.out.w"] == (6, 3, 3, 3, 512)
    assert spec["dec.in.w"] == (512, 3, 3, 3, 6)
    assert spec["dec.up0.w"] == (1024, 3, 3, 3, 256)
    assert spec["dec.out.w"] == (12, 3, 3, 3, 128)
    assert "enc.l0.b0.sc.w" not in spec


def test_latent_shapes():
    assert latent_shape(Arch(), 1, 17, 256, 256) == (1, 5, 32, 32)
    assert latent_shape(Arch(), 1, 17, 720, 1280) == (1, 5, 90, 160)
    assert latent_shape(Arch(), 1, 17, 480, 854) == (1, 5, 60, 107)
    assert latent_shape(Arch(kind="stage", ch=(64, 128)), 1, 9, 64, 64) == (1, 9, 32, 32)


SMALL = Arch(ch=(8, 16, 32), blocks=1)


def _small_params(arch=SMALL, seed=0):
    return S.weights_for(param_spec(arch), seed=seed)


def test_encoder_causal():
    """Latent t depends only on frames <= 4t: perturbing later frames leaves
    latents 0..t bit-identical."""
    o = Oracle(SMALL, _small_params())
    x = S.blurred_noise_clip(1, 1, 9, 16, 16)
    z0 = o.encode_latent(x)
    assert z0.shape == (1, 3, 2, 2, 6)
    rng = np.random.default_rng(0)
    for t in range(3):
        x2 = x.copy()
        x2[:, 4 * t + 1:] = rng.uniform(-1, 1, x2[:, 4 * t + 1:].shape)
        z1 = o.encode_latent(x2)
        np.testing.assert_array_equal(z0[:, :t + 1], z1[:, :t + 1])
        if 4 * t + 1 < 9:
            assert not np.array_equal(z0[:, t + 1:], z1[:, t + 1:])


def test_decoder_causal():
    """Decoded frame f depends only on latents <= ceil(f/4)."""
    o = Oracle(SMALL, _small_params())
    rng = np.random.default_rng(1)
    codes = rng.uniform(-1, 1, (1, 3, 2, 2, 6))
    y0 = o.decode_codes(codes, 16, 16)
    assert y0.shape == (1, 9, 16, 16, 3)
    for k in (1, 2):
        c2 = codes.copy()
        c2[:, k] += 0.5
        y1 = o.decode_codes(c2, 16, 16)
        last_unchanged = 4 * (k - 1)
        np.testing.assert_array_equal(y0[:, :last_unchanged + 1], y1[:, :last_unchanged + 1])
        assert not np.array_equal(y0[:, last_unchanged + 1:], y1[:, last_unchanged + 1:])


# --- an independent build of the network from PyTorch FP64 primitives -------

def _t(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64))


def _tconv(x, p, name, stride=(1, 1, 1)):
    w = _t(p[name + ".w"]).permute(0, 4, 1, 2, 3)
    kt, kh, kw = w.shape[2:]
    if kt > 1:
        x = torch.cat([x[:, :, :1].expand(-1, -1, kt - 1, -1, -1), x], dim=2)
    x = F.pad(x, ((kw - 1) // 2,) * 2 + ((kh - 1) // 2,) * 2 + (0, 0))
    return F.conv3d(x, w, _t(p[name + ".b"]), stride=stride)


def _tgn(x, p, name, groups=32):
    N, C, T, H, W = x.shape
    g = max(1, min(groups, C // 2))
    xf = x.permute(0, 2, 1, 3, 4).reshape(N * T, C, H, W)
    y = F.group_norm(xf, g, _t(p[name + ".g"]), _t(p[name + ".b"]), eps=1e-6)
    return F.silu(y.reshape(N, T, C, H, W).permute(0, 2, 1, 3, 4))


def _tblock(x, p, name):
    h = _tconv(_tgn(x, p, name + ".gn1"), p, name + ".c1")
    h = _tconv(_tgn(h, p, name + ".gn2"), p, name + ".c2")
    s = _tconv(x, p, name + ".sc") if name + ".sc.w" in p else x
    return s + h


def _td2s(y, r):
    N, C, T, H, W = y.shape
    rt, rh, rw = r
    Co = C // (rt * rh * rw)
    y = y.reshape(N, rt, rh, rw, Co, T, H, W).permute(0, 4, 5, 1, 6, 2, 7, 3)
    return y.reshape(N, Co, T * rt, H * rh, W * rw)[:, :, rt - 1:]


def test_stage_matches_torch_fp64():
    a = Arch(kind="stage", ch=(64, 128))
    p = S.weights_for(param_spec(a), seed=3)
    x = S.blurred_noise_clip(0, 1, 5, 16, 16)
    z = Oracle(a, p).encode_latent(x)
    xt = _t(x).permute(0, 4, 1, 2, 3)
    h = _tconv(xt, p, "stage.c0")
    h = _tconv(h, p, "stage.c1", (1, 2, 2))
    zt = _tconv(_tgn(h, p, "stage.gn"), p, "stage.out").permute(0, 2, 3, 4, 1).numpy()
    np.testing.assert_allclose(z, zt, rtol=1e-9, atol=1e-9)


def test_full_model_matches_torch_fp64():
    a = SMALL
    p = _small_params(a, seed=4)
    x = S.blurred_noise_clip(2, 1, 5, 16, 24)
    o = Oracle(a, p)
    z = o.encode_latent(x)
    xt = _t(x).permute(0, 4, 1, 2, 3)
    h = _tconv(xt, p, "enc.stem", (1, 2, 2))
    for l in range(3):
        h = _tblock(h, p, f"enc.l{l}.b0")
        if l < 2:
            h = _tconv(h, p, f"enc.down{l}", (2, 2, 2))
    zt = _tconv(_tgn(h, p, "enc.out_gn"), p, "enc.out")
    np.testing.assert_allclose(z, zt.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-9, atol=1e-9)
    codes = np.random.default_rng(3).uniform(-1, 1, z.shape)
    y = o.decode_codes(codes, 16, 24)
    h = _tconv(_t(codes).permute(0, 4, 1, 2, 3), p, "dec.in")
    for l in (2, 1, 0):
        h = _tblock(h, p, f"dec.l{l}.b0")
        if l > 0:
            h = _td2s(_tconv(h, p, f"dec.up{l - 1}"), (2, 2, 2))
    yt = _td2s(_tconv(_tgn(h, p, "dec.out_gn"), p, "dec.out"), (1, 2, 2))
    np.testing.assert_allclose(y, yt.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-9, atol=1e-9)


def test_block_with_zero_second_conv_is_skip():
    """A residual block whose second conv is zero returns its skip path."""
    a = Arch(ch=(8, 16, 32), blocks=1)
    p = _small_params(a, seed=5)
    for n in ("enc.l0.b0", "enc.l1.b0"):
        p[n + ".c2.w"] = np.zeros_like(p[n + ".c2.w"])
    o = Oracle(a, p)
    x = np.random.default_rng(0).standard_normal((1, 3, 4, 4, 8))
    np.testing.assert_array_equal(o.block("enc.l0.b0", x), x)
    np.testing.assert_allclose(o.block("enc.l1.b0", x), o.conv("enc.l1.b0.sc", x), rtol=0, atol=0)


@pytest.mark.parametrize("H,W", [(20, 30), (17, 33)])
def test_crop_and_pad_shapes(H, W):
    o = Oracle(SMALL, _small_params())
    x = S.blurred_noise_clip(3, 1, 5, H, W)
    idx, z, _ = o.encode(x)
    assert idx.shape == latent_shape(SMALL, 1, 5, H, W)
    y = o.decode(idx, H, W)
    assert y.shape == (1, 5, H, W, 3)


# --- the paper's 8x temporal, 8x8 spatial setting (stem with temporal stride 2) ---

SMALL8 = Arch(ch=(8, 16, 32), blocks=1, t_stem=2)


def test_888_shapes_and_params():
    a = Arch(t_stem=2)
    assert a.s_t == 8 and a.s_hw == 8
    assert latent_shape(a, 1, 9, 720, 1280) == (1, 2, 90, 160)   # a 9-frame GoP: 1 I + 8 P frames
    assert latent_shape(a, 1, 17, 256, 256) == (1, 3, 32, 32)
    spec = {n: s for n, s, _ in param_spec(a)}
    assert spec["dec.out.w"] == (24, 3, 3, 3, 128)                # 3 channels x (2,2,2) depth-to-space


def test_888_encoder_decoder_causal():
    """Latent t depends only on frames <= 8t; decoded frame f only on latents <= ceil(f/8)."""
    o = Oracle(SMALL8, _small_params(SMALL8, seed=6))
    x = S.blurred_noise_clip(3, 1, 17, 16, 16)
    z0 = o.encode_latent(x)
    assert z0.shape == (1, 3, 2, 2, 6)
    rng = np.random.default_rng(0)
    for t in range(3):
        x2 = x.copy()
        x2[:, 8 * t + 1:] = rng.uniform(-1, 1, x2[:, 8 * t + 1:].shape)
        z1 = o.encode_latent(x2)
        np.testing.assert_array_equal(z0[:, :t + 1], z1[:, :t + 1])
    codes = rng.uniform(-1, 1, (1, 3, 2, 2, 6))
    y0 = o.decode_codes(codes, 16, 16)
    assert y0.shape == (1, 17, 16, 16, 3)
    for k in (1, 2):
        c2 = codes.copy()
        c2[:, k] += 0.5
        y1 = o.decode_codes(c2, 16, 16)
        np.testing.assert_array_equal(y0[:, :8 * (k - 1) + 1], y1[:, :8 * (k - 1) + 1])
        assert not np.array_equal(y0[:, 8 * (k - 1) + 1:], y1[:, 8 * (k - 1) + 1:])


def test_888_model_matches_torch_fp64():
    a = SMALL8
    p = _small_params(a, seed=8)
    x = S.blurred_noise_clip(2, 1, 9, 16, 24)
    o = Oracle(a, p)
    z = o.encode_latent(x)
    h = _tconv(_t(x).permute(0, 4, 1, 2, 3), p, "enc.stem", (2, 2, 2))
    for l in range(3):
        h = _tblock(h, p, f"enc.l{l}.b0")
        if l < 2:
            h = _tconv(h, p, f"enc.down{l}", (2, 2, 2))
    zt = _tconv(_tgn(h, p, "enc.out_gn"), p, "enc.out")
    np.testing.assert_allclose(z, zt.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-9, atol=1e-9)
    codes = np.random.default_rng(5).uniform(-1, 1, z.shape)
    y = o.decode_codes(codes, 16, 24)
    assert y.shape[1] == 9
    h = _tconv(_t(codes).permute(0, 4, 1, 2, 3), p, "dec.in")
    for l in (2, 1, 0):
        h = _tblock(h, p, f"dec.l{l}.b0")
        if l > 0:
            h = _td2s(_tconv(h, p, f"dec.up{l - 1}"), (2, 2, 2))
    yt = _td2s(_tconv(_tgn(h, p, "dec.out_gn"), p, "dec.out"), (2, 2, 2))
    np.testing.assert_allclose(y, yt.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-9, atol=1e-9)


# --- BF16 activations: the oracle's rounding points against torch's bf16 casts ---

def _r16(t):
    """torch's own float32 and bfloat16 casts (round to nearest, ties to even)."""
    return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def _tblock16(x, p, name):
    h = _r16(_tconv(_r16(_tgn(x, p, name + ".gn1")), p, name + ".c1"))
    h = _tconv(_r16(_tgn(h, p, name + ".gn2")), p, name + ".c2")
    s = _r16(_tconv(x, p, name + ".sc")) if name + ".sc.w" in p else x
    return _r16(s + h)


def test_bf16_activation_model_matches_torch_bf16_casts():
    """Oracle(act_bf16=True) rounds every stored activation as an FP32 accumulator is
    stored in bf16; an independent torch FP64 build that applies torch's float32 and
    bfloat16 casts at the same points gives the same latent and frames, and both
    differ from the exact FP64 network by bf16-sized amounts."""
    a = SMALL
    p = {k: S.to_bf16_f32(v) for k, v in _small_params(a, seed=12).items()}
    x = S.to_bf16_f32(S.blurred_noise_clip(4, 1, 5, 16, 24))
    o16, o64 = Oracle(a, p, act_bf16=True), Oracle(a, p)
    z16, z64 = o16.encode_latent(x), o64.encode_latent(x)
    h = _r16(_tconv(_t(x).permute(0, 4, 1, 2, 3), p, "enc.stem", (1, 2, 2)))
    for l in range(3):
        h = _tblock16(h, p, f"enc.l{l}.b0")
        if l < 2:
            h = _r16(_tconv(h, p, f"enc.down{l}", (2, 2, 2)))
    zt = _tconv(_r16(_tgn(h, p, "enc.out_gn")), p, "enc.out").permute(0, 2, 3, 4, 1).numpy()
    np.testing.assert_allclose(z16, zt, rtol=1e-9, atol=1e-9)
    d = np.abs(z16 - z64).max() / np.abs(z64).max()
    assert 1e-5 < d < 0.05, d
    codes = np.random.default_rng(3).uniform(-1, 1, z16.shape)
    y16 = o16.decode_codes(codes, 16, 24)
    h = _r16(_tconv(_t(codes).permute(0, 4, 1, 2, 3), p, "dec.in"))
    for l in (2, 1, 0):
        h = _tblock16(h, p, f"dec.l{l}.b0")
        if l > 0:
            h = _r16(_td2s(_tconv(h, p, f"dec.up{l - 1}"), (2, 2, 2)))
    yt = _td2s(_tconv(_r16(_tgn(h, p, "dec.out_gn")), p, "dec.out"), (1, 2, 2))
    np.testing.assert_allclose(y16, yt.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-9, atol=1e-9)
