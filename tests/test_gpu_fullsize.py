"""Parity at the full 720p workload (1 x 3 x 17 x 720 x 1280, channels
128/256/512), in the launch configuration the benchmark times.

The whole network cannot be run by the FP64 oracle at this size, and
GroupNorm statistics span a whole frame, so a crop of the clip does not
reproduce an interior output. Instead:
  * every kernel form the network uses is run at its full-size shape and
    checked on sampled outputs the oracle computes one by one: a conv output
    voxel from its 3 x 3 x 3 input neighbourhood (frame 0, the frame edges and
    the ragged last tile row included), a GroupNorm+SiLU frame in full;
  * the whole coder is checked for properties that hold at any size:
    determinism, causality (frames after t do not change the latents up to
    t) and streaming equal to the whole clip, bit for bit.
Tolerances as in the per-kernel tests: conv 2^-8 |ref| + 2e-4 max|ref| (exact
bf16 products, FP32 accumulation, one bf16 rounding); GN+SiLU 2^-8 |ref| + 4e-3.
"""
import zlib

import numpy as np
import pytest
import torch

from paper_2602_03529_b300 import _lib as _L

import synthetic as S
from oracle import ops

pytestmark = pytest.mark.gpu
T, H, W = 17, 720, 1280


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _sample_voxels(rng, To, Ho, Wo, n):
    pts = [(0, 0, 0), (0, Ho - 1, Wo - 1), (1, Ho - 1, 0), (To - 1, 0, Wo - 1), (To - 1, Ho // 2, Wo // 2)]
    while len(pts) < n:
        pts.append((int(rng.integers(0, To)), int(rng.integers(0, Ho)), int(rng.integers(0, Wo))))
    return pts


def _conv_at(x, w, b, res, t, h, wv, pad):
    """Oracle value of one output voxel of a stride-1 3x3x3 causal conv (all Cout), from
    its input neighbourhood (x: CPU bf16 tensor)."""
    _, Tn, Hn, Wn, _ = x.shape
    t0, h0, w0 = max(0, t - 2), max(0, h - 1), max(0, wv - 1)
    crop = x[:, t0:t + 1, h0:min(Hn, h + 2), w0:min(Wn, wv + 2)].double().numpy()
    y = ops.conv3d(crop, w, b, (1, 1, 1), pad)
    v = y[0, t - t0, h - h0, wv - w0]
    return v + (res[0, t, h, wv].double().numpy() if res is not None else 0.0)


def _bf16_normal(shape, seed, scale=1.0, shift=0.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale + shift).to(torch.bfloat16)


@pytest.mark.parametrize("level", [0, 1, 2, "2@1080p"])
def test_conv_full_size_sampled(P, level):
    """The level-0 (128 -> 128 channels at 17 x 360 x 640), level-1 (256 -> 256 at
    9 x 180 x 320) and level-2 (512 -> 512 at 5 x 90 x 160, 7 x 32 tiles; and at 1080p,
    5 x 135 x 240, 15 x 16 tiles) residual-block convs with their residual add, in the
    swapped halo form."""
    shapes = {0: (T, H // 2, W // 2, 128), 1: (9, H // 4, W // 4, 256), 2: (5, H // 8, W // 8, 512),
              "2@1080p": (5, 135, 240, 512)}
    Tl, Hl, Wl, C = shapes[level]
    level = {"2@1080p": 3}.get(level, level)
    rng = np.random.default_rng(20 + level)
    x = _bf16_normal((1, Tl, Hl, Wl, C), 40 + level)
    res = _bf16_normal((1, Tl, Hl, Wl, C), 50 + level)
    w = S.to_bf16_f32((rng.standard_normal((C, 3, 3, 3, C)) * np.sqrt(2.0 / (27 * C))).astype(np.float32))
    b = (rng.standard_normal(C) * 0.1).astype(np.float32)
    y = P.conv3d(x.cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda(), (1, 1, 1), "replicate",
                 residual=res.cuda())
    torch.cuda.synchronize()
    pts = _sample_voxels(rng, Tl, Hl, Wl, 48)
    got = np.stack([y[0, t, h, wv].float().cpu().numpy() for t, h, wv in pts]).astype(np.float64)
    ref = np.stack([_conv_at(x, w, b, res, t, h, wv, ops.PAD_REPLICATE) for t, h, wv in pts])
    tol = 2.0 ** -8 * np.abs(ref) + 2e-4 * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= tol), float((np.abs(got - ref) / tol).max())


def test_groupnorm_full_size_sampled_frames(P):
    """GroupNorm(32) + SiLU of a 17 x 360 x 640 x 128 activation; frames 0, 8, 16 in full."""
    rng = np.random.default_rng(31)
    x = _bf16_normal((1, T, H // 2, W // 2, 128), 33, 0.7, 0.2)
    ga = (1 + 0.1 * rng.standard_normal(128)).astype(np.float32)
    be = (0.1 * rng.standard_normal(128)).astype(np.float32)
    y = P.groupnorm_silu(x.cuda(), 32, torch.from_numpy(ga).cuda(), torch.from_numpy(be).cuda())
    torch.cuda.synchronize()
    for t in (0, 8, 16):
        ref = ops.silu(ops.group_norm_frames(x[:, t:t + 1].double().numpy(), 32, 1e-6, ga, be))
        got = y[:, t:t + 1].float().cpu().numpy().astype(np.float64)
        tol = 2.0 ** -8 * np.abs(ref) + 4e-3
        assert np.all(np.abs(got - ref) <= tol), (t, float(np.abs(got - ref).max()))


@pytest.fixture(scope="module")
def coder(P):
    tk = P.Tokenizer("bf16")
    tk.set_params(S.weights_for(tk.param_spec(), seed=0))
    tk.reserve(1, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(1000, 1, T, H, W))).to("cuda", torch.bfloat16)
    yield tk, x
    assert tk.check_guards() == 0
    tk.close()


def test_full_size_deterministic_and_valid(P, coder):
    tk, x = coder
    z1, i1 = tk.encode(x)
    x1 = tk.decode(i1, H, W)
    z2, i2 = tk.encode(x)
    x2 = tk.decode(i2, H, W)
    torch.cuda.synchronize()
    assert tk.status() == 0
    assert i1.shape == (1, 5, 90, 160) and x1.shape == (1, T, H, W, 3)
    assert torch.equal(z1, z2) and torch.equal(i1, i2) and torch.equal(x1, x2)
    assert int(i1.min()) >= 0 and int(i1.max()) < 64000
    assert torch.isfinite(x1).all()


def test_full_size_causal(P, coder):
    """Changing frames 13..16 (latent 4) leaves latents 0..3 and decoded frames 0..12 unchanged."""
    tk, x = coder
    z1, i1 = tk.encode(x)
    x2 = x.clone()
    x2[:, 13:] = -x2[:, 13:]
    z2, i2 = tk.encode(x2)
    d1 = tk.decode(i1, H, W)
    d2 = tk.decode(i2, H, W)
    torch.cuda.synchronize()
    assert torch.equal(z1[:, :4], z2[:, :4]) and torch.equal(i1[:, :4], i2[:, :4])
    assert not torch.equal(z1[:, 4], z2[:, 4])
    assert torch.equal(d1[:, :13], d2[:, :13])


def test_full_size_stream_equals_clip(P, coder):
    """The 720p clip coded as a stream of chunks (frame 0, then 4 frames at a time)."""
    tk, x = coder
    z_c, i_c = tk.encode(x)
    x_c = tk.decode(i_c, H, W)
    vid = tk.stream_open(H, W)
    zs, ids, xs = [], [], []
    for k, (a, b) in enumerate([(0, 1)] + [(4 * j - 3, 4 * j + 1) for j in range(1, 5)]):
        z, i = tk.encode(x[:, a:b].contiguous(), video=vid)
        zs.append(z)
        ids.append(i)
        xs.append(tk.decode(i, H, W, video=vid, first_chunk=(k == 0)))
    torch.cuda.synchronize()
    assert _L.tok_stream_check_guards(vid) == 0
    tk.stream_close(vid)
    assert torch.equal(torch.cat(zs, 1), z_c)
    assert torch.equal(torch.cat(ids, 1), i_c)
    assert torch.equal(torch.cat(xs, 1), x_c)


# ------------------------------------------------ every layer form of the 720p step
#
# The coder of the benchmark (default tokenizer, 1 x 3 x 17 x 720 x 1280, BF16,
# persistent conv CTAs, the tile shapes the benchmark's launches choose) is run
# once with layer traces armed; each traced layer is then compared with the
# oracle on its own traced input, so that every check isolates one launch.
# Biases and GroupNorm affine parameters are drawn non-zero for these checks.

ENC_TRACE = ["enc.stem", "enc.l0.b0.gn1", "enc.l0.b0.c1", "enc.l0.b1.c2", "enc.down0", "enc.l1.b0.sc",
             "enc.l1.b0.c2", "enc.down1", "enc.l2.b0.sc", "enc.l2.b0.c1", "enc.out_gn", "enc.out"]
DEC_TRACE = ["dec.in", "dec.l2.b0.c2", "dec.up1", "dec.l1.b0.gn1", "dec.l1.b1.c1", "dec.up0", "dec.l0.b0.gn1",
             "dec.l0.b1.c2", "dec.out"]
# layer -> (input shape, output shape, residual?, kernel size, stride (t, h, w)); None: not traced
_L0, _L1, _L2 = (T, H // 2, W // 2), (9, H // 4, W // 4), (5, H // 8, W // 8)
LAYER = {
    "enc.stem": (None, _L0 + (128,), False, 3, (1, 2, 2)),
    "enc.l0.b0.gn1": (_L0 + (128,), _L0 + (128,), False, 0, None),
    "enc.l0.b0.c1": (_L0 + (128,), _L0 + (128,), False, 3, (1, 1, 1)),
    "enc.l0.b1.c2": (_L0 + (128,), _L0 + (128,), True, 3, (1, 1, 1)),
    "enc.down0": (_L0 + (128,), _L1 + (128,), False, 3, (2, 2, 2)),
    "enc.l1.b0.sc": (_L1 + (128,), _L1 + (256,), False, 1, (1, 1, 1)),
    "enc.l1.b0.c2": (_L1 + (256,), _L1 + (256,), True, 3, (1, 1, 1)),
    "enc.down1": (_L1 + (256,), _L2 + (256,), False, 3, (2, 2, 2)),
    "enc.l2.b0.sc": (_L2 + (256,), _L2 + (512,), False, 1, (1, 1, 1)),
    "enc.l2.b0.c1": (_L2 + (256,), _L2 + (512,), False, 3, (1, 1, 1)),
    "enc.out_gn": (_L2 + (512,), _L2 + (512,), False, 0, None),
    "enc.out": (_L2 + (512,), None, False, 3, (1, 1, 1)),
    "dec.in": (None, _L2 + (512,), False, 3, (1, 1, 1)),
    "dec.l2.b0.c2": (_L2 + (512,), _L2 + (512,), True, 3, (1, 1, 1)),
    "dec.up1": (_L2 + (512,), _L1 + (256,), False, 3, (1, 1, 1)),
    "dec.l1.b0.gn1": (_L1 + (256,), _L1 + (256,), False, 0, None),
    "dec.l1.b1.c1": (_L1 + (256,), _L1 + (256,), False, 3, (1, 1, 1)),
    "dec.up0": (_L1 + (256,), _L0 + (128,), False, 3, (1, 1, 1)),
    "dec.l0.b0.gn1": (_L0 + (128,), _L0 + (128,), False, 0, None),
    "dec.l0.b1.c2": (_L0 + (128,), _L0 + (128,), True, 3, (1, 1, 1)),
    "dec.out": (_L0 + (128,), None, False, 3, (1, 1, 1)),
}


def _perturbed_params(tk):
    """He-normal weights (seed 0) with non-zero biases and GroupNorm affine terms."""
    p = S.weights_for(tk.param_spec(), seed=0)
    rng = np.random.default_rng(77)
    for k in p:
        if k.endswith(".b"):
            p[k] = (0.05 * rng.standard_normal(p[k].shape)).astype(np.float32)
        elif k.endswith(".g"):
            p[k] = (1.0 + 0.1 * rng.standard_normal(p[k].shape)).astype(np.float32)
    return p


@pytest.fixture(scope="module")
def traced(P):
    tk = P.Tokenizer("bf16")
    params = _perturbed_params(tk)
    tk.set_params(params)
    tk.reserve(1, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(1000, 1, T, H, W))).to("cuda", torch.bfloat16)
    bufs = {}
    for name in ENC_TRACE + DEC_TRACE:
        ish, osh, has_res, _, _ = LAYER[name]
        b = {"in": None if ish is None else torch.empty((1,) + ish, device="cuda", dtype=torch.bfloat16),
             "out": None if osh is None else torch.empty((1,) + osh, device="cuda", dtype=torch.bfloat16)}
        b["res"] = torch.empty_like(b["out"]) if has_res else None
        tk.trace_layer(name, b["in"], b["res"], b["out"])
        bufs[name] = b
    z, idx = tk.encode(x)
    xh = tk.decode(idx, H, W)
    torch.cuda.synchronize()
    assert tk.status() == 0
    tk.trace_layer(None)
    oracle_p = {k: (S.to_bf16_f32(v) if k.endswith(".w") else v).astype(np.float64) for k, v in params.items()}
    yield {"x": x, "z": z, "idx": idx, "xh": xh, "bufs": bufs, "p": oracle_p}
    assert tk.check_guards() == 0
    tk.close()


def _block(fetch, shape, t, h, w, k, stride):
    """The k x k x k input neighbourhood of output voxel (t, h, w) of a causal conv
    (frames before 0 replicate frame 0, zeros outside the frame), as a
    (1, k, k, k, C) float64 block: the oracle's conv of the block gives that voxel
    at block position (k-1, (k-1)//2, (k-1)//2)."""
    Tn, Hn, Wn, C = shape
    st, sh, sw = stride
    ti = [max(0, t * st + d - (k - 1)) for d in range(k)]
    hi = [h * sh + d - (k - 1) // 2 for d in range(k)]
    wi = [w * sw + d - (k - 1) // 2 for d in range(k)]
    h0, h1 = max(0, min(hi)), min(Hn, max(hi) + 1)
    w0, w1 = max(0, min(wi)), min(Wn, max(wi) + 1)
    crop = fetch(min(ti), max(ti) + 1, h0, h1, w0, w1)
    blk = np.zeros((1, k, k, k, C))
    for a, tt in enumerate(ti):
        for b, hh in enumerate(hi):
            for c, ww in enumerate(wi):
                if 0 <= hh < Hn and 0 <= ww < Wn:
                    blk[0, a, b, c] = crop[tt - min(ti), hh - h0, ww - w0]
    return blk


def _gpu_fetch(x):
    return lambda t0, t1, h0, h1, w0, w1: x[0, t0:t1, h0:h1, w0:w1].double().cpu().numpy()


def _oracle_voxel(p, name, blk, k):
    c = (k - 1) // 2
    return ops.conv3d(blk, p[name + ".w"], p[name + ".b"], (1, 1, 1), ops.PAD_REPLICATE)[0, k - 1, c, c]


def _check(got, ref, rel, what):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    tol = rel * np.abs(ref) + 2e-4 * np.abs(ref).max()
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (what, int(bad.sum()), float((np.abs(got - ref) / tol).max()))


@pytest.mark.parametrize("name", [n for n in ENC_TRACE + DEC_TRACE if LAYER[n][3] in (1, 3)])
def test_network_conv_layer_sampled(traced, name):
    """One conv launch of the 720p step against the oracle on 40 sampled output voxels
    (frame 0, the frame corners and random voxels), computed from the layer's own
    traced input: plain, residual, stride-2 (parity view), 1x1x1, the stem over its
    im2col matrix (from the pixels), the decoder input (from the token indices), the
    up convs with depth-to-space, the latent head (z; FSQ indices in the next test)
    and the pixel head (depth-to-space, fp32, crop)."""
    ish, osh, has_res, k, stride = LAYER[name]
    b, p = traced["bufs"][name], traced["p"]
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    d2s = name.startswith("dec.up") or name == "dec.out"
    if name == "enc.stem":
        xin = traced["x"]
        fetch, in_shape = _gpu_fetch(xin), tuple(xin.shape[1:])
    elif name == "dec.in":
        codes = ops.fsq_dequantize(traced["idx"].cpu().numpy().astype(np.int64), LEVELS)
        fetch = lambda t0, t1, h0, h1, w0, w1: codes[0, t0:t1, h0:h1, w0:w1]  # noqa: E731
        in_shape = codes.shape[1:]
    else:
        fetch, in_shape = _gpu_fetch(b["in"]), ish
    Ti, Hi, Wi = in_shape[:3]
    To, Ho, Wo = (Ti - 1) // stride[0] + 1, (Hi - 1) // stride[1] + 1, (Wi - 1) // stride[2] + 1
    got, ref = [], []
    for t, h, w in _sample_voxels(rng, To, Ho, Wo, 40):
        v = _oracle_voxel(p, name, _block(fetch, in_shape, t, h, w, k, stride), k)
        if name == "enc.out":
            ref.append(v)
            got.append(traced["z"][0, t, h, w].double().cpu().numpy())
        elif d2s:
            rt = 2 if name.startswith("dec.up") else 1
            sub = ops.depth_to_space(v.reshape(1, 1, 1, 1, -1), (rt, 2, 2), drop_first=0)[0]
            out = b["out"] if name.startswith("dec.up") else traced["xh"]
            for a in range(rt):
                ot = t * rt + a - (rt - 1)
                if ot < 0:
                    continue
                ref.append(sub[a])
                got.append(out[0, ot, 2 * h:2 * h + 2, 2 * w:2 * w + 2].double().cpu().numpy())
        else:
            if has_res:
                v = v + b["res"][0, t, h, w].double().cpu().numpy()
            ref.append(v)
            got.append(b["out"][0, t, h, w].double().cpu().numpy())
    fp32_out = name in ("enc.out", "dec.out")
    _check(np.stack(got), np.stack(ref), 2.0 ** -20 if fp32_out else 2.0 ** -8, name)


LEVELS = (8, 8, 8, 5, 5, 5)


def test_network_latent_head_fsq_indices(traced):
    """The FSQ epilogue of the latent head at 720p (5 x 90 x 160 tokens): the oracle's FSQ
    of the GPU's own z gives the GPU's index at every token outside 2^-16 of a rounding
    tie (the epilogue takes the rounding of the exact bounded value, by thresholds on
    z), and the mismatches inside that band stay under 1e-4 of the tokens."""
    z = traced["z"].double().cpu().numpy()
    idx = traced["idx"].cpu().numpy()
    ref, _, bnd = ops.fsq_quantize(z, LEVELS)
    tie = (np.abs((bnd - np.floor(bnd)) - 0.5) <= 2.0 ** -16).any(-1)
    assert not np.any((idx != ref) & ~tie)
    assert np.mean((idx != ref) & tie) < 1e-4


@pytest.mark.parametrize("name", [n for n in ENC_TRACE + DEC_TRACE if LAYER[n][3] == 0])
def test_network_groupnorm_layer_frames(traced, name):
    """GroupNorm+SiLU inside the 720p step, statistics reduced by the producing conv's
    epilogue (plain or depth-to-space tiles, merged per frame): three whole frames
    against the oracle on the layer's traced input."""
    b, p = traced["bufs"][name], traced["p"]
    C = b["in"].shape[-1]
    G = ops.gn_groups(C, 32)
    Tn = b["in"].shape[1]
    for t in (0, Tn // 2, Tn - 1):
        xin = b["in"][:, t:t + 1].double().cpu().numpy()
        ref = ops.silu(ops.group_norm_frames(xin, G, 1e-6, p[name + ".g"], p[name + ".b"]))
        got = b["out"][:, t:t + 1].double().cpu().numpy()
        tol = 2.0 ** -8 * np.abs(ref) + 4e-3
        assert np.all(np.abs(got - ref) <= tol), (name, t, float(np.abs(got - ref).max()))
