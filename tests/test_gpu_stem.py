"""The encoder stem (Sec. 2.4: causal 3x3x3 conv from the pixels, stride (t_stem, 2, 2))
in the BF16 coder, where its im2col rows are formed on chip, against the oracle on
whole clips: every output voxel, and the GroupNorm+SiLU that consumes the statistics
the stem's epilogue reduced.

The shapes reach the kernel's edges: output rows of 136 and 260 voxels (a ragged last
tile of 8 and 4 voxels after whole 128-voxel tiles), 64 and 128 channels, two
samples, temporal stride 2 (the 8x8x8 setting), frame 0's replicate padding, and a
stream whose later chunks read their first frames from the history.
Tolerances as in the other conv tests: 2^-8 |ref| + 2e-4 max|ref| (exact bf16
products, FP32 accumulation, one bf16 rounding); GN+SiLU 2^-8 |ref| + 4e-3.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import ops

pytestmark = pytest.mark.gpu

CASES = [
    # (first-level channels, t_stem, (N, T, H, W))
    (64, 1, (1, 5, 16, 272)),
    (128, 1, (2, 5, 8, 264)),
    (64, 2, (1, 9, 24, 40)),
    (128, 2, (1, 9, 16, 520)),
]


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _params(tk, seed):
    p = S.weights_for(tk.param_spec(), seed=seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.endswith(".b"):
            p[k] = (0.05 * rng.standard_normal(p[k].shape)).astype(np.float32)
        elif k.endswith(".g"):
            p[k] = (1.0 + 0.1 * rng.standard_normal(p[k].shape)).astype(np.float32)
    return p


def _traced_stem(P, c0, ts, shape, seed):
    N, T, H, W = shape
    tk = P.Tokenizer("bf16", ch=(c0, 2 * c0, 4 * c0), blocks=1, t_stem=ts)
    params = _params(tk, seed)
    tk.set_params(params)
    tk.reserve(N, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(seed, N, T, H, W))).to("cuda", torch.bfloat16)
    To = (T - 1) // ts + 1
    stem = torch.empty((N, To, H // 2, W // 2, c0), device="cuda", dtype=torch.bfloat16)
    gn_in = torch.empty_like(stem)
    gn_out = torch.empty_like(stem)
    tk.trace_layer("enc.stem", None, None, stem)
    tk.trace_layer("enc.l0.b0.gn1", gn_in, None, gn_out)
    tk.encode(x)
    torch.cuda.synchronize()
    assert tk.status() == 0
    tk.trace_layer(None)
    assert tk.check_guards() == 0
    tk.close()
    return x, params, stem, gn_in, gn_out


@pytest.mark.parametrize("c0,ts,shape", CASES)
def test_stem_whole_clip(P, c0, ts, shape):
    x, params, stem, gn_in, gn_out = _traced_stem(P, c0, ts, shape, seed=11 + c0 + ts)
    w = S.to_bf16_f32(params["enc.stem.w"]).astype(np.float64)
    ref = ops.conv3d(x.double().cpu().numpy(), w, params["enc.stem.b"].astype(np.float64), (ts, 2, 2),
                     ops.PAD_REPLICATE)
    got = stem.double().cpu().numpy()
    assert got.shape == ref.shape
    tol = 2.0 ** -8 * np.abs(ref) + 2e-4 * np.abs(ref).max()
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:4].tolist())
    # the block's first GroupNorm reads the stem output with the statistics of the
    # stem's epilogue: every frame against the oracle's statistics of that output
    assert torch.equal(gn_in, stem)
    G = ops.gn_groups(c0, 32)
    xin = gn_in.double().cpu().numpy()
    for n in range(xin.shape[0]):
        for t in range(xin.shape[1]):
            r = ops.silu(ops.group_norm_frames(xin[n:n + 1, t:t + 1], G, 1e-6, params["enc.l0.b0.gn1.g"],
                                               params["enc.l0.b0.gn1.b"]))
            g = gn_out[n:n + 1, t:t + 1].double().cpu().numpy()
            assert np.all(np.abs(g - r) <= 2.0 ** -8 * np.abs(r) + 4e-3), (n, t, float(np.abs(g - r).max()))


@pytest.mark.parametrize("ts", [1, 2])
def test_stem_stream_equals_clip(P, ts):
    """A stream's stem output, chunk by chunk (later chunks read the two frames before
    them from the history), equals the whole clip's bit for bit."""
    c0, (N, T, H, W) = 64, (1, 9, 16, 272)
    tk = P.Tokenizer("bf16", ch=(c0, 2 * c0, 4 * c0), blocks=1, t_stem=ts)
    tk.set_params(_params(tk, 5))
    tk.reserve(N, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(7, N, T, H, W))).to("cuda", torch.bfloat16)
    To = (T - 1) // ts + 1
    clip = torch.empty((N, To, H // 2, W // 2, c0), device="cuda", dtype=torch.bfloat16)
    tk.trace_layer("enc.stem", None, None, clip)
    tk.encode(x)
    st = 4 * ts
    bounds = [(0, 1)] + [(1 + st * j, 1 + st * (j + 1)) for j in range((T - 1) // st)]
    vid = tk.stream_open(H, W)
    outs = []
    for a, b in bounds:
        o = torch.empty((N, (b - a + ts - 1) // ts if a else 1, H // 2, W // 2, c0), device="cuda",
                        dtype=torch.bfloat16)
        tk.trace_layer(None)
        tk.trace_layer("enc.stem", None, None, o)
        tk.encode(x[:, a:b].contiguous(), video=vid)
        outs.append(o)
    torch.cuda.synchronize()
    assert tk.status() == 0
    tk.trace_layer(None)
    tk.stream_close(vid)
    assert tk.check_guards() == 0
    tk.close()
    assert torch.equal(torch.cat(outs, 1), clip)


def _stem_voxel(x, w, b, t, h, wv, ts):
    """Oracle value (all channels) of stem output voxel (t, h, wv) of the pixels x (a
    host array): its 3 x 3 x 3 neighbourhood of pixels (frames before 0 replicate frame 0, zeros outside the
    frame) through the oracle's conv, read at the block's causal centre."""
    _, Tn, Hn, Wn, C = x.shape
    blk = np.zeros((1, 3, 3, 3, C))
    for a in range(3):
        ti = max(0, t * ts + a - 2)
        for r in range(3):
            hh = 2 * h + r - 1
            for c in range(3):
                ww = 2 * wv + c - 1
                if 0 <= hh < Hn and 0 <= ww < Wn:
                    blk[0, a, r, c] = x[0, ti, hh, ww]
    return ops.conv3d(blk, w, b, (1, 1, 1), ops.PAD_REPLICATE)[0, 2, 1, 1]


def test_stem_1080p_sampled(P):
    """The default tokenizer's stem on a 1x3x5x1080x1920 clip: output rows of 960
    voxels (seven whole tiles and a ragged eighth of 64), 40 sampled voxels (frame 0,
    the corners, the ragged tile, random) against the oracle, and frames 0 and 4 of
    the GroupNorm+SiLU fed by the stem's statistics against the oracle's."""
    T, H, W = 5, 1080, 1920
    tk = P.Tokenizer("bf16")
    params = _params(tk, 3)
    tk.set_params(params)
    tk.reserve(1, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(21, 1, T, H, W))).to("cuda", torch.bfloat16)
    stem = torch.empty((1, T, H // 2, W // 2, 128), device="cuda", dtype=torch.bfloat16)
    gn_out = torch.empty_like(stem)
    tk.trace_layer("enc.stem", None, None, stem)
    tk.trace_layer("enc.l0.b0.gn1", None, None, gn_out)
    tk.encode(x, want_z=False)
    torch.cuda.synchronize()
    assert tk.status() == 0
    tk.trace_layer(None)
    assert tk.check_guards() == 0
    tk.close()
    w = S.to_bf16_f32(params["enc.stem.w"]).astype(np.float64)
    b = params["enc.stem.b"].astype(np.float64)
    Ho, Wo = H // 2, W // 2
    rng = np.random.default_rng(4)
    pts = [(0, 0, 0), (0, Ho - 1, Wo - 1), (T - 1, 0, Wo - 1), (T - 1, Ho - 1, 0), (2, 100, 896), (3, 17, 959)]
    while len(pts) < 40:
        pts.append((int(rng.integers(0, T)), int(rng.integers(0, Ho)), int(rng.integers(0, Wo))))
    xc = x.double().cpu().numpy()
    ref = np.stack([_stem_voxel(xc, w, b, t, h, wv, 1) for t, h, wv in pts])
    got = np.stack([stem[0, t, h, wv].double().cpu().numpy() for t, h, wv in pts])
    tol = 2.0 ** -8 * np.abs(ref) + 2e-4 * np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= tol), float((np.abs(got - ref) / tol).max())
    G = ops.gn_groups(128, 32)
    for t in (0, T - 1):
        xin = stem[:, t:t + 1].double().cpu().numpy()
        r = ops.silu(ops.group_norm_frames(xin, G, 1e-6, params["enc.l0.b0.gn1.g"], params["enc.l0.b0.gn1.b"]))
        g = gn_out[:, t:t + 1].double().cpu().numpy()
        assert np.all(np.abs(g - r) <= 2.0 ** -8 * np.abs(r) + 4e-3), (t, float(np.abs(g - r).max()))
