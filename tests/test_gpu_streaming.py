"""Chunked streaming equals the whole clip, bitwise (the conv caches carry the
causal left context across chunks; GoP-style segment coding of Sec. 4.2/4.3).

Chunk 0 is frame 0 (latent 0); chunk k >= 1 is frames s(k-1)+1..sk (latent k),
s = 4 frames per latent frame (8 with the temporal-stride-2 stem). Decoding
latent k of a stream gives frame 0 (k = 0) or frames s(k-1)+1..sk.
Every convolution computes each output with the same sequence of tensor-core
(or FMA) operations whatever frames share its launch, and GroupNorm's
per-frame reduction order does not depend on the frame count, so the
concatenated chunk outputs must equal the clip outputs exactly.
"""
import numpy as np
import pytest
import torch

from paper_2602_03529_b300 import _lib as _L

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _run(P, prec, kw, T, H, W, seed=0):
    tk = P.Tokenizer(prec, **kw)
    tk.set_params(S.weights_for(tk.param_spec(), seed=seed))
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    x = torch.from_numpy(S.moving_rects_clip(seed, T, H, W)[None]).to("cuda", dt)
    tk.reserve(1, T, H, W)
    z_c, idx_c = tk.encode(x)
    xh_c = tk.decode(idx_c, H, W)
    vid = tk.stream_open(H, W)
    assert tk.stream_bytes(H, W) > 0
    st = tk.s_t
    bounds = [(0, 1)] + [(st * (k - 1) + 1, st * k + 1) for k in range(1, (T - 1) // st + 1)]
    zs, ids = [], []
    for a, b in bounds:
        z, idx = tk.encode(x[:, a:b].contiguous(), video=vid)
        zs.append(z)
        ids.append(idx)
    xs = [tk.decode(idx, H, W, video=vid, first_chunk=(k == 0)) for k, idx in enumerate(ids)]
    torch.cuda.synchronize()
    assert tk.status() == 0
    assert _L.tok_stream_check_guards(vid) == 0
    tk.stream_close(vid)
    out = dict(z=(torch.cat(zs, 1), z_c), idx=(torch.cat(ids, 1), idx_c), x=(torch.cat(xs, 1), xh_c))
    assert tk.check_guards() == 0
    tk.close()
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("pad", ["replicate", "zero"])
def test_stream_equals_clip_small(P, prec, pad):
    out = _run(P, prec, dict(ch=(64, 128, 256), blocks=1, time_pad=pad), 13, 40, 56, seed=3)
    for k, (s, c) in out.items():
        assert s.shape == c.shape, k
        assert torch.equal(s, c), (k, float((s.float() - c.float()).abs().max()))


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("pad", ["replicate", "zero"])
def test_stream_equals_clip_8x8x8(P, prec, pad):
    """8 frames per chunk: the stem's stride-2 taps reach one frame back into the cache."""
    out = _run(P, prec, dict(ch=(64, 128, 256), blocks=1, time_pad=pad, t_stem=2), 25, 40, 56, seed=6)
    for k, (s, c) in out.items():
        assert s.shape == c.shape, k
        assert torch.equal(s, c), (k, float((s.float() - c.float()).abs().max()))


def test_stream_equals_clip_default_bf16(P):
    out = _run(P, "bf16", {}, 9, 64, 96, seed=4)
    for k, (s, c) in out.items():
        assert torch.equal(s, c), k


def test_stream_rejects_wrong_chunk_sizes(P):
    from paper_2602_03529_b300 import _lib as L
    tk = P.Tokenizer("bf16", ch=(64, 128, 256), blocks=1)
    vid = tk.stream_open(32, 32)
    x4 = torch.zeros((1, 4, 32, 32, 3), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(L.TokError) as e:
        tk.encode(x4, video=vid)           # the first chunk must be one frame
    assert e.value.code == L.TOK_ESHAPE
    tk.encode(x4[:, :1].contiguous(), video=vid)
    with pytest.raises(L.TokError):
        tk.encode(x4[:, :1].contiguous(), video=vid)  # later chunks are 4 frames
    tk.stream_reset(vid)
    tk.encode(x4[:, :1].contiguous(), video=vid)      # after a reset: a new first chunk
    torch.cuda.synchronize()
    assert _L.tok_stream_check_guards(vid) == 0
    tk.stream_close(vid)
    assert tk.check_guards() == 0
    tk.close()
