"""Grouped launches: one conv / GroupNorm launch per layer over inputs of
different sizes (clips of several resolutions, chunks of several streams).

A tile never spans two inputs and every tile is computed by the same sequence
of operations as in a launch of its input alone, and the GroupNorm chunking of
a frame depends on the frame's size only, so each item of a batch must equal
its own single call bitwise: latents, indices and reconstructions. The single
calls are pinned to the FP64 oracle by the model tests.
"""
import numpy as np
import pytest
import torch

from paper_2602_03529_b300 import _lib as _L

import synthetic as S

pytestmark = pytest.mark.gpu

# (N, T, H, W): ragged widths (not multiples of 8), several frame counts and a
# batch of 2, so tiles are ragged and the problems have different tile counts
SHAPES = [(1, 9, 64, 96), (1, 5, 40, 56), (2, 5, 48, 60), (1, 13, 32, 32)]


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _tok(P, prec, seed=5, **kw):
    kw = dict(dict(ch=(64, 128, 256), blocks=1), **kw)
    tk = P.Tokenizer(prec, **kw)
    tk.set_params(S.weights_for(tk.param_spec(), seed=seed))
    return tk


def _clips(prec, shapes):
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    return [torch.from_numpy(S.moving_rects_clip(10 + i, T, H, W)[None].repeat(N, 0)).to("cuda", dt)
            for i, (N, T, H, W) in enumerate(shapes)]


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_batch_equals_single_calls(P, prec):
    tk = _tok(P, prec)
    xs = _clips(prec, SHAPES)
    tk.reserve_batch(SHAPES)
    zb, ib = tk.encode_batch(xs)
    xb = tk.decode_batch(ib, [(H, W) for (_, _, H, W) in SHAPES])
    torch.cuda.synchronize()
    assert tk.status() == 0
    for i, (x, (N, T, H, W)) in enumerate(zip(xs, SHAPES)):
        z1, i1 = tk.encode(x)
        x1 = tk.decode(i1, H, W)
        torch.cuda.synchronize()
        assert torch.equal(zb[i], z1), i
        assert torch.equal(ib[i], i1), i
        assert torch.equal(xb[i], x1), i
    assert tk.status() == 0
    assert tk.check_guards() == 0
    tk.close()


def test_batch_of_one_equals_single_call(P):
    tk = _tok(P, "bf16")
    (x,) = _clips("bf16", SHAPES[:1])
    _, _, H, W = SHAPES[0]
    tk.reserve(*SHAPES[0])
    z1, i1 = tk.encode(x)
    (zb,), (ib,) = tk.encode_batch([x])
    torch.cuda.synchronize()
    assert torch.equal(z1, zb) and torch.equal(i1, ib)
    assert tk.check_guards() == 0
    tk.close()


def test_streams_in_mixed_batches_equal_streams_alone(P):
    """Three streams of different sizes; at every step the ready subset of
    streams (plus a whole clip) goes through one batch. Each stream's chunk
    outputs equal those of the same stream advanced on its own."""
    tk = _tok(P, "bf16")
    sizes = [(40, 56), (32, 48), (24, 40)]
    T = 9
    clips = [torch.from_numpy(S.moving_rects_clip(20 + i, T, H, W)[None]).to("cuda", torch.bfloat16)
             for i, (H, W) in enumerate(sizes)]
    bounds = [(0, 1), (1, 5), (5, 9)]
    shapes = [(1, tk.s_t, H, W) for (H, W) in sizes] + [(1, 5, 40, 56)]
    tk.reserve_batch(shapes)
    # alone
    alone = []
    for (H, W), x in zip(sizes, clips):
        v = tk.stream_open(H, W)
        ids, xs = [], []
        for k, (a, b) in enumerate(bounds):
            _, idx = tk.encode(x[:, a:b].contiguous(), video=v)
            ids.append(idx)
            xs.append(tk.decode(idx, H, W, video=v, first_chunk=(k == 0)))
        assert _L.tok_stream_check_guards(v) == 0
        tk.stream_close(v)
        alone.append((torch.cat(ids, 1), torch.cat(xs, 1)))
    # batched: stream 2 starts one step late, and a clip rides along in step 1
    vids = [tk.stream_open(H, W) for (H, W) in sizes]
    extra = _clips("bf16", [(1, 5, 40, 56)])[0]
    start = [0, 0, 1]
    got = [([], []) for _ in sizes]
    for step in range(4):
        act = [i for i in range(3) if 0 <= step - start[i] < len(bounds)]
        xs_in, vs, ks = [], [], []
        for i in act:
            a, b = bounds[step - start[i]]
            xs_in.append(clips[i][:, a:b].contiguous())
            vs.append(vids[i])
            ks.append(step - start[i])
        if step == 1:
            xs_in.append(extra)
            vs.append(None)
        _, ids = tk.encode_batch(xs_in, videos=vs)
        n = len(act)
        outs = tk.decode_batch(ids[:n], [sizes[i] for i in act], videos=vs[:n], first_chunks=[k == 0 for k in ks])
        for j, i in enumerate(act):
            got[i][0].append(ids[j])
            got[i][1].append(outs[j])
    torch.cuda.synchronize()
    assert tk.status() == 0
    for i in range(3):
        assert torch.equal(torch.cat(got[i][0], 1), alone[i][0]), i
        assert torch.equal(torch.cat(got[i][1], 1), alone[i][1]), i
    for v in vids:
        assert _L.tok_stream_check_guards(v) == 0
        tk.stream_close(v)
    assert tk.check_guards() == 0
    tk.close()


def test_batch_argument_errors(P):
    from paper_2602_03529_b300 import _lib as L
    tk = _tok(P, "bf16")
    x = _clips("bf16", [(1, 5, 32, 32)])[0]
    tk.reserve(1, 5, 32, 32)
    with pytest.raises(L.TokError) as e:
        tk.encode_batch([x] * (L.TOK_MAX_BATCH + 1))
    assert e.value.code == L.TOK_EINVAL
    # the same stream twice in one batch
    v = tk.stream_open(32, 32)
    x0 = x[:, :1].contiguous()
    with pytest.raises(L.TokError) as e:
        tk.encode_batch([x0, x0], videos=[v, v])
    assert e.value.code == L.TOK_EINVAL
    # workspace for one clip, not for three
    big = _clips("bf16", [(1, 5, 256, 256)])[0]
    with pytest.raises(L.TokError) as e:
        tk.encode_batch([big, big, big])
    assert e.value.code == L.TOK_ENOMEM
    torch.cuda.synchronize()
    assert tk.status() == 0
    assert _L.tok_stream_check_guards(v) == 0
    tk.stream_close(v)
    assert tk.check_guards() == 0
    tk.close()


@pytest.mark.parametrize("tiles", [1, 3])
def test_short_lived_ctas_give_the_same_result(P, tiles):
    """Conv CTAs of at most `tiles` tiles (a context that yields SMs to higher-priority
    work) compute every tile exactly as the persistent CTAs do."""
    tk = _tok(P, "bf16")
    xs = _clips("bf16", SHAPES[:2])
    tk.reserve_batch(SHAPES[:2])
    zr, ir = tk.encode_batch(xs)
    xr = tk.decode_batch(ir, [(H, W) for (_, _, H, W) in SHAPES[:2]])
    tk.set_cta_tiles(tiles)
    zt, it = tk.encode_batch(xs)
    xt = tk.decode_batch(it, [(H, W) for (_, _, H, W) in SHAPES[:2]])
    torch.cuda.synchronize()
    assert tk.status() == 0
    for a, b in zip(zr + ir + xr, zt + it + xt):
        assert torch.equal(a, b)
    assert tk.check_guards() == 0
    tk.close()
