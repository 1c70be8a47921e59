"""GoP boundary smoothing (Eq. 1, 2) on the GPU against the FP64 oracle.

Blending is a fixed convex combination per frame (float32 on the GPU: error
within a few float32 ulps of the values); the loss sums squares in FP64 in a
fixed order (relative 1e-6), and its gradient is d/(N n ||d||) in float32
(relative 1e-5 per element)."""
import numpy as np
import pytest
import torch

from oracle import ops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


@pytest.mark.parametrize("shape,Tp,n", [((2, 9, 16, 24, 3), 9, 4), ((1, 5, 7, 9, 3), 8, 5), ((3, 4, 720, 1280, 3), 4, 2),
                                         ((1, 6, 5, 5, 3), 6, 0)])
def test_blend(P, shape, Tp, n):
    rng = np.random.default_rng(n + Tp)
    N, T, H, W, C = shape
    prev = rng.uniform(-1, 1, (N, Tp, H, W, C)).astype(np.float32)
    curr = rng.uniform(-1, 1, shape).astype(np.float32)
    out = P.gop_blend(torch.from_numpy(prev).cuda(), torch.from_numpy(curr).cuda(), n)
    inplace = torch.from_numpy(curr).cuda()
    P.gop_blend(torch.from_numpy(prev).cuda(), inplace, n, out=inplace)
    torch.cuda.synchronize()
    ref = ops.gop_blend(prev, curr, n)
    assert np.abs(out.cpu().numpy() - ref).max() <= 4e-7
    assert torch.equal(out, inplace)


@pytest.mark.parametrize("shape,Tp,n", [((2, 9, 16, 24, 3), 9, 4), ((1, 5, 7, 9, 3), 8, 5), ((2, 4, 360, 640, 3), 6, 3)])
def test_temporal_loss(P, shape, Tp, n):
    rng = np.random.default_rng(Tp)
    N, T, H, W, C = shape
    xp = rng.uniform(-1, 1, (N, Tp, H, W, C)).astype(np.float32)
    xc = rng.uniform(-1, 1, shape).astype(np.float32)
    xc[0, 0] = xp[0, Tp - n]                         # one zero difference: zero gradient there
    loss, g = P.temporal_loss(torch.from_numpy(xc).cuda(), torch.from_numpy(xp).cuda(), n)
    torch.cuda.synchronize()
    L, gref = ops.temporal_loss(xc, xp, n)
    assert abs(float(loss.item()) - L) <= 1e-6 * L
    gg = g.cpu().numpy()
    assert np.abs(gg - gref).max() <= 1e-5 * np.abs(gref).max()
    assert not gg[0, 0].any() and not gg[:, n:].any()


@pytest.mark.parametrize("prec,kw,shape,n", [
    ("bf16", dict(ch=(64, 128, 256), blocks=1), (1, 9, 40, 56), 4),         # pixel head: dw-rows form
    ("bf16", dict(ch=(64, 128, 256), blocks=1, t_stem=2), (2, 9, 24, 40), 8),  # 8x8x8: (2,2,2) pixel head
    ("fp32", dict(ch=(64, 128, 256), blocks=1), (1, 5, 24, 36), 3),          # CUDA-core path
    ("bf16", dict(ch=(64, 128, 256), blocks=1), (1, 5, 24, 40), 0),          # no blend
])
def test_decode_with_fused_boundary_blend(P, prec, kw, shape, n):
    """tok_decode_gop (Eq. 2 in the pixel head's epilogue) gives bit for bit what
    tok_decode followed by the stand-alone blend gives, and that blend matches the
    oracle's Eq. 2 on the decoded frames; frames after the first n are the plain
    decode."""
    import synthetic as S
    N, T, H, W = shape
    tk = P.Tokenizer(prec, **kw)
    tk.set_params(S.weights_for(tk.param_spec(), seed=2))
    Tq, Hq, Wq = tk.latent_shape(T, H, W)
    idx = torch.from_numpy(np.random.default_rng(7).integers(0, 64000, (N, Tq, Hq, Wq)).astype(np.int32)).cuda()
    Tp = T + 2
    prev = torch.from_numpy(np.random.default_rng(8).uniform(-1, 1, (N, Tp, H, W, 3)).astype(np.float32)).cuda()
    tk.reserve(N, T, H, W)
    plain = tk.decode(idx, H, W)
    fused = tk.decode_gop(idx, H, W, prev, n)
    two_pass = P.gop_blend(prev, plain, n)
    torch.cuda.synchronize()
    assert tk.status() == 0
    assert torch.equal(fused, two_pass)
    assert torch.equal(fused[:, n:], plain[:, n:])
    ref = ops.gop_blend(prev.cpu().numpy(), plain.cpu().numpy(), n)
    assert np.abs(fused.cpu().numpy() - ref).max() <= 4e-7
    tk.close()
