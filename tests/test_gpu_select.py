"""Similarity-based token selection (Eq. 3) on the GPU against the oracle.

The selection is an integer decision taken on float32 similarities that both
sides compute with the same rounding steps, so similarities, dropped
indices and packet keep bits must all match bit for bit: random tokens,
tie-heavy tokens (P equal to I, zero vectors), ragged widths, all rates from
nothing to everything, the latents of an encoded clip, and a 1080p-sized
batch checked on sampled frames.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import ops

pytestmark = pytest.mark.gpu
LV = [8, 8, 8, 5, 5, 5]


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _check(P, ip, ii, rate, frames=None):
    dp, di = (torch.from_numpy(a.astype(np.int32)).cuda() for a in (ip, ii))
    out, kb, sim = P.similarity_mask(dp, di, rate, LV, want_sim=True)
    torch.cuda.synchronize()
    out, kb, sim = out.cpu().numpy(), kb.cpu().numpy().view(np.uint32), sim.cpu().numpy()
    N, Tp = ip.shape[:2]
    for b, t in (frames or [(b, t) for b in range(N) for t in range(Tp)]):
        Sref = ops.token_similarity(ip[b:b + 1, t:t + 1], ii[b:b + 1], LV)[0, 0]
        dref = ops.similarity_drop(ip[b:b + 1, t:t + 1], ii[b:b + 1], LV, rate)[0, 0]
        assert np.array_equal(sim[b, t].view(np.uint32), Sref.view(np.uint32)), (b, t)
        assert np.array_equal(out[b, t], ops.apply_drop(ip[b, t], dref, LV)), (b, t)
        assert np.array_equal(kb[b, t], ops.keep_bits_from_mask(dref[None])[0]), (b, t)


@pytest.mark.parametrize("rate", [0.0, 0.07, 0.25, 0.3, 1.0])
@pytest.mark.parametrize("shape", [(2, 3, 9, 40), (1, 4, 17, 70), (3, 1, 5, 33), (2, 2, 9, 64), (1, 2, 90, 160)])
def test_random_tokens(P, rate, shape):
    """Ragged rows, and rows of whole 32-token mask words (64, and 160 as in a 720p
    latent frame), which the last pass walks word by word without dividing."""
    rng = np.random.default_rng(hash((shape, rate)) % 2 ** 32)
    N, Tp, H, W = shape
    ip = rng.integers(0, 64000, shape)
    ii = rng.integers(0, 64000, (N, 1, H, W))
    _check(P, ip, ii, rate)


def test_ties_and_zero_vectors(P):
    """Most P tokens equal their I token (S = 1, one big tie broken by index), some are
    the zero code (S = 0), the rest random."""
    rng = np.random.default_rng(11)
    N, Tp, H, W = 2, 3, 12, 45
    ii = rng.integers(0, 64000, (N, 1, H, W))
    ip = np.repeat(ii, Tp, axis=1).copy()
    r = rng.random(ip.shape)
    ip[r < 0.2] = ops.fsq_zero_index(LV)
    ip[(r >= 0.2) & (r < 0.35)] = rng.integers(0, 64000, ip.shape)[(r >= 0.2) & (r < 0.35)]
    ii[:, :, :2] = ops.fsq_zero_index(LV)          # a zero reference row
    for rate in (0.1, 0.5, 0.9):
        _check(P, ip, ii, rate)
    # the same on rows of whole mask words
    ii2 = rng.integers(0, 64000, (N, 1, 12, 64))
    ip2 = np.repeat(ii2, Tp, axis=1).copy()
    r2 = rng.random(ip2.shape)
    ip2[r2 < 0.2] = ops.fsq_zero_index(LV)
    for rate in (0.1, 0.9):
        _check(P, ip2, ii2, rate)


def test_encoded_clip_latents(P):
    """Indices of a real encode (moving rectangles): P latents 1..T'-1 against latent 0."""
    tk = P.Tokenizer("bf16", ch=(64, 128, 256), blocks=1)
    tk.set_params(S.weights_for(tk.param_spec(), seed=2))
    T, H, W = 13, 96, 160
    x = torch.from_numpy(S.moving_rects_clip(4, T, H, W)[None]).to("cuda", torch.bfloat16)
    tk.reserve(1, T, H, W)
    _, idx = tk.encode(x, want_z=False)
    torch.cuda.synchronize()
    ids = idx.cpu().numpy().astype(np.int64)
    tk.close()
    _check(P, ids[:, 1:], ids[:, :1], 0.25)


def test_1080p_batch_sampled(P):
    """64 streams' 1080p P latents (135 x 240 tokens) in one call; frames sampled."""
    rng = np.random.default_rng(2)
    N, Tp, H, W = 16, 4, 135, 240
    ii = rng.integers(0, 64000, (N, 1, H, W))
    ip = np.where(rng.random((N, Tp, H, W)) < 0.5, np.repeat(ii, Tp, axis=1), rng.integers(0, 64000, (N, Tp, H, W)))
    _check(P, ip, ii, 0.3, frames=[(0, 0), (7, 2), (15, 3)])


def test_argument_errors(P):
    from paper_2602_03529_b300 import _lib as L
    dp = torch.zeros((1, 2, 4, 4), dtype=torch.int32, device="cuda")
    di = torch.zeros((1, 1, 4, 4), dtype=torch.int32, device="cuda")
    out = torch.empty_like(dp)
    ws = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.TokError) as e:
        L.tok_similarity_mask(dp.data_ptr(), di.data_ptr(), 1, 2, 4, 4, LV, 0.5, out.data_ptr(), None, None,
                              ws.data_ptr(), ws.numel(), None)
    assert e.value.code == L.TOK_ENOMEM
    with pytest.raises(L.TokError) as e:
        L.tok_similarity_mask(dp.data_ptr(), di.data_ptr(), 1, 2, 4, 4, [8, 1], 0.5, out.data_ptr(), None, None,
                              ws.data_ptr(), 10 ** 6, None)
    assert e.value.code == L.TOK_EINVAL


def test_large_frames_take_the_three_kernel_form(P):
    """Frames above the fused kernel's shared-memory budget (240 x 256 = 61440 tokens)."""
    rng = np.random.default_rng(9)
    N, Tp, H, W = 1, 2, 240, 256
    ii = rng.integers(0, 64000, (N, 1, H, W))
    ip = np.where(rng.random((N, Tp, H, W)) < 0.3, np.repeat(ii, Tp, axis=1), rng.integers(0, 64000, (N, Tp, H, W)))
    for rate in (0.0, 0.2, 1.0):
        _check(P, ip, ii, rate)


def _bucket_codes():
    """Against the I token 12345: P codes of two distinct similarities that share one of
    the 2048 similarity buckets (width ~1e-3) the selection's first pass uses, and codes
    of clearly lower similarity."""
    ip = np.arange(64000).reshape(1, 1, 1, -1)
    S = ops.token_similarity(ip, np.full((1, 1, 1, 64000), 12345), LV)[0, 0, 0]
    b = np.floor((S.astype(np.float32) + np.float32(1)) * np.float32(1023.5)).astype(int)
    for bb in range(2047, 0, -1):
        vals = np.unique(S[b == bb])
        if len(vals) >= 2:
            c1 = int(np.nonzero(S == vals[0])[0][0])
            c2 = int(np.nonzero(S == vals[-1])[0][0])
            low = np.nonzero(S < vals[0] - 0.05)[0]
            return c1, c2, low
    raise AssertionError("no bucket with two similarities")


@pytest.mark.parametrize("per_value,rate", [(1500, 0.3), (300, 0.05), (300, 0.13)])
def test_bucket_with_distinct_similarities(P, per_value, rate):
    """The k-th largest similarity falls in a bucket holding two different values: more
    tokens there than the candidate list takes (whole-frame radix select) or fewer
    (radix select over the bucket's candidates)."""
    c1, c2, low = _bucket_codes()
    rng = np.random.default_rng(per_value)
    N, Tp, H, W = 1, 2, 60, 80
    ip = rng.choice(low, size=(N, Tp, H, W))
    for t in range(Tp):
        pos = rng.permutation(H * W)[:2 * per_value]
        flat = ip[0, t].reshape(-1)
        flat[pos[:per_value]] = c1
        flat[pos[per_value:]] = c2
    ii = np.full((N, 1, H, W), 12345)
    _check(P, ip, ii, rate)
