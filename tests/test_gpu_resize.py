"""Resolution-control downsampling (Sec. 5) on the GPU against the oracle.

The mean is computed on both sides in float32 with the same rounding steps
and rounded to the output type, so every output must match bit for bit:
uint8 / bf16 / fp32 inputs, bf16 / fp32 outputs, the compiled factors 2 and 3
and the runtime form (1, 4, 5, 8), ragged sizes whose trailing rows and
columns take no part, and 1080p frames at 2x and 3x (the paper's 960x540 and
640x360 encoder inputs).
"""
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


def _input(rng, dtype, shape):
    if dtype == torch.uint8:
        a = rng.integers(0, 256, shape, dtype=np.uint8)
        return torch.from_numpy(a), a
    t = torch.from_numpy(rng.uniform(-1.2, 1.2, shape).astype(np.float32)).to(dtype)
    return t, t.float().numpy()


@pytest.mark.parametrize("in_dtype", [torch.uint8, torch.bfloat16, torch.float32])
@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 8])
def test_bit_exact_against_oracle(P, in_dtype, out_dtype, s):
    rng = np.random.default_rng(s)
    shape = (3, 5 * s + s - 1, 7 * s + 1, 3)        # ragged: trailing rows / columns unused
    x, xo = _input(rng, in_dtype, shape)
    y = P.downsample(x.cuda(), s, out_dtype)
    torch.cuda.synchronize()
    ref = ops.box_downsample(xo, s, out_bf16=out_dtype == torch.bfloat16)
    got = y.float().cpu().numpy()
    assert got.shape == ref.shape
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("C", [1, 4])
def test_channel_counts(P, C):
    rng = np.random.default_rng(C)
    x, xo = _input(rng, torch.float32, (2, 12, 18, C))
    y = P.downsample(x.cuda(), 3, torch.float32)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), ops.box_downsample(xo, 3))


@pytest.mark.parametrize("s", [2, 3])
def test_1080p_frames(P, s):
    """A batch of 1080p uint8 frames (6 streams x 4 frames, 5-D), every output checked."""
    rng = np.random.default_rng(10 + s)
    x = rng.integers(0, 256, (6, 4, 1080, 1920, 3), dtype=np.uint8)
    y = P.downsample(torch.from_numpy(x).cuda(), s, torch.bfloat16)
    torch.cuda.synchronize()
    assert y.shape == (6, 4, 1080 // s, 1920 // s, 3)
    ref = ops.box_downsample(x.reshape(24, 1080, 1920, 3), s, out_bf16=True).reshape(y.shape)
    assert np.array_equal(y.float().cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_empty_and_errors(P):
    from paper_2602_03529_b300 import _lib as L
    x = torch.zeros((0, 8, 8, 3), device="cuda", dtype=torch.uint8)
    assert P.downsample(x, 2).shape == (0, 4, 4, 3)
    x = torch.zeros((1, 8, 8, 3), device="cuda", dtype=torch.uint8)
    y = torch.empty((1, 1, 1, 3), device="cuda", dtype=torch.float32)
    with pytest.raises(L.TokError) as e:
        L.tok_downsample(L.TOK_PIX_U8, x.data_ptr(), 1, 8, 8, 3, 9, L.TOK_FP32, y.data_ptr(), None)
    assert e.value.code == L.TOK_EINVAL
    with pytest.raises(L.TokError) as e:
        L.tok_downsample(7, x.data_ptr(), 1, 8, 8, 3, 2, L.TOK_FP32, y.data_ptr(), None)
    assert e.value.code == L.TOK_EINVAL
    with pytest.raises(L.TokError) as e:
        L.tok_downsample(L.TOK_PIX_U8, x.data_ptr(), 1, 2, 8, 3, 3, L.TOK_FP32, y.data_ptr(), None)
    assert e.value.code == L.TOK_ESHAPE
