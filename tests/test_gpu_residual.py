"""Pixel residuals (Eq. 4) on the GPU against the oracle.

The threshold decides which elements exist, so the window means are computed
with the same float32 rounding steps on both sides and everything is compared
bit for bit: the dense thresholded residual, its sparse form (positions,
values, segment offsets) and the receiver's frames after the residual is
added back; bf16 and fp32 inputs, ragged last windows, thresholds from zero
to everything, and the residual of a real encode/decode.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import ops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _check(P, x, xh, window, theta, dt):
    xd = torch.from_numpy(x).to("cuda", dt)
    xr = xd.float().cpu().numpy()                      # the values the kernel sees
    hd = torch.from_numpy(xh).cuda()
    r = P.residual(xd, hd, window, theta)
    pos, val, offs = P.residual_sparse(r)
    back = P.residual_apply(hd.clone(), window, pos, val, offs)
    torch.cuda.synchronize()
    rref = ops.residual_mean(xr, xh, window, theta)
    assert np.array_equal(r.cpu().numpy().view(np.uint32), rref.view(np.uint32))
    pref, vref, oref = ops.residual_sparse(rref)
    o = offs.cpu().numpy()
    assert np.array_equal(o, oref)
    assert np.array_equal(pos.cpu().numpy()[:o[-1]], pref)
    assert np.array_equal(val.cpu().numpy()[:o[-1]].view(np.uint32), vref.view(np.uint32))
    bref = ops.residual_apply(xh, pref, vref, oref, window)
    assert np.array_equal(back.cpu().numpy().view(np.uint32), bref.view(np.uint32))
    return int(o[-1])


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("window,theta", [(3, 0.0), (3, 0.05), (4, 0.2), (7, 10.0), (1, 0.01)])
def test_random_residuals(P, dt, window, theta):
    rng = np.random.default_rng(hash((window, theta)) % 2 ** 32)
    N, T, H, W, C = 2, 7, 12, 20, 3
    x = rng.uniform(-1, 1, (N, T, H, W, C)).astype(np.float32)
    xh = (x + rng.normal(0, 0.1, x.shape)).astype(np.float32)
    nnz = _check(P, x, xh, window, theta, dt)
    if theta >= 10.0:
        assert nnz == 0


def test_encode_decode_residual(P):
    """The residual of a real reconstruction (a small tokenizer on a moving-rectangle clip),
    4-frame windows aligned to the chunk structure after frame 0 handled as its own call."""
    tk = P.Tokenizer("bf16", ch=(64, 128, 256), blocks=1)
    tk.set_params(S.weights_for(tk.param_spec(), seed=3))
    T, H, W = 9, 64, 96
    x = S.to_bf16_f32(S.moving_rects_clip(6, T, H, W)[None])
    xd = torch.from_numpy(x).to("cuda", torch.bfloat16)
    tk.reserve(1, T, H, W)
    _, idx = tk.encode(xd, want_z=False)
    xh = tk.decode(idx, H, W)
    torch.cuda.synchronize()
    xh = xh.cpu().numpy()
    tk.close()
    _check(P, x[:, :1], xh[:, :1], 1, 0.05, torch.bfloat16)
    nnz = _check(P, x[:, 1:], xh[:, 1:], 4, 0.05, torch.bfloat16)
    assert nnz > 0


def test_720p_clip_window4(P):
    rng = np.random.default_rng(4)
    N, T, H, W, C = 1, 9, 720, 1280, 3
    x = rng.uniform(-1, 1, (N, T, H, W, C)).astype(np.float32)
    xh = (x + rng.laplace(0, 0.02, x.shape)).astype(np.float32)
    _check(P, x, xh, 4, 0.03, torch.bfloat16)
