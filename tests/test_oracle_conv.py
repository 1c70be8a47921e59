"""Pins of the oracle's causal 3D convolution (forward, dgrad, wgrad).

The oracle is checked against things other than itself: PyTorch's FP64
conv3d (a library routine) on explicitly padded input, hand-computed closed
forms, causality, and the adjoint identities that tie dgrad/wgrad to the
forward.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import ops


def torch_causal_conv(x, w, b, stride, pad_mode):
    """Library special case: pad explicitly, then torch's cross-correlation."""
    xt = torch.from_numpy(np.ascontiguousarray(x)).permute(0, 4, 1, 2, 3)  # N C T H W
    wt = torch.from_numpy(np.ascontiguousarray(w)).permute(0, 4, 1, 2, 3)  # O I kt kh kw
    kt, kh, kw = w.shape[1:4]
    ph, pw = (kh - 1) // 2, (kw - 1) // 2
    if kt > 1:
        if pad_mode == ops.PAD_REPLICATE:
            first = xt[:, :, :1].expand(-1, -1, kt - 1, -1, -1)
        else:
            first = torch.zeros_like(xt[:, :, :1]).expand(-1, -1, kt - 1, -1, -1)
        xt = torch.cat([first, xt], dim=2)
    xt = F.pad(xt, (pw, pw, ph, ph, 0, 0))
    y = F.conv3d(xt, wt, None if b is None else torch.from_numpy(b), stride=stride)
    return y.permute(0, 2, 3, 4, 1).numpy()


@pytest.mark.parametrize("shape,k,stride,pad", [
    ((2, 5, 6, 7, 3), (3, 3, 3), (1, 1, 1), ops.PAD_REPLICATE),
    ((1, 5, 6, 7, 4), (3, 3, 3), (1, 1, 1), ops.PAD_ZERO),
    ((1, 9, 8, 10, 5), (3, 3, 3), (2, 2, 2), ops.PAD_REPLICATE),
    ((1, 9, 8, 10, 5), (3, 3, 3), (2, 2, 2), ops.PAD_ZERO),
    ((1, 4, 9, 7, 3), (3, 3, 3), (1, 2, 2), ops.PAD_REPLICATE),
    ((2, 3, 5, 5, 6), (1, 1, 1), (1, 1, 1), ops.PAD_REPLICATE),
])
def test_conv_matches_torch_fp64(shape, k, stride, pad):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape)
    cout = 7
    w = rng.standard_normal((cout, *k, shape[-1]))
    b = rng.standard_normal(cout)
    y = ops.conv3d(x, w, b, stride, pad)
    ref = torch_causal_conv(x, w, b, stride, pad)
    assert y.shape == ref.shape
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_conv_temporal_closed_form():
    """Temporal taps [1, 10, 100] on a 1x1 frame sequence [1, 2, 3]:
    y_t = x_{t-2} + 10 x_{t-1} + 100 x_t with the past padded by frame 0
    (replicate) or by zeros."""
    x = np.array([1.0, 2.0, 3.0]).reshape(1, 3, 1, 1, 1)
    w = np.zeros((1, 3, 3, 3, 1))
    w[0, :, 1, 1, 0] = [1.0, 10.0, 100.0]
    y = ops.conv3d(x, w, None, (1, 1, 1), ops.PAD_REPLICATE).ravel()
    assert y.tolist() == [111.0, 1 + 10 + 200.0, 1 + 20 + 300.0]
    y = ops.conv3d(x, w, None, (1, 1, 1), ops.PAD_ZERO).ravel()
    assert y.tolist() == [100.0, 10 + 200.0, 1 + 20 + 300.0]
    # stride 2 in time: outputs at frames 0 and 2
    y = ops.conv3d(x, w, None, (2, 1, 1), ops.PAD_REPLICATE).ravel()
    assert y.tolist() == [111.0, 1 + 20 + 300.0]


def test_conv_spatial_one_hot_shifts():
    """A one-hot kernel at spatial tap (dh, dw) shifts the frame by (dh-1, dw-1)
    and reads zeros past the border."""
    x = np.arange(1, 1 + 4 * 5, dtype=np.float64).reshape(1, 1, 4, 5, 1)
    for dh in range(3):
        for dw in range(3):
            w = np.zeros((1, 1, 3, 3, 1))
            w[0, 0, dh, dw, 0] = 1.0
            y = ops.conv3d(x, w, None).reshape(4, 5)
            xp = np.pad(x.reshape(4, 5), 1)
            np.testing.assert_array_equal(y, xp[dh:dh + 4, dw:dw + 5])


def test_conv_output_shapes():
    assert ops.conv_out_shape(17, 256, 256, (3, 3, 3), (1, 2, 2)) == (17, 128, 128)
    assert ops.conv_out_shape(17, 128, 128, (3, 3, 3), (2, 2, 2)) == (9, 64, 64)
    assert ops.conv_out_shape(9, 64, 64, (3, 3, 3), (2, 2, 2)) == (5, 32, 32)
    assert ops.conv_out_shape(5, 45, 80, (3, 3, 3), (2, 2, 2)) == (3, 23, 40)


@pytest.mark.parametrize("stride", [(1, 1, 1), (2, 2, 2)])
@pytest.mark.parametrize("pad", [ops.PAD_REPLICATE, ops.PAD_ZERO])
def test_conv_causal(stride, pad):
    """Output frame t reads only frames <= t*st: perturbing later frames
    leaves it bit-identical."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 9, 6, 6, 3))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    y0 = ops.conv3d(x, w, None, stride, pad)
    for t in range(y0.shape[1]):
        x2 = x.copy()
        x2[:, t * stride[0] + 1:] += rng.standard_normal(x2[:, t * stride[0] + 1:].shape)
        y1 = ops.conv3d(x2, w, None, stride, pad)
        np.testing.assert_array_equal(y0[:, :t + 1], y1[:, :t + 1])


@pytest.mark.parametrize("shape,k,stride,pad", [
    ((1, 5, 6, 7, 3), (3, 3, 3), (1, 1, 1), ops.PAD_REPLICATE),
    ((2, 9, 8, 6, 4), (3, 3, 3), (2, 2, 2), ops.PAD_REPLICATE),
    ((1, 5, 6, 6, 3), (3, 3, 3), (1, 2, 2), ops.PAD_ZERO),
    ((1, 3, 4, 4, 5), (1, 1, 1), (1, 1, 1), ops.PAD_REPLICATE),
])
def test_conv_grads_match_torch_autograd(shape, k, stride, pad):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(shape)
    w = rng.standard_normal((5, *k, shape[-1]))
    b = rng.standard_normal(5)
    y = ops.conv3d(x, w, b, stride, pad)
    dy = rng.standard_normal(y.shape)
    dx = ops.conv3d_dgrad(dy, w, x.shape, stride, pad)
    dw, db = ops.conv3d_wgrad(dy, x, k, stride, pad)
    xt = torch.from_numpy(x).requires_grad_(True)
    wt = torch.from_numpy(w).requires_grad_(True)
    bt = torch.from_numpy(b).requires_grad_(True)
    # torch reference with explicit padding, as in torch_causal_conv
    xx = xt.permute(0, 4, 1, 2, 3)
    kt, kh, kw = k
    if kt > 1:
        first = xx[:, :, :1] if pad == ops.PAD_REPLICATE else torch.zeros_like(xx[:, :, :1])
        xx = torch.cat([first.expand(-1, -1, kt - 1, -1, -1), xx], dim=2)
    xx = F.pad(xx, ((kw - 1) // 2,) * 2 + ((kh - 1) // 2,) * 2 + (0, 0))
    yt = F.conv3d(xx, wt.permute(0, 4, 1, 2, 3), bt, stride=stride).permute(0, 2, 3, 4, 1)
    (yt * torch.from_numpy(dy)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(dw, wt.grad.numpy(), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-11, atol=1e-11)


def test_conv_adjoint_identities():
    """<conv(x), dy> = <x, dgrad(dy)> and <conv_w(x), dy> = <w, wgrad(dy)>."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 7, 5, 6, 3))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    for stride in [(1, 1, 1), (2, 2, 2)]:
        y = ops.conv3d(x, w, None, stride)
        dy = rng.standard_normal(y.shape)
        dx = ops.conv3d_dgrad(dy, w, x.shape, stride)
        dw, _ = ops.conv3d_wgrad(dy, x, (3, 3, 3), stride)
        lhs = float((y * dy).sum())
        assert abs(lhs - float((x * dx).sum())) < 1e-9 * max(1.0, abs(lhs))
        assert abs(lhs - float((w * dw).sum())) < 1e-9 * max(1.0, abs(lhs))


@pytest.mark.parametrize("shape,k,stride,pad", [
    ((1, 5, 6, 7, 3), (3, 3, 3), (1, 1, 1), ops.PAD_REPLICATE),
    ((2, 9, 8, 6, 4), (3, 3, 3), (2, 2, 2), ops.PAD_REPLICATE),
    ((1, 5, 6, 6, 3), (3, 3, 3), (1, 2, 2), ops.PAD_ZERO),
    ((1, 3, 4, 4, 5), (1, 1, 1), (1, 1, 1), ops.PAD_REPLICATE),
])
def test_gradient_entries_match_full_gradients(shape, k, stride, pad):
    """The single-entry weight and input gradients (used to check large clips on
    samples) equal the full dgrad / wgrad at every entry and every point; the
    magnitudes bound the values and are positive where a term exists."""
    rng = np.random.default_rng(9)
    x = rng.standard_normal(shape)
    w = rng.standard_normal((5, *k, shape[-1]))
    y = ops.conv3d(x, w, None, stride, pad)
    dy = rng.standard_normal(y.shape)
    dx = ops.conv3d_dgrad(dy, w, x.shape, stride, pad)
    dw, _ = ops.conv3d_wgrad(dy, x, k, stride, pad)
    entries = [tuple(int(v) for v in e) for e in np.ndindex(dw.shape)]
    vals, mags = ops.conv3d_wgrad_entries(dy, x, k, entries, stride, pad)
    np.testing.assert_allclose(vals, dw.reshape(-1), rtol=1e-12, atol=1e-12)
    assert np.all(mags >= np.abs(vals) - 1e-12)
    N, T, H, W, _ = shape
    points = [(n, t, h, wv) for n in range(N) for t in range(T) for h in range(H) for wv in range(W)]
    vals, mags = ops.conv3d_dgrad_entries(dy, w, x.shape, points, stride, pad)
    np.testing.assert_allclose(vals, dx.reshape(len(points), -1), rtol=1e-12, atol=1e-12)
    assert np.all(mags >= np.abs(vals) - 1e-12)
