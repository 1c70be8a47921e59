"""Parity of the individual CUDA kernels against the FP64 oracle, through the C-ABI.

Tolerances (each with the arithmetic it follows from):
  * conv, FP32 path: the oracle gets the same fp32 inputs; FP32 accumulation
    of K terms plus one fp32 rounding: |gpu - ref| <= 1e-5 |ref| + 2e-6 * s * r,
    s = max |ref|, r = max(1, sqrt(K / 3456)) (rounding errors of a long sum
    grow as sqrt(K); the constant was set for K = 27 * 128).
  * conv, BF16 path: the oracle gets the bf16-rounded inputs and weights, so
    products are exact; FP32 accumulation plus one bf16 output rounding:
    |gpu - ref| <= 2^-8 |ref| + 2e-4 * s.
  * GroupNorm+SiLU: FP32 statistics; fp32 output 1e-5 relative to the output
    scale, bf16 output 2^-8 |ref| + 4e-3 (the input is bf16 already).
  * FSQ, drop mask, packets: integer results, bit-exact (FSQ: away from a
    rounding tie band of 2^-16 around .5, inside it counted).
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import ops

pytestmark = pytest.mark.gpu
LV = (8, 8, 8, 5, 5, 5)


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


CONV_CASES = [
    # (N, T, H, W, Cin, Cout, k, stride, pad)
    (1, 5, 16, 16, 64, 64, 3, (1, 1, 1), 0),
    (1, 5, 12, 20, 64, 128, 3, (1, 1, 1), 1),          # ragged tiles in h and w
    (2, 3, 8, 8, 128, 256, 3, (1, 1, 1), 0),            # batch, N tile 256
    (1, 9, 16, 24, 64, 64, 3, (2, 2, 2), 0),            # strided (parity view)
    (1, 9, 16, 24, 64, 64, 3, (2, 2, 2), 1),
    (1, 4, 10, 12, 64, 128, 3, (1, 2, 2), 0),           # stride (1,2,2)
    (1, 3, 7, 9, 128, 64, 1, (1, 1, 1), 0),             # 1x1x1 shortcut
    # one voxel per thread: whole 64-channel groups staged in shared memory and
    # stored as whole lines, the rest 16 channels at a time
    (1, 3, 9, 24, 128, 256, 1, (1, 1, 1), 1),           # four staged groups, ragged tiles
    (1, 3, 7, 9, 128, 200, 1, (1, 1, 1), 0),            # second channel tile: one group + 8 channels
    (1, 5, 16, 24, 64, 256, 3, (2, 2, 2), 0),           # strided, 256 channels
    (1, 3, 9, 40, 64, 16, 3, (1, 1, 1), 0),             # 16-channel head (dw rows)
    (1, 2, 6, 130, 64, 512, 3, (1, 1, 1), 0),           # W > 128, two N tiles of 256
    # stride-1 3x3x3 layers of 128k channels and narrow heads share one input box among
    # the three dh taps; a layer of less than one wave of (tile, 128-channel) units on
    # 148 SMs takes 8 x 16 tiles (ragged edges)
    (1, 3, 10, 70, 128, 128, 3, (1, 1, 1), 0),
    (1, 3, 5, 130, 128, 128, 3, (1, 1, 1), 1),
    (1, 2, 4, 128, 64, 128, 3, (1, 1, 1), 0),
    (1, 3, 9, 40, 128, 12, 3, (1, 1, 1), 0),            # pixel head (dw rows)
    (1, 3, 30, 32, 128, 128, 3, (1, 1, 1), 0),
    (2, 2, 12, 20, 128, 256, 3, (1, 1, 1), 1),          # two channel tiles
    # larger layers take the tile that minimises waves x (voxels + 48); one column
    # past a whole number of tiles
    (1, 38, 4, 33, 64, 256, 3, (1, 1, 1), 0),           # 4 x 64
    (1, 38, 8, 17, 64, 256, 3, (1, 1, 1), 1),           # 8 x 32
    (1, 38, 5, 17, 64, 256, 3, (1, 1, 1), 0),           # 5 x 32 (N = 160)
    (1, 38, 7, 17, 64, 256, 3, (1, 1, 1), 1),           # 7 x 32 (N = 224)
    (1, 25, 13, 17, 64, 256, 3, (1, 1, 1), 0),          # 13 x 16 (N = 208)
    (1, 25, 15, 17, 64, 256, 3, (1, 1, 1), 1),          # 15 x 16 (N = 240)
    (1, 25, 12, 33, 64, 128, 3, (1, 1, 1), 0),          # 12 x 16 (N = 192)
    (1, 25, 9, 33, 64, 128, 3, (1, 1, 1), 1),           # 2 x 64 (N = 128)
    (1, 3, 11, 37, 64, 24, 3, (1, 1, 1), 1),            # narrow head, 32 weight rows
    (1, 3, 7, 9, 128, 6, 1, (1, 1, 1), 0),              # narrow 1x1x1 (swapped form)
    # 3x3x3 heads with spatial taps as MMA rows, 30 output columns per 32-column input
    # box (ragged last tile, frames narrower than a box): all nine taps when
    # 9 * Cout <= 128 and Cin >= 256 (6 output rows per 8-row box), else the three dw
    # taps up to 16 channels
    (1, 3, 9, 61, 64, 3, 3, (1, 1, 1), 1),              # dw rows; tiles of 30 + 30 + 1 columns
    (1, 3, 9, 61, 256, 3, 3, (1, 1, 1), 1),             # nine taps; tiles of 30 + 30 + 1 columns
    (2, 4, 17, 30, 192, 1, 3, (1, 1, 1), 0),            # dw rows, one output channel, W = 30
    (2, 4, 17, 30, 256, 1, 3, (1, 1, 1), 0),            # nine taps, one output channel, W = 30
    (1, 2, 8, 31, 512, 6, 3, (1, 1, 1), 0),             # nine taps, latent-head width, W = 31
    (1, 3, 13, 45, 256, 12, 3, (1, 1, 1), 0),           # nine taps, pixel-head width (108 rows), 13 rows
    (1, 2, 7, 33, 256, 14, 3, (1, 1, 1), 1),            # nine taps, 126 rows
    (1, 3, 3, 5, 64, 16, 3, (1, 1, 1), 1),              # dw rows; frame smaller than one box
    (1, 3, 10, 62, 128, 15, 3, (1, 1, 1), 0),           # dw rows, 15 channels
]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("case", CONV_CASES)
def test_conv3d_parity(P, prec, case):
    N, T, H, W, Cin, Cout, k, stride, pad = case
    rng = np.random.default_rng(hash(case) % 2**32)
    x = rng.standard_normal((N, T, H, W, Cin)).astype(np.float32)
    w = (rng.standard_normal((Cout, k, k, k, Cin)) * np.sqrt(2.0 / (Cin * k ** 3))).astype(np.float32)
    b = rng.standard_normal(Cout).astype(np.float32) * 0.1
    if prec == "bf16":
        x, w = S.to_bf16_f32(x), S.to_bf16_f32(w)
    ref = ops.conv3d(x, w, b, stride, pad)
    res = rng.standard_normal(ref.shape).astype(np.float32)
    if prec == "bf16":
        res = S.to_bf16_f32(res)
    ref_r = ref + res
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    tp = "replicate" if pad == 0 else "zero"
    y = P.conv3d(_dev(x, dt), _dev(w), _dev(b), stride, tp)
    yr = P.conv3d(_dev(x, dt), _dev(w), _dev(b), stride, tp, residual=_dev(res, dt))
    torch.cuda.synchronize()
    for got, want in ((y, ref), (yr, ref_r)):
        g = got.float().cpu().numpy().astype(np.float64)
        s = np.abs(want).max()
        if prec == "fp32":
            tol = 1e-5 * np.abs(want) + 2e-6 * s * max(1.0, np.sqrt(k ** 3 * Cin / 3456))
        else:
            tol = 2.0 ** -8 * np.abs(want) + 2e-4 * s
        err = np.abs(g - want)
        assert g.shape == want.shape
        assert np.all(err <= tol), (float(err.max()), float((err / (tol + 1e-30)).max()))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("shape,G", [((1, 3, 16, 16, 128), 32), ((2, 2, 8, 12, 256), 32),
                                     ((1, 2, 4, 4, 512), 32), ((1, 3, 5, 7, 16), 8), ((1, 2, 9, 9, 64), 32),
                                     # a chunk's last bulk-copy segment partly filled; frames of
                                     # several chunks with a ragged last one
                                     ((1, 2, 10, 13, 128), 32), ((2, 3, 40, 60, 128), 32)])
def test_groupnorm_silu_parity(P, prec, shape, G):
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(shape) * 2 + 0.5).astype(np.float32)
    C = shape[-1]
    gam = (1 + 0.1 * rng.standard_normal(C)).astype(np.float32)
    bet = (0.1 * rng.standard_normal(C)).astype(np.float32)
    if prec == "bf16":
        x = S.to_bf16_f32(x)
    ref = ops.silu(ops.group_norm_frames(x, G, 1e-6, gam, bet))
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    y = P.groupnorm_silu(_dev(x, dt), G, _dev(gam), _dev(bet), 1e-6)
    torch.cuda.synchronize()
    g = y.float().cpu().numpy()
    err = np.abs(g - ref)
    tol = (1e-5 * (np.abs(ref) + 1.0)) if prec == "fp32" else (2.0 ** -8 * np.abs(ref) + 4e-3)
    assert np.all(err <= tol), float(err.max())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_groupnorm_silu_in_place(P, prec):
    """y may alias x: every chunk is in shared memory before any of its outputs is
    written (frames of several chunks, a ragged last one)."""
    rng = np.random.default_rng(11)
    shape, G = (2, 2, 40, 60, 128), 32
    x = (rng.standard_normal(shape) * 2 + 0.5).astype(np.float32)
    if prec == "bf16":
        x = S.to_bf16_f32(x)
    ref = ops.silu(ops.group_norm_frames(x, G, 1e-6, None, None))
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    xd = _dev(x, dt)
    y = P.groupnorm_silu(xd, G, None, None, 1e-6, out=xd)
    torch.cuda.synchronize()
    assert y.data_ptr() == xd.data_ptr()
    g = xd.float().cpu().numpy()
    tol = (1e-5 * (np.abs(ref) + 1.0)) if prec == "fp32" else (2.0 ** -8 * np.abs(ref) + 4e-3)
    assert np.all(np.abs(g - ref) <= tol), float(np.abs(g - ref).max())


@pytest.mark.parametrize("n,off", [(1 << 20, 0), (1001, 0), (1003, 1)])
def test_fsq_parity_with_tie_band(P, n, off):
    """The kernel rounds the exactly computed bounded value (thresholds on z), so its
    index differs from the FP64 oracle's only where the oracle's own rounding error
    (~1e-16) could flip a decision: a band of 1e-9 around the rounding ties. Token
    counts with a partial group of four, and an input that starts one token into its
    buffer (24 bytes: the element-wise form)."""
    rng = np.random.default_rng(11)
    z = (rng.standard_normal((n, 6)) * 1.5).astype(np.float32)
    idx_ref, codes_ref, b = ops.fsq_quantize(z.astype(np.float64), LV)
    zd = _dev(np.concatenate([np.zeros((off, 6), np.float32), z]))[off:]
    idx, codes = P.quantize(zd, LV, codes=True)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    near_tie = (np.abs(np.abs(b - np.floor(b)) - 0.5) <= 1e-9).any(axis=1)
    mism = idx != idx_ref
    assert not np.any(mism & ~near_tie)
    ok = ~mism
    np.testing.assert_array_equal(codes.cpu().numpy()[ok], codes_ref[ok].astype(np.float32))


def _oracle_digit(c, zc):
    z = np.zeros((len(zc), len(LV)))
    z[:, c] = zc
    return ops.fsq_index_to_digits(ops.fsq_quantize(z, LV)[0], LV)[:, c]


def test_fsq_every_rounding_boundary(P):
    """At every digit boundary of every channel: the smallest float32 z that the FP64
    oracle puts past the boundary, and the float32 just below it. The kernel's digit
    must equal the oracle's at both (a threshold rounded the wrong way, an off-by-one
    boundary or a wrong shift fails here)."""
    h, o, s, hw, _ = ops.fsq_constants(LV)
    zs, cs, ks = [], [], []
    for c, L in enumerate(LV):
        for k in range(L - 1):
            f = np.float32(np.arctanh((k + 0.5 - hw[c] + o[c]) / h[c]) - s[c])
            while _oracle_digit(c, [f])[0] <= k:
                f = np.nextafter(f, np.float32(np.inf))
            while _oracle_digit(c, [np.nextafter(f, np.float32(-np.inf))])[0] > k:
                f = np.nextafter(f, np.float32(-np.inf))
            for zz in (f, np.nextafter(f, np.float32(-np.inf))):
                zs.append(zz)
                cs.append(c)
                ks.append(k)
    z = np.zeros((len(zs), len(LV)), np.float32)
    z[np.arange(len(zs)), cs] = zs
    ref = ops.fsq_quantize(z.astype(np.float64), LV)[0]
    idx = P.quantize(_dev(z), LV).cpu().numpy()
    np.testing.assert_array_equal(idx, ref)
    dig = ops.fsq_index_to_digits(ref, LV)[np.arange(len(zs)), cs]
    assert np.array_equal(dig[0::2], np.array(ks[0::2]) + 1) and np.array_equal(dig[1::2], np.array(ks[1::2]))


def test_fsq_closed_forms_on_gpu(P):
    z = torch.zeros((4, 6), device="cuda")
    z[1] = 50.0
    z[2] = -50.0
    idx = P.quantize(z, LV).cpu().numpy()
    assert idx.tolist()[:3] == [32036, 63999, 0]
    all_idx = torch.arange(64000, device="cuda", dtype=torch.int32)
    codes = P.dequantize(all_idx, LV).cpu().numpy()
    np.testing.assert_array_equal(codes, ops.fsq_dequantize(np.arange(64000), LV).astype(np.float32))


@pytest.mark.parametrize("rate", [0.0, 0.13, 0.3, 1.0])
@pytest.mark.parametrize("shape", [(1, 5, 45, 80), (2, 1, 7, 37), (1, 3, 135, 240), (3, 2, 9, 131),
                                   (1, 1, 3, 301)])
def test_drop_mask_bit_exact(P, rate, shape):
    """Rows whose first token is or is not on a multiple of 4 (one or two Philox blocks
    per lane), one to three 128-token segments per row, ragged last mask word."""
    N, Tq, Hq, Wq = shape
    rng = np.random.default_rng(3)
    idx = rng.integers(0, 64000, size=shape).astype(np.int32)
    seed, sid, cid = (7 << 32) | 1234, 5, 9
    out, kb = P.drop_mask(_dev(idx, torch.int32), rate, seed, sid, cid, LV)
    torch.cuda.synchronize()
    dropped = ops.drop_mask(N, Tq, Hq, Wq, rate, seed, sid, cid)
    np.testing.assert_array_equal(out.cpu().numpy(), ops.apply_drop(idx, dropped, LV))
    np.testing.assert_array_equal(kb.cpu().numpy().view(np.uint32), ops.keep_bits_from_mask(dropped))


def test_packets_bit_exact(P):
    N, Tq, Hq, Wq = 1, 2, 60, 107
    rng = np.random.default_rng(4)
    idx = rng.integers(0, 64000, size=(N, Tq, Hq, Wq)).astype(np.int32)
    out, kb = P.drop_mask(_dev(idx, torch.int32), 0.25, 99, 1, 2, LV)
    payload, offs = P.pack_rows(out, kb)
    torch.cuda.synchronize()
    dropped = ops.drop_mask(N, Tq, Hq, Wq, 0.25, 99, 1, 2)
    kb_ref = ops.keep_bits_from_mask(dropped)
    pay_ref, offs_ref = ops.pack_rows(idx, kb_ref, Wq)
    np.testing.assert_array_equal(offs.cpu().numpy(), offs_ref)
    np.testing.assert_array_equal(payload.cpu().numpy()[:len(pay_ref)], pay_ref)
    rows = N * Tq * Hq
    recv = np.ones(rows, np.uint8)
    recv[[0, 17, rows - 1]] = 0
    got = P.unpack_rows(payload, offs, kb, _dev(recv, torch.uint8), (N, Tq, Hq, Wq), LV)
    torch.cuda.synchronize()
    ref = ops.unpack_rows(pay_ref, offs_ref, kb_ref, recv.astype(bool), Wq, 32036).reshape(N, Tq, Hq, Wq)
    np.testing.assert_array_equal(got.cpu().numpy(), ref)


def test_guard_bands_catch_a_write_outside_the_workspace(P):
    """The check behind every test's closing guard assertion: a byte written into the
    arena's trailing band is reported, and the restored band passes again."""
    from paper_2602_03529_b300 import _lib as L
    tk = P.Tokenizer("bf16", kind="stage", ch=(64, 128))
    assert L.tok_selftest_guards(tk.ctx) == L.TOK_ESTATE   # nothing reserved yet
    tk.reserve(1, 5, 32, 32)
    assert L.tok_selftest_guards(tk.ctx) == L.TOK_OK
    assert tk.check_guards() == L.TOK_OK
    tk.close()


def test_bounded_wait_times_out_and_context_survives(P):
    from paper_2602_03529_b300 import _lib as L
    tk = P.Tokenizer("bf16", kind="stage", ch=(64, 128))
    assert tk.status() == L.TOK_OK
    L.tok_selftest_timeout(tk.ctx, 20_000_000, torch.cuda.current_stream().cuda_stream)
    assert tk.status() == L.TOK_ETIMEOUT
    assert tk.status() == L.TOK_OK          # cleared once read
    x = torch.ones(4, device="cuda")        # the CUDA context is still usable
    assert float(x.sum()) == 4.0
    tk.close()
