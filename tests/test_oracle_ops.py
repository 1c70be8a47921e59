"""Pins of the oracle's GroupNorm, SiLU, FSQ, Philox drop mask, row packets
and depth-to-space: library routines, closed forms, invariants and the
published Philox known-answer vectors."""
import json
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import ops

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- GroupNorm

def test_gn_matches_torch_group_norm_per_frame():
    """Per-frame GroupNorm equals torch's group_norm applied to each frame."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 5, 6, 16)) * 3 + 1
    g = rng.standard_normal(16)
    b = rng.standard_normal(16)
    y = ops.group_norm_frames(x, 8, 1e-6, g, b)
    xt = torch.from_numpy(x).reshape(6, 5, 6, 16).permute(0, 3, 1, 2)
    ref = F.group_norm(xt, 8, torch.from_numpy(g), torch.from_numpy(b), eps=1e-6)
    ref = ref.permute(0, 2, 3, 1).reshape(x.shape).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-10, atol=1e-10)


def test_gn_moments_closed_form():
    """Without affine, every (sample, group, frame) slice has mean 0 and
    variance sigma^2 / (sigma^2 + eps)."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 4, 3, 3, 8)) * np.arange(1, 9)
    eps = 1e-2
    y = ops.group_norm_frames(x, 4, eps)
    xg = x.reshape(1, 4, 9, 4, 2)
    yg = y.reshape(1, 4, 9, 4, 2)
    var = xg.var(axis=(2, 4))
    np.testing.assert_allclose(yg.mean(axis=(2, 4)), 0.0, atol=1e-12)
    np.testing.assert_allclose(yg.var(axis=(2, 4)), var / (var + eps), rtol=1e-12)


def test_gn_frames_independent():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 3, 3, 8))
    y0 = ops.group_norm_frames(x, 4)
    x[:, 2] *= 5.0
    x[:, 2] += 3.0
    y1 = ops.group_norm_frames(x, 4)
    np.testing.assert_array_equal(y0[:, :2], y1[:, :2])
    np.testing.assert_array_equal(y0[:, 3:], y1[:, 3:])


def test_gn_groups_reading():
    assert ops.gn_groups(128) == 32 and ops.gn_groups(512) == 32
    assert ops.gn_groups(16) == 8 and ops.gn_groups(32) == 16 and ops.gn_groups(64) == 32


def test_silu_matches_torch():
    x = np.linspace(-20, 20, 401)
    np.testing.assert_allclose(ops.silu(x), F.silu(torch.from_numpy(x)).numpy(), rtol=1e-14, atol=1e-300)
    assert ops.silu(np.array([0.0]))[0] == 0.0


# ---------------------------------------------------------------------- FSQ

G = _gold("fsq_8_8_8_5_5_5.json")
LV = G["levels"]


def test_fsq_closed_forms():
    _, _, _, hw, basis = ops.fsq_constants(LV)
    assert basis.tolist() == G["basis"]
    assert int(np.prod(LV)) == G["codebook_size"]
    assert ops.fsq_zero_index(LV) == G["zero_index"]
    assert abs(math.log2(G["codebook_size"]) - G["bits_per_token"]) < 1e-12
    idx, codes, b = ops.fsq_quantize(np.zeros((1, 6)), LV)
    assert int(idx[0]) == G["zero_index"]
    assert np.all(codes == 0.0)
    np.testing.assert_allclose(b, 0.0, atol=1e-15)


def test_fsq_extremes():
    idx, _, _ = ops.fsq_quantize(np.full((1, 6), 50.0), LV)
    assert int(idx[0]) == G["max_index"]
    idx, codes, _ = ops.fsq_quantize(np.full((1, 6), -50.0), LV)
    assert int(idx[0]) == 0
    assert np.all(codes == -1.0)


def test_fsq_bijection_exhaustive():
    """Every one of the 64000 digit vectors maps to a distinct index in
    [0, 64000), and index -> digits inverts it."""
    grids = np.meshgrid(*[np.arange(l) for l in LV], indexing="ij")
    d = np.stack([g.ravel() for g in grids], axis=-1)
    _, _, _, _, basis = ops.fsq_constants(LV)
    idx = (d * basis).sum(-1)
    assert np.array_equal(np.sort(idx), np.arange(64000))
    np.testing.assert_array_equal(ops.fsq_index_to_digits(idx, LV), d)


def test_fsq_grid_points_fixed():
    """Quantising the pre-image of every grid code returns that code
    (idempotence of quantise o dequantise on the grid)."""
    h, o, s, hw, basis = ops.fsq_constants(LV)
    for ch, L in enumerate(LV):
        for dgt in range(L):
            q = dgt - L // 2
            # the bound's range is (-h-o, h-o): the lowest even-level digit is
            # reached only by rounding, so aim just inside the range there
            bt = min(max(q, -h[ch] - o[ch] + 0.01), h[ch] - o[ch] - 0.01)
            zc = np.arctanh((bt + o[ch]) / h[ch]) - s[ch]
            z = np.zeros((1, 6))
            z[0, ch] = zc
            idx, codes, _ = ops.fsq_quantize(z, LV)
            assert ops.fsq_index_to_digits(idx, LV)[0, ch] == dgt
            assert codes[0, ch] == q / (L // 2)
            np.testing.assert_allclose(ops.fsq_dequantize(idx, LV), codes)


def test_fsq_monotone():
    z = np.linspace(-6, 6, 2001)
    for ch in range(6):
        zz = np.zeros((z.size, 6))
        zz[:, ch] = z
        d = ops.fsq_index_to_digits(ops.fsq_quantize(zz, LV)[0], LV)[:, ch]
        assert np.all(np.diff(d) >= 0)
        assert d[0] == 0 and d[-1] == LV[ch] - 1


def test_fsq_codes_in_range():
    rng = np.random.default_rng(5)
    idx, codes, _ = ops.fsq_quantize(rng.standard_normal((1000, 6)) * 3, LV)
    assert idx.min() >= 0 and idx.max() < 64000
    assert np.all(np.abs(codes) <= 1.0)


# ------------------------------------------------------------ Philox + mask

def test_philox_known_answers():
    for v in _gold("philox4x32_10_kat.json")["vectors"]:
        c = [int(a, 16) for a in v["ctr"]]
        k = [int(a, 16) for a in v["key"]]
        out = ops.philox4x32_10(*c, *k)
        assert [int(o) for o in out] == [int(a, 16) for a in v["out"]]


@pytest.mark.parametrize("rate", [0.05, 0.25, 0.3])
def test_drop_rate_binomial(rate):
    m = ops.drop_mask(2, 3, 45, 80, rate, seed=1234, stream_id=7, chunk_id=3)
    n = m.size
    k = int(m.sum())
    sd = math.sqrt(n * rate * (1 - rate))
    assert abs(k - n * rate) < 5 * sd


def test_drop_rate_extremes_and_keys():
    assert not ops.drop_mask(1, 2, 4, 5, 0.0, 1, 0, 0).any()
    assert ops.drop_mask(1, 2, 4, 5, 1.0, 1, 0, 0).all()
    a = ops.drop_mask(1, 1, 30, 40, 0.5, 9, 1, 2)
    assert np.array_equal(a, ops.drop_mask(1, 1, 30, 40, 0.5, 9, 1, 2))
    assert not np.array_equal(a, ops.drop_mask(1, 1, 30, 40, 0.5, 9, 1, 3))
    assert not np.array_equal(a, ops.drop_mask(1, 1, 30, 40, 0.5, 9, 2, 2))
    assert not np.array_equal(a, ops.drop_mask(1, 1, 30, 40, 0.5, 10, 1, 2))


def test_drop_uses_philox_word():
    """Token j of sample n takes word j&3 of Philox(counter (j>>2, n, chunk,
    stream), key (seed lo, seed hi)) and drops iff it is below floor(rate*2^32)."""
    seed, sid, cid, rate = (5 << 32) | 17, 3, 11, 0.4
    m = ops.drop_mask(2, 1, 3, 5, rate, seed, sid, cid).reshape(2, -1)
    thr = int(np.floor(float(np.float32(rate)) * 2 ** 32))
    for n in range(2):
        for j in range(15):
            w = ops.philox4x32_10(j >> 2, n, cid, sid, 17, 5)[j & 3]
            assert bool(m[n, j]) == (int(w) < thr)


def test_packets_roundtrip_and_lost_rows():
    rng = np.random.default_rng(6)
    idx = rng.integers(0, 64000, size=(2, 1, 7, 37))
    dropped = ops.drop_mask(2, 1, 7, 37, 0.3, 1, 2, 3)
    kb = ops.keep_bits_from_mask(dropped)
    assert kb.shape == (2, 1, 7, 2)
    payload, offs = ops.pack_rows(idx, kb, 37)
    assert len(payload) == int((~dropped).sum()) and offs[-1] == len(payload)
    z = ops.fsq_zero_index(LV)
    rows = 2 * 7
    got = ops.unpack_rows(payload, offs, kb, np.ones(rows, bool), 37, z).reshape(idx.shape)
    np.testing.assert_array_equal(got, ops.apply_drop(idx, dropped, LV))
    recv = np.ones(rows, bool)
    recv[[1, 9]] = False
    got = ops.unpack_rows(payload, offs, kb, recv, 37, z).reshape(rows, 37)
    assert np.all(got[[1, 9]] == z)
    ref = ops.apply_drop(idx, dropped, LV).reshape(rows, 37)
    np.testing.assert_array_equal(got[recv], ref[recv])


# ----------------------------------------------------------- depth-to-space

def test_d2s_channel_order_closed_form():
    """Channel ((a*2+b)*2+c) of latent (t,h,w) lands at (2t+a-1, 2h+b, 2w+c)."""
    y = np.arange(8, dtype=np.float64).reshape(1, 1, 1, 1, 8)
    o = ops.depth_to_space(y, (2, 2, 2), drop_first=0)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                assert o[0, a, b, c, 0] == (a * 2 + b) * 2 + c
    o = ops.depth_to_space(y, (2, 2, 2))
    assert o.shape == (1, 1, 2, 2, 1)
    assert o[0, 0, :, :, 0].tolist() == [[4, 5], [6, 7]]


def test_d2s_s2d_inverse():
    rng = np.random.default_rng(7)
    y = rng.standard_normal((2, 5, 3, 4, 8 * 3))
    x = ops.depth_to_space(y, (2, 2, 2))
    assert x.shape == (2, 9, 6, 8, 3)
    yy = ops.space_to_depth(x, (2, 2, 2))
    yy[:, 0, ..., :3 * 1] = y[:, 0, ..., :3]  # the dropped frame's channels are gone
    np.testing.assert_array_equal(yy[:, 1:], y[:, 1:])
    np.testing.assert_array_equal(ops.depth_to_space(ops.space_to_depth(x, (2, 2, 2)), (2, 2, 2)), x)
    y2 = rng.standard_normal((1, 3, 2, 2, 12))
    np.testing.assert_array_equal(ops.space_to_depth(ops.depth_to_space(y2, (1, 2, 2)), (1, 2, 2)), y2)


def test_edge_pad():
    x = np.arange(2 * 3 * 5, dtype=np.float64).reshape(1, 1, 3 * 2, 5, 1)[:, :, :3]
    p = ops.edge_pad_to_multiple(x, 4)
    assert p.shape == (1, 1, 4, 8, 1)
    np.testing.assert_array_equal(p[0, 0, 3], p[0, 0, 2])
    np.testing.assert_array_equal(p[0, 0, :, 7], p[0, 0, :, 4])


# ------------------------------------------------- similarity-based selection (Eq. 3)

LV = [8, 8, 8, 5, 5, 5]


def _idx_of_digits(d, levels=LV):
    _, _, _, _, basis = ops.fsq_constants(levels)
    return int((np.asarray(d) * basis).sum())


def test_similarity_closed_forms():
    """Identical codes give 1, opposite codes -1, orthogonal codes 0, a zero code 0."""
    hw = [4, 4, 4, 2, 2, 2]
    a = [hw[0] + 2, hw[1], hw[2], hw[3] + 1, hw[4], hw[5]]          # code (0.5, 0, 0, 0.5, 0, 0)
    neg = [hw[0] - 2, hw[1], hw[2], hw[3] - 1, hw[4], hw[5]]        # (-0.5, 0, 0, -0.5, 0, 0)
    orth = [hw[0], hw[1] + 3, hw[2], hw[3], hw[4], hw[5] + 2]        # (0, 0.75, 0, 0, 0, 1)
    zero = hw
    I = np.array([[[[_idx_of_digits(a)]]]])
    P = np.array([[[[_idx_of_digits(a)]], [[_idx_of_digits(neg)]], [[_idx_of_digits(orth)]],
                   [[_idx_of_digits(zero)]]]])
    S = ops.token_similarity(P, I, LV)
    assert S.reshape(-1).tolist() == [1.0, -1.0, 0.0, 0.0]
    assert ops.fsq_zero_index(LV) == _idx_of_digits(zero)
    # a zero reference makes every similarity 0
    S0 = ops.token_similarity(P, np.array([[[[_idx_of_digits(zero)]]]]), LV)
    assert not S0.any()


def test_similarity_matches_a_float64_cosine():
    """The float32 similarity is the cosine of the two code vectors (independent fp64
    formula through numpy.linalg), to float32 rounding."""
    rng = np.random.default_rng(3)
    P = rng.integers(0, 64000, (2, 3, 6, 9))
    I = rng.integers(0, 64000, (2, 1, 6, 9))
    p = ops.fsq_dequantize(P, LV)
    q = np.broadcast_to(ops.fsq_dequantize(I, LV), p.shape)
    num = np.einsum("...c,...c->...", p, q)
    den = np.linalg.norm(p, axis=-1) * np.linalg.norm(q, axis=-1)
    ref = np.where(den > 0, num / np.where(den > 0, den, 1), 0)
    S = ops.token_similarity(P, I, LV)
    assert np.abs(S - ref).max() <= 2 ** -22


def test_similarity_drop_counts_order_and_ties():
    rng = np.random.default_rng(5)
    P = rng.integers(0, 64000, (2, 4, 7, 11))
    I = rng.integers(0, 64000, (2, 1, 7, 11))
    S = ops.token_similarity(P, I, LV)
    n = 7 * 11
    for rate in (0.0, 0.1, 0.25, 0.5, 1.0):
        d = ops.similarity_drop(P, I, LV, rate)
        k = min(n, int(np.floor(float(np.float32(rate)) * n)))
        assert (d.sum(axis=(2, 3)) == k).all()
        for b in range(2):
            for t in range(4):
                s, m = S[b, t], d[b, t]
                if 0 < k < n:
                    assert s[m].min() >= s[~m].max()    # tau separates dropped from kept
    # all similarities equal (P = I everywhere): the lowest linear indices go first
    P2 = np.repeat(I, 3, axis=1)
    d2 = ops.similarity_drop(P2, I, LV, 0.3)
    k = int(np.floor(float(np.float32(0.3)) * n))
    flat = d2.reshape(2, 3, n)
    assert (flat[..., :k]).all() and not (flat[..., k:]).any()
    # among equal S at the threshold, the lower index is dropped, the higher kept
    s = S[0, 0].reshape(-1).copy()
    P3 = P.copy()
    P3[0, 0].reshape(-1)[[10, 20]] = I[0, 0].reshape(-1)[[10, 20]]   # two tokens with S = 1
    d3 = ops.similarity_drop(P3, I, LV, 1.0 / n + 1e-7)             # k = 1
    assert d3[0, 0].reshape(-1)[10] and not d3[0, 0].reshape(-1)[20]


# ------------------------------------------------------------- pixel residuals (Eq. 4)

def test_residual_mean_closed_forms():
    """A residual constant in time averages to itself; a residual linear in t averages to
    its value at the window's mid-time; windows tile the clip with a shorter last one;
    |r| < theta is zeroed and |r| >= theta kept."""
    rng = np.random.default_rng(0)
    N, T, H, W, C = 2, 7, 3, 5, 3
    xh = rng.standard_normal((N, T, H, W, C)).astype(np.float32)
    c = (rng.integers(-8, 9, (N, 1, H, W, C)) / 8).astype(np.float32)          # exact in float32
    r = ops.residual_mean(xh + c, xh, 3, 0.0)
    assert ops.residual_windows(7, 3) == [(0, 3), (3, 6), (6, 7)]
    assert r.shape == (N, 3, H, W, C)
    assert np.abs(r - c).max() <= 1e-6
    ramp = (np.arange(T, dtype=np.float32)[None, :, None, None, None] * 0.25).astype(np.float32)
    r2 = ops.residual_mean(xh * 0 + ramp, xh * 0, 4, 0.0)                      # windows [0,4), [4,7)
    assert np.allclose(r2[:, 0], 0.25 * 1.5) and np.allclose(r2[:, 1], 0.25 * 5.0)
    r3 = ops.residual_mean(xh * 0 + ramp, xh * 0, 4, 0.375)
    assert (r3[:, 0] == 0.375).all() and (r3[:, 1] == 1.25).all()
    r4 = ops.residual_mean(xh * 0 + ramp, xh * 0, 4, 0.376)
    assert (r4[:, 0] == 0).all()


def test_residual_sparse_round_trip_and_apply():
    """dense -> sparse -> apply: every frame of a window gets its residual; with theta 0
    and a residual constant over time the receiver recovers x exactly."""
    rng = np.random.default_rng(1)
    N, T, H, W, C = 2, 6, 4, 5, 3
    xh = (rng.integers(-64, 64, (N, T, H, W, C)) / 32).astype(np.float32)
    c = (rng.integers(-8, 9, (N, 1, H, W, C)) / 8).astype(np.float32)
    c[rng.random(c.shape) < 0.5] = 0
    x = xh + c
    r = ops.residual_mean(x, xh, 3, 0.0)
    pos, val, offs = ops.residual_sparse(r)
    assert offs[-1] == len(pos) == np.count_nonzero(r)
    dense = np.zeros(r.reshape(N * 2, -1).shape, dtype=np.float32)
    for s in range(N * 2):
        dense[s, pos[offs[s]:offs[s + 1]]] = val[offs[s]:offs[s + 1]]
    assert np.array_equal(dense.reshape(r.shape), r)
    assert (np.diff(pos[offs[0]:offs[1]]) > 0).all()
    assert np.array_equal(ops.residual_apply(xh, pos, val, offs, 3), x)


# ------------------------------------------------------- GoP boundary smoothing (Eq. 1, 2)

def test_gop_blend_weights():
    """a_i = (n - i)/n: frame n is the current frame unchanged, frame 1 is mostly the
    previous GoP's frame T-n+1; weights sum to one (blending equal frames is the identity);
    frames past n are untouched."""
    rng = np.random.default_rng(0)
    N, T, H, W, C, n = 2, 6, 3, 4, 3, 3
    prev = rng.standard_normal((N, T, H, W, C))
    curr = rng.standard_normal((N, T, H, W, C))
    out = ops.gop_blend(prev, curr, n)
    assert np.array_equal(out[:, n - 1], curr[:, n - 1])
    assert np.allclose(out[:, 0], (2 / 3) * prev[:, T - 3] + (1 / 3) * curr[:, 0])
    assert np.allclose(out[:, 1], (1 / 3) * prev[:, T - 2] + (2 / 3) * curr[:, 1])
    assert np.array_equal(out[:, n:], curr[:, n:])
    same = np.repeat(curr[:, :1], T, axis=1)
    assert np.allclose(ops.gop_blend(same, same, n), same)


def test_temporal_loss_closed_form_and_finite_differences():
    rng = np.random.default_rng(1)
    N, T, H, W, C, n = 2, 5, 3, 4, 3, 2
    xp = rng.standard_normal((N, T, H, W, C))
    c = 0.5
    xc = np.zeros((N, T, H, W, C))
    xc[:, :n] = xp[:, T - n:] + c                     # every boundary difference is c
    L, g = ops.temporal_loss(xc, xp, n)
    assert abs(L - c * np.sqrt(H * W * C)) < 1e-12
    assert not g[:, n:].any()
    xc = rng.standard_normal((N, T, H, W, C))
    L, g = ops.temporal_loss(xc, xp, n)
    h = 1e-6
    for idx in [(0, 0, 1, 2, 1), (1, 1, 2, 0, 0), (0, 1, 0, 3, 2), (1, 3, 1, 1, 1)]:
        e = np.zeros_like(xc)
        e[idx] = h
        fd = (ops.temporal_loss(xc + e, xp, n)[0] - ops.temporal_loss(xc - e, xp, n)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 + 1e-6 * abs(g[idx])


# ---------------------------------------------------------------- RSA resize (Sec. 5)

def test_round_to_bf16_matches_torch_cast():
    """The oracle's bfloat16 rounding against torch's CPU float32 -> bfloat16 cast,
    on random values, exact half-way ties (both parities), and special values."""
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000)).astype(np.float32)
    base = rng.integers(0, 2 ** 31, 4000, dtype=np.uint64).astype(np.uint32)
    ties = ((base & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)   # remainder exactly 1/2
    near = ((base & np.uint32(0xFFFF0000)) | np.uint32(0x7FFF)).view(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 3.4028235e38, -3.4028235e38, 1e-40, -1e-45,
                        1.0, 1.00390625, 1.005859375], dtype=np.float32)
    x = np.concatenate([v, ties, near, special])
    x = x[np.isfinite(x) | np.isinf(x)]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = ops.round_to_bf16(x)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert np.isnan(ops.round_to_bf16(np.array([np.nan], np.float32))).all()


def test_box_downsample_hand_example():
    x = np.arange(16, dtype=np.float32).reshape(1, 4, 4, 1)
    y = ops.box_downsample(x, 2)
    assert np.array_equal(y[0, :, :, 0], np.array([[2.5, 4.5], [10.5, 12.5]], np.float32))
    y3 = ops.box_downsample(np.arange(81, dtype=np.float32).reshape(1, 9, 9, 1), 3)
    # block means of a 9x9 ramp: the centre values 10, 13, 16 / 37, 40, 43 / 64, 67, 70
    assert np.array_equal(y3[0, :, :, 0], np.array([[10, 13, 16], [37, 40, 43], [64, 67, 70]], np.float32))


@pytest.mark.parametrize("s", [1, 2, 3])
def test_box_downsample_against_avg_pool(s):
    """Float input: equal to torch's avg_pool2d (kernel = stride = s, floor mode) in float64,
    up to float32 rounding; trailing rows / columns take no part."""
    rng = np.random.default_rng(s)
    x = rng.uniform(-1, 1, (3, 20, 31, 3)).astype(np.float32)
    y = ops.box_downsample(x, s)
    ref = F.avg_pool2d(torch.from_numpy(x.astype(np.float64)).permute(0, 3, 1, 2), s, s).permute(0, 2, 3, 1).numpy()
    assert y.shape == (3, 20 // s, 31 // s, 3)
    assert np.abs(y - ref).max() <= 4e-7 * s * s
    if s == 1:
        assert np.array_equal(y, x)
    x2 = x.copy()
    x2[:, (20 // s) * s:] = 99.0
    x2[:, :, (31 // s) * s:] = -99.0
    assert np.array_equal(ops.box_downsample(x2, s), y)


def test_box_downsample_linear_ramp_and_constants():
    """The mean of a linear function over a block is its value at the block centre."""
    s = 3
    h, w = np.meshgrid(np.arange(12), np.arange(15), indexing="ij")
    x = (0.25 * h - 0.125 * w + 0.5).astype(np.float32)[None, :, :, None]
    y = ops.box_downsample(x, s)[0, :, :, 0]
    ho, wo = np.meshgrid(np.arange(4), np.arange(5), indexing="ij")
    ref = 0.25 * (s * ho + 1) - 0.125 * (s * wo + 1) + 0.5
    assert np.abs(y - ref).max() <= 1e-6
    c = np.full((2, 9, 9, 3), 0.3, np.float32)
    assert np.array_equal(ops.box_downsample(c, 3, out_bf16=True), np.full((2, 3, 3, 3), ops.round_to_bf16(
        np.float32(0.3 * 9) / np.float32(9)), np.float32))


def test_box_downsample_u8_mapping():
    """uint8 input: the block mean mapped to [-1, 1] (m / 127.5 - 1): 0 -> -1, 255 -> 1,
    a 2x2 block {0, 255, 255, 0} -> 0; random blocks against the float64 definition."""
    assert np.array_equal(ops.box_downsample(np.zeros((1, 4, 4, 3), np.uint8), 2), np.full((1, 2, 2, 3), -1, np.float32))
    assert np.array_equal(ops.box_downsample(np.full((1, 6, 6, 3), 255, np.uint8), 3), np.ones((1, 2, 2, 3), np.float32))
    b = np.array([[0, 255], [255, 0]], np.uint8)[None, :, :, None]
    assert ops.box_downsample(b, 2)[0, 0, 0, 0] == 0.0
    rng = np.random.default_rng(4)
    x = rng.integers(0, 256, (2, 30, 33, 3), dtype=np.uint8)
    for s in (2, 3):
        ref = F.avg_pool2d(torch.from_numpy(x.astype(np.float64)).permute(0, 3, 1, 2), s, s).permute(0, 2, 3, 1).numpy()
        assert np.abs(ops.box_downsample(x, s) - (ref / 127.5 - 1)).max() <= 3e-7
