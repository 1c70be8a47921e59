"""End-to-end parity of the tokenizer (encode -> FSQ indices, decode) against
the FP64 oracle, through the C-ABI, on both precision paths.

Index parity (the target: bit-exact away from rounding ties). For every token
the margin m = min_i |frac(b_i) - 0.5| of the oracle's bounded latent b to the
nearest rounding boundary is computed. The band is a fixed constant per
comparison, set from the latent error each path is allowed (never from the
error of the case under test); tokens with m > band must match exactly, and
the mismatches inside the band are bounded as a fraction of the tokens:
  FP32 path vs the FP64 oracle: band 2e-4 (FP32 z error <= 5e-5 measured,
    |db/dz| <= h <= 3.5), mismatches <= 1e-4 of the tokens;
  BF16 path, against the exact FP64 oracle and against the BF16-activation
    oracle (every stored activation rounded to bf16 as the GPU stores it):
    band 0.1 (the bounded values of the BF16 path differ from either oracle's
    by at most 0.08 on these cases: bf16 rounding of ~30 stored activations,
    reading 10), mismatches <= 10% of the tokens + 3. On the single-stage
    case (9216 tokens, two bf16 roundings before the latent) the
    BF16-activation oracle removes most of the difference: mismatches
    <= 0.2% of the tokens against it (measured 0.04%), <= 5% against the
    exact oracle (measured 2%). In the deeper networks the two oracles sit
    equally far from the GPU (the rounding decisions that the accumulation
    order flips spread through the layers as far as the rounding itself).

Latent / reconstruction error bounds (max-abs, on [-1,1]-scale outputs):
  FP32 path  z: 1e-3, x_hat: 1e-3       (FP32 accumulation through ~30 convs)
  BF16 path  z: 0.15, x_hat: 0.10       (bf16 activations between layers)
The decoder is compared on identical indices (the oracle's).
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import Arch, Oracle, ops, param_spec

pytestmark = pytest.mark.gpu
LV = (8, 8, 8, 5, 5, 5)
TOL = {"fp32": {"z": 1e-3, "x": 1e-3}, "bf16": {"z": 0.15, "x": 0.10}}
BAND_FP32, MISMATCH_FP32 = 2e-4, 1e-4
BAND_BF16, MISMATCH_BF16 = 0.1, 0.1


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def index_parity(idx_gpu, z_gpu, b_ref, idx_ref, band, levels=LV):
    b_gpu = ops.fsq_bound(z_gpu.astype(np.float64), levels)
    frac = b_ref - np.floor(b_ref)
    margin = np.abs(frac - 0.5).min(axis=-1)
    mism = idx_gpu != idx_ref
    return dict(band=band, b_err=float(np.abs(b_gpu - b_ref).max()), mismatches=int(mism.sum()),
                out_of_band=int((mism & (margin > band)).sum()), in_band_tokens=int((margin <= band).sum()),
                tokens=int(mism.size))


def check_indices(prec, rep):
    """The index assertions of a case (see the module docstring)."""
    n = rep["tokens"]
    if prec == "fp32":
        assert rep["out_of_band"] == 0
        assert rep["mismatches"] <= MISMATCH_FP32 * n
    else:
        for r in (rep, rep["vs_bf16_oracle"]):
            assert r["out_of_band"] == 0, r
            assert r["mismatches"] <= MISMATCH_BF16 * n + 3, r


def run_case(P, prec, arch_kw, oarch, N, T, H, W, seed=0, decode=True):
    tk = P.Tokenizer(prec, **arch_kw)
    spec = tk.param_spec()
    assert [(n, tuple(s)) for n, s, _ in spec] == [(n, tuple(s)) for n, s, _ in param_spec(oarch)]
    params = S.weights_for(spec, seed=seed)
    tk.set_params(params)
    x = S.blurred_noise_clip(seed, N, T, H, W)
    if prec == "bf16":
        x = S.to_bf16_f32(x)
        p_or = {k: S.to_bf16_f32(v) for k, v in params.items()}
    else:
        p_or = params
    orc = Oracle(oarch, p_or)
    idx_ref, z_ref, b_ref = orc.encode(x)
    tk.reserve(N, T, H, W)
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    z, idx = tk.encode(torch.from_numpy(x).to("cuda", dt))
    torch.cuda.synchronize()
    assert tk.status() == 0
    z = z.cpu().numpy()
    idx = idx.cpu().numpy()
    rep = index_parity(idx, z, b_ref, idx_ref, BAND_FP32 if prec == "fp32" else BAND_BF16)
    rep["z_err"] = float(np.abs(z - z_ref).max())
    if prec == "bf16":
        i16, z16, b16 = Oracle(oarch, p_or, act_bf16=True).encode(x)
        rep["vs_bf16_oracle"] = index_parity(idx, z, b16, i16, BAND_BF16)
        rep["vs_bf16_oracle"]["z_err"] = float(np.abs(z - z16).max())
    if decode:
        xh_ref = orc.decode(idx_ref, H, W)
        xh = tk.decode(torch.from_numpy(idx_ref.astype(np.int32)).cuda(), H, W)
        torch.cuda.synchronize()
        rep["x_err"] = float(np.abs(xh.cpu().numpy() - xh_ref).max())
        rep["x_shape_ok"] = xh.shape == xh_ref.shape
    assert tk.check_guards() == 0
    tk.close()
    return rep


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_stage_cfg0(P, prec):
    """Single encoder stage + FSQ, 1x3x9x64x64 (the plain-FP32 stage config)."""
    rep = run_case(P, prec, dict(kind="stage", ch=(64, 128)), Arch(kind="stage", ch=(64, 128)),
                   1, 9, 64, 64, seed=0, decode=False)
    print(prec, rep)
    check_indices(prec, rep)
    assert rep["z_err"] <= TOL[prec]["z"]
    if prec == "bf16":
        assert rep["vs_bf16_oracle"]["mismatches"] <= 0.002 * rep["tokens"], rep
        assert rep["mismatches"] <= 0.05 * rep["tokens"], rep


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", [(1, 9, 32, 48), (2, 5, 24, 40), (1, 5, 20, 30)])
def test_small_tokenizer(P, prec, shape):
    """Full architecture with narrow channels; ragged H/W (edge pad + crop)."""
    kw = dict(ch=(64, 128, 256), blocks=1)
    rep = run_case(P, prec, kw, Arch(ch=(64, 128, 256), blocks=1), *shape, seed=1)
    print(prec, shape, rep)
    assert rep["x_shape_ok"]
    check_indices(prec, rep)
    assert rep["z_err"] <= TOL[prec]["z"]
    assert rep["x_err"] <= TOL[prec]["x"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_default_tokenizer_64px(P, prec):
    """The 128/256/512, 2-blocks-per-level tokenizer on a 1x3x9x64x64 clip."""
    rep = run_case(P, prec, {}, Arch(), 1, 9, 64, 64, seed=2)
    print(prec, rep)
    check_indices(prec, rep)
    assert rep["z_err"] <= TOL[prec]["z"]
    assert rep["x_err"] <= TOL[prec]["x"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", [(1, 17, 32, 48), (2, 9, 24, 40)])
def test_8x8x8_tokenizer(P, prec, shape):
    """The 8x temporal / 8x8 spatial setting (Sec. 4.1): stem stride (2,2,2), pixel head
    with depth-to-space (2,2,2); 8 frames per latent frame, ragged H/W."""
    kw = dict(ch=(64, 128, 256), blocks=1, t_stem=2)
    rep = run_case(P, prec, kw, Arch(ch=(64, 128, 256), blocks=1, t_stem=2), *shape, seed=5)
    print(prec, shape, rep)
    assert rep["x_shape_ok"]
    check_indices(prec, rep)
    assert rep["z_err"] <= TOL[prec]["z"]
    assert rep["x_err"] <= TOL[prec]["x"]


def test_t_stem_validation(P):
    from paper_2602_03529_b300 import _lib as L
    with pytest.raises(L.TokError) as e:
        P.Tokenizer("bf16", ch=(64, 128, 256), blocks=1, t_stem=3)
    assert e.value.code == L.TOK_EINVAL
    tk = P.Tokenizer("bf16", ch=(64, 128, 256), blocks=1, t_stem=2)
    assert tk.s_t == 8
    assert tuple(tk.latent_shape(17, 64, 64)) == (3, 8, 8)
    with pytest.raises(L.TokError) as e:
        tk.latent_shape(13, 64, 64)        # a clip's T - 1 must be a multiple of 8
    assert e.value.code == L.TOK_ESHAPE
    assert tk.check_guards() == 0
    tk.close()
