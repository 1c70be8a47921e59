"""GroupNorm+SiLU without a workspace (tok_groupnorm_silu_noalloc).

Callers that cannot allocate device memory (a host callback, a real-time
thread that must not enter the allocator, an embedding with a fixed memory
budget) use this entry point; it keeps its scratch in a fixed array inside the
library instead of a caller-provided workspace. These tests call it through
the C-ABI and compare it with tok_groupnorm_silu, the entry point that takes a
workspace, with the tolerances of the other GroupNorm tests, on two calls in
a row (the second sees the first call's leftovers in the shared scratch).

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2602_03529_b300 import _lib
    _lib.load()
    return _lib


def _ptr(t):
    return None if t is None else t.data_ptr()


def _with_workspace(L, prec, x, G, g, b, eps):
    N, T, H, W, C = x.shape
    y = torch.empty_like(x)
    nb = L.tok_groupnorm_workspace_bytes(prec, N * T, H * W, C, G)
    ws = torch.empty(nb, device="cuda", dtype=torch.uint8)
    L.tok_groupnorm_silu(prec, _ptr(x), N * T, H * W, C, G, _ptr(g), _ptr(b), eps, _ptr(y), _ptr(ws), nb,
                         torch.cuda.current_stream().cuda_stream)
    return y


def _no_alloc(L, prec, x, G, g, b, eps):
    N, T, H, W, C = x.shape
    y = torch.empty_like(x)
    L.tok_groupnorm_silu_noalloc(prec, _ptr(x), N * T, H * W, C, G, _ptr(g), _ptr(b), eps, _ptr(y),
                                 torch.cuda.current_stream().cuda_stream)
    return y


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_matches_workspace_entry_on_two_calls(L, prec):
    code = L.TOK_BF16 if prec == "bf16" else L.TOK_FP32
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    rng = np.random.default_rng(21)
    # two different problems back to back: the second call reuses the shared scratch
    for shape, G in [((1, 5, 36, 64, 128), 32), ((2, 3, 17, 20, 256), 32)]:
        C = shape[-1]
        x = torch.from_numpy((rng.standard_normal(shape) * 1.5 + 0.3).astype(np.float32)).to("cuda", dt)
        g = torch.from_numpy((1 + 0.1 * rng.standard_normal(C)).astype(np.float32)).cuda()
        b = torch.from_numpy((0.1 * rng.standard_normal(C)).astype(np.float32)).cuda()
        ref = _with_workspace(L, code, x, G, g, b, 1e-6).float()
        got = _no_alloc(L, code, x, G, g, b, 1e-6).float()
        torch.cuda.synchronize()
        err = (got - ref).abs()
        tol = (2.0 ** -8 * ref.abs() + 4e-3) if prec == "bf16" else (1e-5 * (ref.abs() + 1.0))
        assert bool((err <= tol).all()), float(err.max())


def test_refuses_problems_larger_than_its_scratch(L):
    frames, HW, C, G = 4096, 1 << 16, 512, 32
    need = L.tok_groupnorm_workspace_bytes(L.TOK_BF16, frames, HW, C, G)
    assert need > (4 << 20)
    with pytest.raises(L.TokError) as e:
        # never launched: the size check comes first, so the pointers are not read
        L.tok_groupnorm_silu_noalloc(L.TOK_BF16, 16, frames, HW, C, G, None, None, 1e-6, 16,
                                     torch.cuda.current_stream().cuda_stream)
    assert e.value.code == L.TOK_ENOMEM
