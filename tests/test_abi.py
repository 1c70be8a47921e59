"""The C-ABI library loads and exports every entry point include/tok.h declares
(no compute calls: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tok.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tok_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_03529_b300 import build
    path = build.build()
    from paper_2602_03529_b300 import _lib
    _lib.load()
    return path


def test_header_declares_the_hot_path(lib):
    d = _declared()
    for name in ["tok_encode", "tok_quantize", "tok_drop_mask", "tok_decode", "tok_pack_rows",
                 "tok_unpack_rows", "tok_conv3d", "tok_groupnorm_silu"]:
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tok_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_2602_03529_b300 import _lib
    assert sorted(_lib.exported_names()) == _declared()


def test_host_only_entry_points(lib):
    from paper_2602_03529_b300 import _lib as L
    assert L.tok_zero_index([8, 8, 8, 5, 5, 5]) == 32036
    assert L.tok_zero_index([2, 3]) == 1 + 2
    assert L.tok_strerror(L.TOK_ETIMEOUT) == "device-side bounded wait timed out"
    a = L.tok_arch_default()
    assert list(a.ch)[:3] == [128, 256, 512] and list(a.levels)[:6] == [8, 8, 8, 5, 5, 5]
    assert L.tok_conv3d_workspace_bytes(L.TOK_BF16, 128, 128, 3) == 128 * 27 * 128 * 2
    assert L.tok_conv3d_workspace_bytes(L.TOK_FP32, 3, 12, 3) == 256 * ((16 * 88 * 4 + 255) // 256)


def test_create_needs_a_device(lib):
    import torch
    from paper_2602_03529_b300 import _lib as L
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.TokError) as e:
        L.tok_create(L.tok_arch_default(), L.TOK_BF16)
    assert e.value.code == L.TOK_EDEVICE


def test_arch_validation_is_host_side(lib):
    from paper_2602_03529_b300 import _lib as L
    a = L.tok_arch_default()
    a.nlev = 9
    with pytest.raises(L.TokError) as e:
        L.tok_create(a, L.TOK_BF16)
    assert e.value.code == L.TOK_EINVAL
    a = L.tok_arch_default()
    a.ch[0] = 96  # not a multiple of 64: no BF16 tensor-core path
    with pytest.raises(L.TokError) as e:
        L.tok_create(a, L.TOK_BF16)
    assert e.value.code == L.TOK_EINVAL
