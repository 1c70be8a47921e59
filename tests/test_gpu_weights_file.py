"""Checkpoint / resume on the device: a context saved to a weights file and created
again from it has bitwise the same parameters and encodes bitwise the same tokens, on
both precision paths; a training run resumed from a file continues as the original
does; a corrupted payload is refused (hash)."""
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu
KW = dict(ch=(64, 128, 256), blocks=1)


@pytest.fixture(scope="module")
def P():
    import paper_2602_03529_b300 as P
    P._lib.load()
    return P


def _flat(P, tk):
    from paper_2602_03529_b300 import _lib as L
    n = L.tok_param_total(tk.ctx)
    out = torch.empty(n, device="cuda", dtype=torch.float32)
    L.tok_get_params(tk.ctx, out.data_ptr(), None)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_save_and_create_from_file(P, tmp_path, prec):
    tk = P.Tokenizer(prec, **KW)
    tk.set_params(S.weights_for(tk.param_spec(), seed=6))
    f = str(tmp_path / "w.tokw")
    tk.save(f)
    tk2 = P.Tokenizer.from_file(f, prec)
    assert tk2.arch_kw["ch"] == KW["ch"] and tk2.arch_kw["blocks"] == 1 and tk2.levels == tk.levels
    assert torch.equal(_flat(P, tk), _flat(P, tk2))
    N, T, H, W = 1, 5, 32, 48
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    x = torch.from_numpy(S.blurred_noise_clip(2, N, T, H, W)).to("cuda", dt)
    outs = []
    for t in (tk, tk2):
        t.reserve(N, T, H, W)
        z, idx = t.encode(x)
        xh = t.decode(idx, H, W)
        torch.cuda.synchronize()
        assert t.status() == 0
        outs.append((z.clone(), idx.clone(), xh.clone()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    tk.close()
    tk2.close()


def test_resumed_training_continues_bitwise(P, tmp_path):
    from paper_2602_03529_b300.train import Trainer
    N, T, H, W = 1, 5, 32, 32
    x = torch.from_numpy(S.blurred_noise_clip(4, N, T, H, W)).to("cuda", torch.bfloat16)
    tk = P.Tokenizer("bf16", **KW)
    tk.set_params(S.weights_for(tk.param_spec(), seed=8))
    tr = Trainer(tk, N, T, H, W)
    for i in range(2):
        tr.step(x, 0.1, 1, i, lr=0.05)
    f = str(tmp_path / "ckpt.tokw")
    tk.save(f)
    l_a = [float(tr.step(x, 0.1, 1, i, lr=0.05).item()) for i in (2, 3)]
    p_a = _flat(P, tk)
    tk2 = P.Tokenizer.from_file(f, "bf16")
    tr2 = Trainer(tk2, N, T, H, W)
    l_b = [float(tr2.step(x, 0.1, 1, i, lr=0.05).item()) for i in (2, 3)]
    p_b = _flat(P, tk2)
    assert tk.status() == 0 and tk2.status() == 0
    assert l_a == l_b
    assert torch.equal(p_a, p_b)
    tk.close()
    tk2.close()


def test_corrupted_payload_is_refused(P, tmp_path):
    from paper_2602_03529_b300 import _lib as L
    tk = P.Tokenizer("bf16", **KW)
    tk.set_params(S.weights_for(tk.param_spec(), seed=9))
    f = tmp_path / "w.tokw"
    tk.save(str(f))
    tk.close()
    b = bytearray(f.read_bytes())
    b[104 + 4 * 1000 + 1] ^= 0x10  # one bit of one parameter
    f.write_bytes(bytes(b))
    L.tok_read_weights_header(str(f))  # the header is still well formed
    with pytest.raises(L.TokError) as e:
        P.Tokenizer.from_file(str(f), "bf16")
    assert e.value.code == L.TOK_EFILE
