"""The streaming server on the GPU: continuous batching over several lanes with
chunks of different streams in flight together (and, in the second form,
grouped into one launch per layer, with an urgent lane on the highest stream
priority), and every stream's tokens and decoded frames bitwise the same when
it is served alone and in the mix."""
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu
ARCH = dict(ch=(64, 128, 256), blocks=1)
RES = [(48, 64), (64, 96), (40, 56)]


def _svc(spec):
    # pretend the 64x96 streams are too large for the target: background class
    return 0.050 if (spec.H, spec.W) == RES[1] else 0.001


def _run(specs, lanes, params, max_batch=1, classes=False, memory=None):
    """memory: None for a fixed table of 2 slots per resolution, else a byte budget for
    slots opened on demand (MemoryPool)."""
    from paper_2602_03529_b300.serve import GpuExecutor, MemoryPool, Server
    if memory is None:
        slots = {r: 2 for r in RES}
        ex = GpuExecutor(lanes, params, slots, keep_outputs=True, arch=ARCH, max_batch=max_batch,
                         priorities=classes)
    else:
        ex = GpuExecutor(lanes, params, None, keep_outputs=True, arch=ARCH, max_batch=max_batch,
                         priorities=classes, resolutions=RES)
        slots = MemoryPool(ex, memory)
    rep = Server(ex, lanes, slots, 1e30, stall_timeout=5.0, service_time=_svc if classes else None,
                 max_batch=max_batch).run(specs, horizon=2.0)
    torch.cuda.synchronize()
    assert all(s == 0 for s in ex.status())
    outs = {k: torch.cat(v, 1) for k, v in ex.outputs.items()}
    toks = {k: torch.cat(v, 1) for k, v in ex.tokens.items()}
    ex.close()
    return rep, outs, toks


@pytest.mark.parametrize("max_batch,classes", [(1, False), (3, True)])
def test_alone_equals_mix(max_batch, classes):
    import paper_2602_03529_b300 as P
    from paper_2602_03529_b300.serve import StreamSpec
    tk = P.Tokenizer("bf16", **ARCH)
    params = S.weights_for(tk.param_spec(), seed=5)
    tk.close()
    specs = [StreamSpec(i, *RES[i % 3], start=0.004 * i, n_chunks=4) for i in range(6)]
    rep, out_mix, tok_mix = _run(specs, 3 if not classes else 2, params, max_batch, classes)
    assert rep["chunks"] == 24 and rep["admitted_total"] == 6 and rep["timed_out"] == 0
    assert rep["max_concurrent"] >= 2
    for s in specs:
        assert out_mix[s.sid].shape == (1, 13, s.H, s.W, 3)
    for s in specs[:3]:
        _, out1, tok1 = _run([StreamSpec(s.sid, s.H, s.W, 0.0, 4)], 1, params)
        assert torch.equal(tok1[s.sid], tok_mix[s.sid])
        assert torch.equal(out1[s.sid], out_mix[s.sid])


def test_memory_admission_on_the_device():
    """Slots opened by a MemoryPool on the device: a budget of two streams' bytes
    admits two streams at a time, reuses the freed caches for the next stream of the
    same resolution (reset to chunk 0), and every stream's output equals its output
    served alone."""
    import paper_2602_03529_b300 as P
    from paper_2602_03529_b300.serve import GpuExecutor, StreamSpec
    tk = P.Tokenizer("bf16", **ARCH)
    params = S.weights_for(tk.param_spec(), seed=5)
    tk.close()
    probe = GpuExecutor(1, params, None, arch=ARCH, resolutions=[RES[0]])
    two = 2 * probe.stream_bytes(RES[0]) + 1
    probe.close()
    specs = [StreamSpec(i, *RES[0], start=0.004 * i, n_chunks=3) for i in range(4)]
    rep, out_mix, tok_mix = _run(specs, 2, params, memory=two)
    assert rep["chunks"] == 12 and rep["admitted_total"] == 4 and rep["max_concurrent"] == 2
    for s in specs:
        _, out1, tok1 = _run([StreamSpec(s.sid, s.H, s.W, 0.0, 3)], 1, params)
        assert torch.equal(tok1[s.sid], tok_mix[s.sid])
        assert torch.equal(out1[s.sid], out_mix[s.sid])
