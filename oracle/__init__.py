"""The oracle: a plain, slow FP64 CPU tokenizer that the CUDA path is checked against.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
link anything in this package. The product path (the C-ABI library and its
Python binding) never does, and this package imports nothing from it.

Contents:
  conv3d.c   FP64 direct-loop causal conv (forward, dgrad, wgrad), OpenMP
  ops.py     GroupNorm, SiLU, FSQ, Philox-4x32-10, drop mask, row packets,
             depth-to-space, edge padding
  model.py   the tokenizer's layer list, encoder, decoder
  grad.py    the analytic FP64 gradient of the straight-through surrogate

Pins (tests that fix the oracle to something other than itself) live in
``tests/test_oracle_*.py``. Functions without such a pin are listed as
"parity unpinned" in their docstrings; currently there are none.
"""
from . import ops  # noqa: F401
from .model import Arch, Oracle, latent_shape, param_spec  # noqa: F401
