"""Fixed workloads for profiling runs (ncu captures name these commands).

    python -m paper_2602_03529_b300.cases clip  [--N 1 --T 5 --H 720 --W 1280]
        one encode + decode of a seeded blurred-noise clip, BF16
    python -m paper_2602_03529_b300.cases train [--N 2 --T 17 --H 256 --W 256]
        one training step (forward with 10% drop, MSE, backward, SGD), then one
        more forward + backward

Inputs come from the seeded generators in `synthetic`; weights are He-normal
from seed 0. Both exit non-zero if the library's device status word reports
an error.
"""
from __future__ import annotations

import argparse
import sys


def clip(N: int, T: int, H: int, W: int) -> None:
    import torch

    import synthetic as S
    from . import Tokenizer

    tk = Tokenizer("bf16")
    tk.set_params(S.weights_for(tk.param_spec(), seed=0))
    tk.reserve(N, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(1, N, T, H, W))).to("cuda", torch.bfloat16)
    _, idx = tk.encode(x, want_z=False)
    tk.decode(idx, H, W)
    torch.cuda.synchronize()
    if tk.status() != 0:
        sys.exit(f"device status {tk.status()}")
    print("clip ok", N, T, H, W, f"{tk.workspace_bytes(N, T, H, W) / 1e9:.2f} GB workspace")


def train(N: int, T: int, H: int, W: int) -> None:
    import torch

    import synthetic as S
    from . import Tokenizer
    from .train import Trainer

    tk = Tokenizer("bf16")
    tk.set_params(S.weights_for(tk.param_spec(), seed=0))
    tr = Trainer(tk, N, T, H, W)
    x = torch.from_numpy(S.blurred_noise_clip(7, N, T, H, W)).to("cuda", torch.bfloat16)
    tr.step(x, 0.1, 1, 0, 1e-5)
    tr.forward(x, 0.1, 1, 1)
    tr.backward()
    torch.cuda.synchronize()
    if tk.status() != 0:
        sys.exit(f"device status {tk.status()}")
    print("train ok", N, T, H, W)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["clip", "train"])
    ap.add_argument("--N", type=int)
    ap.add_argument("--T", type=int)
    ap.add_argument("--H", type=int)
    ap.add_argument("--W", type=int)
    a = ap.parse_args()
    dflt = {"clip": (1, 5, 720, 1280), "train": (2, 17, 256, 256)}[a.case]
    shape = [v if v is not None else d for v, d in zip((a.N, a.T, a.H, a.W), dflt)]
    (clip if a.case == "clip" else train)(*shape)


if __name__ == "__main__":
    main()
