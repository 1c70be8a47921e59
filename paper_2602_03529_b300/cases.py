"""Fixed workloads for profiling runs (ncu captures name these commands).

    python -m paper_2602_03529_b300.cases clip  [--N 1 --T 5 --H 720 --W 1280]
        one encode + decode of a seeded blurred-noise clip, BF16
    python -m paper_2602_03529_b300.cases train [--N 2 --T 17 --H 256 --W 256]
        one training step (forward with 10% drop, MSE, backward, SGD), then one
        more forward + backward
    python -m paper_2602_03529_b300.cases downsample [--N 4 --T 17 --H 1080 --W 1920 --s 3]
        three s x s area downsamples of seeded uint8 frames to bf16 (the
        resolution control of the 1080p encoder input)

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


def downsample(N: int, T: int, H: int, W: int, s: int) -> None:
    import numpy as np
    import torch

    from . import downsample as ds

    x = torch.from_numpy(np.random.default_rng(8).integers(0, 256, (N, T, H, W, 3), dtype=np.uint8)).cuda()
    y = ds(x, s, torch.bfloat16)
    for _ in range(2):
        ds(x, s, torch.bfloat16, out=y)
    torch.cuda.synchronize()
    print("downsample ok", tuple(y.shape))


def select(N: int, T: int, H: int, W: int) -> None:
    """Token selection over N streams x T P latent frames of H x W tokens (half of the P
    tokens equal to the I token at their position), drop rate 0.25."""
    import numpy as np
    import torch

    from . import similarity_mask

    rng = np.random.default_rng(5)
    ii = rng.integers(0, 64000, (N, 1, H, W))
    ip = np.where(rng.random((N, T, H, W)) < 0.5, np.repeat(ii, T, axis=1), rng.integers(0, 64000, (N, T, H, W)))
    dp = torch.from_numpy(ip.astype(np.int32)).cuda()
    di = torch.from_numpy(ii.astype(np.int32)).cuda()
    for _ in range(3):
        out, kb, _ = similarity_mask(dp, di, 0.25)
    torch.cuda.synchronize()
    print("select ok", tuple(out.shape), int((out == 32036).sum()))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["clip", "train", "downsample", "select"])
    ap.add_argument("--N", type=int)
    ap.add_argument("--T", type=int)
    ap.add_argument("--H", type=int)
    ap.add_argument("--W", type=int)
    ap.add_argument("--s", type=int, default=3)
    a = ap.parse_args()
    dflt = {"clip": (1, 5, 720, 1280), "train": (2, 17, 256, 256), "downsample": (4, 17, 1080, 1920),
            "select": (256, 4, 90, 160)}[a.case]
    shape = [v if v is not None else d for v, d in zip((a.N, a.T, a.H, a.W), dflt)]
    if a.case == "downsample":
        downsample(*shape, a.s)
    elif a.case == "select":
        select(*shape)
    else:
        (clip if a.case == "clip" else train)(*shape)


if __name__ == "__main__":
    main()
