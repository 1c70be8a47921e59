"""Joint encoder/decoder training step through the masked decode (torch autograd front end).

The step runs entirely in the CUDA library: tok_train_forward (encode ->
Bernoulli token drop with zero fill -> decode -> MSE loss and its gradient)
and tok_backward (hand-written backward with straight-through FSQ). By
default the forward keeps only each residual block's input and the backward
rebuilds the block's interior from it (per-residual-block recomputation);
recompute=False keeps the interiors instead (more memory, no recomputed
convs, bitwise the same gradients). This module only marshals tensors:
`TokenizerLoss.apply(params, x, ...)` returns the loss as a torch scalar whose
.backward() fills params.grad through tok_backward.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .tokenizer import Tokenizer, _ptr, _stream_ptr


class _DeviceFloats:
    """n float32 values at a device address, as a CUDA array interface (for a zero-copy
    torch view; the memory stays owned by its context)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}


class Trainer:
    """Holds a view of a Tokenizer's flat FP32 parameters (the context's own memory: valid
    while the Tokenizer is open) and reserves its training workspace."""

    def __init__(self, tk: Tokenizer, N: int, T: int, H: int, W: int, recompute: bool = True):
        self.tk = tk
        self.shape = (N, T, H, W)
        L.tok_set_train_mode(tk.ctx, L.TOK_TRAIN_RECOMPUTE if recompute else L.TOK_TRAIN_KEEP)
        L.tok_reserve_train(tk.ctx, N, T, H, W)
        self.workspace_bytes = L.tok_train_workspace_bytes(tk.ctx, N, T, H, W)
        n = L.tok_param_total(tk.ctx)
        # a view of the context's own flat parameters (no copy): SGD updates them in
        # place and only the packed layouts are rebuilt
        self.params = torch.as_tensor(_DeviceFloats(L.tok_params(tk.ctx), n), device="cuda")
        self.grads = torch.zeros_like(self.params)
        self.xhat = torch.empty((N, T, H, W, 3), device="cuda", dtype=torch.float32)
        self.dxhat = torch.empty_like(self.xhat)
        self.loss = torch.zeros(1, device="cuda", dtype=torch.float32)

    def load(self, params: torch.Tensor | None = None):
        """Push the flat parameters (default: self.params, the context's own) into the
        context's device layouts."""
        p = self.params if params is None else params
        if p.data_ptr() == self.params.data_ptr():
            L.tok_repack(self.tk.ctx, _stream_ptr(None))
        else:
            L.tok_set_params_device(self.tk.ctx, _ptr(p), _stream_ptr(None))

    def forward(self, x: torch.Tensor, drop_rate: float, seed: int, step: int, keep_bits: torch.Tensor | None = None):
        """keep_bits (optional): row masks (N, T', H', ceil(W'/32)) int32 replacing the random drop."""
        N, T, H, W = self.shape
        L.tok_train_forward(self.tk.ctx, _ptr(x), N, T, H, W, float(drop_rate), int(seed), int(step),
                            _ptr(keep_bits), _ptr(self.xhat), _ptr(self.loss), _ptr(self.dxhat), _stream_ptr(None))
        return self.loss

    def backward(self, dxhat: torch.Tensor | None = None):
        d = self.dxhat if dxhat is None else dxhat
        L.tok_backward(self.tk.ctx, _ptr(d), _ptr(self.grads), _stream_ptr(None))
        return self.grads

    def sgd(self, lr: float):
        L.tok_sgd(_ptr(self.params), _ptr(self.grads), self.params.numel(), float(lr), _stream_ptr(None))
        self.load()

    def step(self, x, drop_rate, seed, step, lr):
        loss = self.forward(x, drop_rate, seed, step)
        self.backward()
        self.sgd(lr)
        return loss


class TokenizerLoss(torch.autograd.Function):
    """loss = mean((g(drop(FSQ(f(x)))) - x)^2) as an autograd node over the flat parameters."""

    @staticmethod
    def forward(ctx, params, x, trainer: Trainer, drop_rate: float, seed: int, step: int):
        trainer.load(params)
        loss = trainer.forward(x, drop_rate, seed, step)
        ctx.trainer = trainer
        return loss.clone().reshape(())

    @staticmethod
    def backward(ctx, grad_loss):
        tr = ctx.trainer
        g = tr.backward()
        if grad_loss is not None and float(grad_loss) != 1.0:
            g = g * grad_loss
        return g.clone(), None, None, None, None, None
