"""B300-native causal video tokenizer (encoder f_phi, FSQ, packet-drop
masking, decoder g_theta) behind a C-ABI library of sm_103a CUDA kernels.

``_lib`` is the ctypes binding of include/tok.h; ``tokenizer`` is a thin
torch-tensor front end. Importing this package does not load the CUDA
library; the first call that needs it does, and fails loudly if it has not
been built.
"""
from . import _lib  # noqa: F401
from .tokenizer import (Tokenizer, conv3d, dequantize, groupnorm_silu, drop_mask, make_arch, pack_rows, quantize,  # noqa: F401
                        similarity_mask, residual, residual_sparse, residual_apply, gop_blend, temporal_loss, downsample,
                        unpack_rows, zero_index)
