"""ctypes binding of the tokenizer's C-ABI (include/tok.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and forwards
plain pointers and sizes; all computation happens in the CUDA library. The
library must have been built (``python -m paper_2602_03529_b300.build``):
loading fails loudly otherwise, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmorphe_tok.so")

(TOK_OK, TOK_EINVAL, TOK_ESHAPE, TOK_ENOMEM, TOK_ECUDA, TOK_ETIMEOUT, TOK_EDEVICE, TOK_ESTATE, TOK_EFILE,
 TOK_EGUARD) = range(10)
TOK_BF16, TOK_FP32 = 1, 2
TOK_PAD_REPLICATE, TOK_PAD_ZERO = 0, 1
TOK_ARCH_FULL, TOK_ARCH_STAGE = 0, 1
TOK_PIX_U8, TOK_PIX_BF16, TOK_PIX_FP32 = 0, 1, 2


class tok_arch(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("in_ch", C.c_int),
        ("nlevels", C.c_int),
        ("ch", C.c_int * 4),
        ("blocks", C.c_int),
        ("nlev", C.c_int),
        ("levels", C.c_int * 8),
        ("gn_groups", C.c_int),
        ("gn_eps", C.c_float),
        ("time_pad", C.c_int),
        ("t_stem", C.c_int),
    ]


class tok_profile_stats(C.Structure):
    _fields_ = [
        ("conv_launches", C.c_int64), ("conv_ms", C.c_double), ("conv_flop", C.c_double),
        ("gn_launches", C.c_int64), ("gn_ms", C.c_double), ("gn_bytes", C.c_double),
        ("other_launches", C.c_int64), ("other_ms", C.c_double), ("other_bytes", C.c_double),
    ]


class tok_profile_record(C.Structure):
    _fields_ = [("cls", C.c_int), ("ms", C.c_float), ("work", C.c_double), ("name", C.c_char * 40)]


TOK_MAX_BATCH = 8


class tok_shape(C.Structure):
    _fields_ = [("N", C.c_int), ("T", C.c_int), ("H", C.c_int), ("W", C.c_int)]


class tok_enc_item(C.Structure):
    _fields_ = [("d_x", C.c_void_p), ("N", C.c_int), ("T", C.c_int), ("H", C.c_int), ("W", C.c_int),
                ("d_z", C.c_void_p), ("d_idx", C.c_void_p), ("s", C.c_void_p)]


class tok_dec_item(C.Structure):
    _fields_ = [("d_idx", C.c_void_p), ("N", C.c_int), ("Tq", C.c_int), ("Hq", C.c_int), ("Wq", C.c_int),
                ("H", C.c_int), ("W", C.c_int), ("d_xhat", C.c_void_p), ("s", C.c_void_p)]


class TokError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {tok_strerror(code)} (code {code})")
        self.code = code


_lib = None
vp, i32, i64, u64, f32, sz = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_float, C.c_size_t

_SIGS = {
    "tok_arch_default": (None, [C.POINTER(tok_arch)]),
    "tok_create": (i32, [C.POINTER(tok_arch), i32, C.POINTER(vp)]),
    "tok_save_params": (i32, [vp, C.c_char_p]),
    "tok_create_from_file": (i32, [C.c_char_p, i32, C.POINTER(vp)]),
    "tok_read_weights_header": (i32, [C.c_char_p, C.POINTER(tok_arch), C.POINTER(i64)]),
    "tok_destroy": (None, [vp]),
    "tok_param_count": (i32, [vp]),
    "tok_param_info": (i32, [vp, i32, C.POINTER(C.c_char_p), C.POINTER(i32), C.POINTER(i64)]),
    "tok_set_param": (i32, [vp, C.c_char_p, vp, i64]),
    "tok_workspace_bytes": (sz, [vp, i32, i32, i32, i32]),
    "tok_reserve": (i32, [vp, i32, i32, i32, i32]),
    "tok_latent_shape": (i32, [vp, i32, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    "tok_encode": (i32, [vp, vp, i32, i32, i32, i32, vp, vp, vp, vp]),
    "tok_decode": (i32, [vp, vp, i32, i32, i32, i32, i32, i32, vp, vp, vp]),
    "tok_set_cta_tiles": (i32, [vp, i32]),
    "tok_trace_layer": (i32, [vp, C.c_char_p, vp, sz, vp, sz, vp, sz]),
    "tok_downsample": (i32, [i32, vp, i32, i32, i32, i32, i32, i32, vp, vp]),
    "tok_gop_blend": (i32, [vp, i32, vp, vp, i32, i32, i32, i32, i32, i32, vp]),
    "tok_decode_gop": (i32, [vp, vp, i32, i32, i32, i32, i32, i32, vp, i32, i32, vp, vp]),
    "tok_temporal_loss_workspace_bytes": (sz, [i32, i32, i32, i32, i32]),
    "tok_temporal_loss": (i32, [vp, vp, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, sz, vp]),
    "tok_residual": (i32, [i32, vp, vp, i32, i32, i32, i32, i32, i32, f32, vp, vp]),
    "tok_residual_sparse_workspace_bytes": (sz, [i32, i32, i32, i32, i32]),
    "tok_residual_sparse": (i32, [vp, i32, i32, i32, i32, i32, vp, vp, vp, vp, sz, vp]),
    "tok_residual_apply": (i32, [vp, i32, i32, i32, i32, i32, i32, vp, vp, vp, i64, vp]),
    "tok_similarity_workspace_bytes": (sz, [i32, i32, i32, i32]),
    "tok_similarity_mask": (i32, [vp, vp, i32, i32, i32, i32, C.POINTER(i32), i32, f32, vp, vp, vp, vp, sz, vp]),
    "tok_batch_workspace_bytes": (sz, [vp, C.POINTER(tok_shape), i32]),
    "tok_reserve_batch": (i32, [vp, C.POINTER(tok_shape), i32]),
    "tok_encode_batch": (i32, [vp, C.POINTER(tok_enc_item), i32, vp]),
    "tok_decode_batch": (i32, [vp, C.POINTER(tok_dec_item), i32, vp]),
    "tok_quantize": (i32, [vp, i64, vp, i32, vp, vp, vp]),
    "tok_dequantize": (i32, [vp, i64, vp, i32, vp, vp]),
    "tok_zero_index": (i32, [vp, i32]),
    "tok_drop_mask": (i32, [vp, i32, i32, i32, i32, f32, u64, u64, u64, i32, vp, vp, vp]),
    "tok_pack_rows": (i32, [vp, vp, i64, i32, vp, vp, vp]),
    "tok_unpack_rows": (i32, [vp, vp, vp, vp, i64, i32, i32, vp, vp]),
    "tok_stream_bytes": (sz, [vp, i32, i32]),
    "tok_stream_open": (i32, [vp, i32, i32, C.POINTER(vp)]),
    "tok_stream_close": (None, [vp]),
    "tok_stream_reset": (i32, [vp]),
    "tok_conv3d_workspace_bytes": (sz, [i32, i32, i32, i32]),
    "tok_conv3d": (i32, [i32, vp, i32, i32, i32, i32, i32, vp, vp, i32, i32, i32, i32, i32, i32, vp, vp, vp, sz,
                         vp]),
    "tok_groupnorm_workspace_bytes": (sz, [i32, i64, i64, i32, i32]),
    "tok_groupnorm_silu": (i32, [i32, vp, i64, i64, i32, i32, vp, vp, f32, vp, vp, sz, vp]),
    "tok_set_train_mode": (i32, [vp, i32]),
    "tok_param_total": (i64, [vp]),
    "tok_get_params": (i32, [vp, vp, vp]),
    "tok_set_params_device": (i32, [vp, vp, vp]),
    "tok_params": (vp, [vp]),
    "tok_repack": (i32, [vp, vp]),
    "tok_train_workspace_bytes": (sz, [vp, i32, i32, i32, i32]),
    "tok_reserve_train": (i32, [vp, i32, i32, i32, i32]),
    "tok_train_forward": (i32, [vp, vp, i32, i32, i32, i32, f32, u64, u64, vp, vp, vp, vp, vp]),
    "tok_backward": (i32, [vp, vp, vp, vp]),
    "tok_sgd": (i32, [vp, vp, i64, f32, vp]),
    "tok_groupnorm_silu_noalloc": (i32, [i32, vp, i64, i64, i32, i32, vp, vp, f32, vp, vp]),
    "tok_status": (i32, [vp]),
    "tok_strerror": (C.c_char_p, [i32]),
    "tok_check_guards": (i32, [vp]),
    "tok_stream_check_guards": (i32, [vp]),
    "tok_selftest_guards": (i32, [vp]),
    "tok_selftest_timeout": (i32, [vp, i64, vp]),
    "tok_launch_count": (i64, [vp]),
    "tok_profile_enable": (i32, [vp, i32]),
    "tok_profile_records": (i32, [vp, vp, i32, C.POINTER(i32)]),
    "tok_profile_read": (i32, [vp, C.POINTER(tok_profile_stats)]),
}


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -m paper_2602_03529_b300.build`)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_names():
    return list(_SIGS)


def _call(name, *args):
    return getattr(load(), name)(*args)


def _ck(code, what):
    if code != TOK_OK:
        raise TokError(code, what)


def _levels_arr(levels):
    arr = (C.c_int * len(levels))(*levels)
    return arr


# --- one wrapper per entry point (same names as include/tok.h) -------------

def tok_arch_default() -> tok_arch:
    a = tok_arch()
    _call("tok_arch_default", C.byref(a))
    return a


def tok_create(arch: tok_arch, precision: int) -> int:
    h = vp()
    _ck(_call("tok_create", C.byref(arch), precision, C.byref(h)), "tok_create")
    return h.value


def tok_save_params(ctx: int, path: str) -> None:
    _ck(_call("tok_save_params", ctx, os.fsencode(path)), "tok_save_params")


def tok_create_from_file(path: str, precision: int) -> int:
    h = vp()
    _ck(_call("tok_create_from_file", os.fsencode(path), precision, C.byref(h)), "tok_create_from_file")
    return h.value


def tok_read_weights_header(path: str):
    """(tok_arch, parameter count) of a weights file; host only."""
    a = tok_arch()
    n = i64()
    _ck(_call("tok_read_weights_header", os.fsencode(path), C.byref(a), C.byref(n)), "tok_read_weights_header")
    return a, n.value


def tok_check_guards(ctx: int) -> int:
    """TOK_OK or TOK_EGUARD (a kernel wrote outside the context's workspaces)."""
    return _call("tok_check_guards", ctx)


def tok_stream_check_guards(st: int) -> int:
    return _call("tok_stream_check_guards", st)


def tok_selftest_guards(ctx: int) -> int:
    return _call("tok_selftest_guards", ctx)


def tok_destroy(ctx: int) -> None:
    _call("tok_destroy", ctx)


def tok_param_count(ctx: int) -> int:
    return _call("tok_param_count", ctx)


def tok_param_info(ctx: int, i: int):
    name = C.c_char_p()
    nd = i32()
    dims = (i64 * 5)()
    _ck(_call("tok_param_info", ctx, i, C.byref(name), C.byref(nd), dims), "tok_param_info")
    return name.value.decode(), tuple(dims[k] for k in range(nd.value))


def tok_set_param(ctx: int, name: str, host_ptr: int, count: int) -> None:
    _ck(_call("tok_set_param", ctx, name.encode(), host_ptr, count), f"tok_set_param({name})")


def tok_workspace_bytes(ctx: int, N: int, T: int, H: int, W: int) -> int:
    return _call("tok_workspace_bytes", ctx, N, T, H, W)


def tok_reserve(ctx: int, N: int, T: int, H: int, W: int) -> None:
    _ck(_call("tok_reserve", ctx, N, T, H, W), "tok_reserve")


def tok_latent_shape(ctx: int, T: int, H: int, W: int):
    a, b, c = i32(), i32(), i32()
    _ck(_call("tok_latent_shape", ctx, T, H, W, C.byref(a), C.byref(b), C.byref(c)), "tok_latent_shape")
    return a.value, b.value, c.value


def tok_encode(ctx, x_ptr, N, T, H, W, z_ptr, idx_ptr, stream_handle, cuda_stream) -> None:
    _ck(_call("tok_encode", ctx, x_ptr, N, T, H, W, z_ptr, idx_ptr, stream_handle, cuda_stream), "tok_encode")


def tok_decode(ctx, idx_ptr, N, Tq, Hq, Wq, H, W, xhat_ptr, stream_handle, cuda_stream) -> None:
    _ck(_call("tok_decode", ctx, idx_ptr, N, Tq, Hq, Wq, H, W, xhat_ptr, stream_handle, cuda_stream),
        "tok_decode")


def tok_similarity_workspace_bytes(N, Tp, Hq, Wq) -> int:
    return int(_call("tok_similarity_workspace_bytes", N, Tp, Hq, Wq))


def tok_similarity_mask(idx_p, idx_i, N, Tp, Hq, Wq, levels, rate, out, keep_bits, sim, ws, ws_bytes,
                        cuda_stream) -> None:
    lv = (i32 * len(levels))(*levels)
    _ck(_call("tok_similarity_mask", idx_p, idx_i, N, Tp, Hq, Wq, lv, len(levels), float(rate), out, keep_bits,
              sim, ws, ws_bytes, cuda_stream), "tok_similarity_mask")


def tok_residual(precision, x, xhat, N, T, H, W, C, window, theta, r, cuda_stream) -> None:
    _ck(_call("tok_residual", precision, x, xhat, N, T, H, W, C, window, float(theta), r, cuda_stream),
        "tok_residual")


def tok_residual_sparse_workspace_bytes(N, nwin, H, W, C) -> int:
    return int(_call("tok_residual_sparse_workspace_bytes", N, nwin, H, W, C))


def tok_residual_sparse(r, N, nwin, H, W, C, pos, val, seg_off, ws, ws_bytes, cuda_stream) -> None:
    _ck(_call("tok_residual_sparse", r, N, nwin, H, W, C, pos, val, seg_off, ws, ws_bytes, cuda_stream),
        "tok_residual_sparse")


def tok_residual_apply(xhat, N, T, H, W, C, window, pos, val, seg_off, capacity, cuda_stream) -> None:
    _ck(_call("tok_residual_apply", xhat, N, T, H, W, C, window, pos, val, seg_off, capacity, cuda_stream),
        "tok_residual_apply")


def tok_downsample(in_type, x, F, H, W, C, s, out_precision, y, cuda_stream) -> None:
    _ck(_call("tok_downsample", in_type, x, F, H, W, C, s, out_precision, y, cuda_stream), "tok_downsample")


def tok_gop_blend(prev, Tp, curr, out, N, T, H, W, C, n, cuda_stream) -> None:
    _ck(_call("tok_gop_blend", prev, Tp, curr, out, N, T, H, W, C, n, cuda_stream), "tok_gop_blend")


def tok_decode_gop(ctx, idx, N, Tq, Hq, Wq, H, W, prev, Tp, n, xhat, cuda_stream) -> None:
    _ck(_call("tok_decode_gop", ctx, idx, N, Tq, Hq, Wq, H, W, prev, Tp, n, xhat, cuda_stream), "tok_decode_gop")


def tok_temporal_loss_workspace_bytes(N, n, H, W, C) -> int:
    return int(_call("tok_temporal_loss_workspace_bytes", N, n, H, W, C))


def tok_temporal_loss(xc, xp, N, Tc, Tp, H, W, C, n, loss, grad, ws, ws_bytes, cuda_stream) -> None:
    _ck(_call("tok_temporal_loss", xc, xp, N, Tc, Tp, H, W, C, n, loss, grad, ws, ws_bytes, cuda_stream),
        "tok_temporal_loss")


def tok_set_cta_tiles(ctx, tiles: int) -> None:
    _ck(_call("tok_set_cta_tiles", ctx, tiles), "tok_set_cta_tiles")


def tok_trace_layer(ctx, name, d_in, in_bytes, d_res, res_bytes, d_out, out_bytes) -> None:
    _ck(_call("tok_trace_layer", ctx, None if name is None else name.encode(), d_in, in_bytes, d_res, res_bytes,
              d_out, out_bytes), "tok_trace_layer")


def _shapes(shapes):
    arr = (tok_shape * len(shapes))()
    for i, (N, T, H, W) in enumerate(shapes):
        arr[i] = tok_shape(N, T, H, W)
    return arr


def tok_batch_workspace_bytes(ctx, shapes) -> int:
    """shapes: list of (N, T, H, W)."""
    return int(_call("tok_batch_workspace_bytes", ctx, _shapes(shapes), len(shapes)))


def tok_reserve_batch(ctx, shapes) -> None:
    _ck(_call("tok_reserve_batch", ctx, _shapes(shapes), len(shapes)), "tok_reserve_batch")


def tok_encode_batch(ctx, items, cuda_stream) -> None:
    """items: list of (x_ptr, N, T, H, W, z_ptr, idx_ptr, stream_handle)."""
    arr = (tok_enc_item * len(items))()
    for i, it in enumerate(items):
        arr[i] = tok_enc_item(*it)
    _ck(_call("tok_encode_batch", ctx, arr, len(items), cuda_stream), "tok_encode_batch")


def tok_decode_batch(ctx, items, cuda_stream) -> None:
    """items: list of (idx_ptr, N, Tq, Hq, Wq, H, W, xhat_ptr, stream_handle)."""
    arr = (tok_dec_item * len(items))()
    for i, it in enumerate(items):
        arr[i] = tok_dec_item(*it)
    _ck(_call("tok_decode_batch", ctx, arr, len(items), cuda_stream), "tok_decode_batch")


def tok_quantize(z_ptr, ntok, levels, idx_ptr, codes_ptr, cuda_stream) -> None:
    lv = _levels_arr(levels)
    _ck(_call("tok_quantize", z_ptr, ntok, C.cast(lv, vp), len(levels), idx_ptr, codes_ptr, cuda_stream),
        "tok_quantize")


def tok_dequantize(idx_ptr, ntok, levels, codes_ptr, cuda_stream) -> None:
    lv = _levels_arr(levels)
    _ck(_call("tok_dequantize", idx_ptr, ntok, C.cast(lv, vp), len(levels), codes_ptr, cuda_stream),
        "tok_dequantize")


def tok_zero_index(levels) -> int:
    lv = _levels_arr(levels)
    return _call("tok_zero_index", C.cast(lv, vp), len(levels))


def tok_drop_mask(idx_ptr, N, Tq, Hq, Wq, rate, seed, stream_id, chunk_id, zero_index, out_ptr, keep_ptr,
                  cuda_stream) -> None:
    _ck(_call("tok_drop_mask", idx_ptr, N, Tq, Hq, Wq, rate, seed, stream_id, chunk_id, zero_index, out_ptr,
              keep_ptr, cuda_stream), "tok_drop_mask")


def tok_pack_rows(idx_ptr, keep_ptr, rows, Wq, payload_ptr, offs_ptr, cuda_stream) -> None:
    _ck(_call("tok_pack_rows", idx_ptr, keep_ptr, rows, Wq, payload_ptr, offs_ptr, cuda_stream), "tok_pack_rows")


def tok_unpack_rows(payload_ptr, offs_ptr, keep_ptr, received_ptr, rows, Wq, zero_index, idx_ptr,
                    cuda_stream) -> None:
    _ck(_call("tok_unpack_rows", payload_ptr, offs_ptr, keep_ptr, received_ptr, rows, Wq, zero_index, idx_ptr,
              cuda_stream), "tok_unpack_rows")


def tok_stream_bytes(ctx, H, W) -> int:
    return _call("tok_stream_bytes", ctx, H, W)


def tok_stream_open(ctx, H, W) -> int:
    h = vp()
    _ck(_call("tok_stream_open", ctx, H, W, C.byref(h)), "tok_stream_open")
    return h.value


def tok_stream_close(s) -> None:
    _call("tok_stream_close", s)


def tok_stream_reset(s) -> None:
    _ck(_call("tok_stream_reset", s), "tok_stream_reset")


def tok_conv3d_workspace_bytes(precision, Cin, Cout, k) -> int:
    return _call("tok_conv3d_workspace_bytes", precision, Cin, Cout, k)


def tok_conv3d(precision, x_ptr, N, T, H, W, Cin, w_ptr, b_ptr, Cout, k, st, sh, sw, time_pad, res_ptr, y_ptr,
               ws_ptr, ws_bytes, cuda_stream) -> None:
    _ck(_call("tok_conv3d", precision, x_ptr, N, T, H, W, Cin, w_ptr, b_ptr, Cout, k, st, sh, sw, time_pad,
              res_ptr, y_ptr, ws_ptr, ws_bytes, cuda_stream), "tok_conv3d")


def tok_groupnorm_workspace_bytes(precision, frames, HW, C, G) -> int:
    return _call("tok_groupnorm_workspace_bytes", precision, frames, HW, C, G)


def tok_groupnorm_silu(precision, x_ptr, frames, HW, C, G, g_ptr, b_ptr, eps, y_ptr, ws_ptr, ws_bytes,
                       cuda_stream) -> None:
    _ck(_call("tok_groupnorm_silu", precision, x_ptr, frames, HW, C, G, g_ptr, b_ptr, eps, y_ptr, ws_ptr,
              ws_bytes, cuda_stream), "tok_groupnorm_silu")


def tok_groupnorm_silu_noalloc(precision, x_ptr, frames, HW, C, G, g_ptr, b_ptr, eps, y_ptr, cuda_stream) -> None:
    """GroupNorm+SiLU with library-owned fixed scratch (no workspace, no allocation)."""
    _ck(_call("tok_groupnorm_silu_noalloc", precision, x_ptr, frames, HW, C, G, g_ptr, b_ptr, eps, y_ptr,
              cuda_stream), "tok_groupnorm_silu_noalloc")


def tok_status(ctx) -> int:
    return _call("tok_status", ctx)


def tok_strerror(code: int) -> str:
    return _call("tok_strerror", code).decode()


def tok_selftest_timeout(ctx, limit_ns, cuda_stream) -> None:
    _ck(_call("tok_selftest_timeout", ctx, limit_ns, cuda_stream), "tok_selftest_timeout")


def tok_launch_count(ctx) -> int:
    return _call("tok_launch_count", ctx)


def tok_profile_enable(ctx, on: bool) -> None:
    _ck(_call("tok_profile_enable", ctx, 1 if on else 0), "tok_profile_enable")


def tok_profile_read(ctx) -> dict:
    st = tok_profile_stats()
    _ck(_call("tok_profile_read", ctx, C.byref(st)), "tok_profile_read")
    return {f: getattr(st, f) for f, _ in tok_profile_stats._fields_}


def tok_profile_records(ctx) -> list:
    n = i32()
    _ck(_call("tok_profile_records", ctx, None, 0, C.byref(n)), "tok_profile_records")
    arr = (tok_profile_record * max(n.value, 1))()
    _ck(_call("tok_profile_records", ctx, C.cast(arr, C.c_void_p), n.value, C.byref(n)), "tok_profile_records")
    return [{"cls": r.cls, "ms": r.ms, "work": r.work, "name": r.name.decode()} for r in arr[:n.value]]


def tok_param_total(ctx) -> int:
    return _call("tok_param_total", ctx)


def tok_get_params(ctx, d_flat, cuda_stream) -> None:
    _ck(_call("tok_get_params", ctx, d_flat, cuda_stream), "tok_get_params")


def tok_set_params_device(ctx, d_flat, cuda_stream) -> None:
    _ck(_call("tok_set_params_device", ctx, d_flat, cuda_stream), "tok_set_params_device")


def tok_params(ctx) -> int:
    """Device address of the context's flat FP32 parameters (owned by the context)."""
    return _call("tok_params", ctx)


def tok_repack(ctx, cuda_stream) -> None:
    _ck(_call("tok_repack", ctx, cuda_stream), "tok_repack")


def tok_train_workspace_bytes(ctx, N, T, H, W) -> int:
    return _call("tok_train_workspace_bytes", ctx, N, T, H, W)


TOK_TRAIN_RECOMPUTE, TOK_TRAIN_KEEP = 0, 1


def tok_set_train_mode(ctx, mode: int) -> None:
    _ck(_call("tok_set_train_mode", ctx, mode), "tok_set_train_mode")


def tok_reserve_train(ctx, N, T, H, W) -> None:
    _ck(_call("tok_reserve_train", ctx, N, T, H, W), "tok_reserve_train")


def tok_train_forward(ctx, x_ptr, N, T, H, W, rate, seed, step, keep_ptr, xhat_ptr, loss_ptr, dxhat_ptr,
                      cuda_stream) -> None:
    _ck(_call("tok_train_forward", ctx, x_ptr, N, T, H, W, rate, seed, step, keep_ptr, xhat_ptr, loss_ptr,
              dxhat_ptr, cuda_stream), "tok_train_forward")


def tok_backward(ctx, dxhat_ptr, dparams_ptr, cuda_stream) -> None:
    _ck(_call("tok_backward", ctx, dxhat_ptr, dparams_ptr, cuda_stream), "tok_backward")


def tok_sgd(p_ptr, g_ptr, n, lr, cuda_stream) -> None:
    _ck(_call("tok_sgd", p_ptr, g_ptr, n, lr, cuda_stream), "tok_sgd")
