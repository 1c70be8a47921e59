"""Weights files (checkpoint / resume): the header reader on the host against files
written here from the documented layout, with the parameter count taken from the
oracle's parameter list; every malformed variant is refused with TOK_EFILE."""
import struct

import numpy as np
import pytest

from oracle import Arch, param_spec

MAGIC, VERSION = b"TOKW", 1


def _count(arch: Arch) -> int:
    return int(sum(np.prod(shape) for _, shape, _ in param_spec(arch)))


def _fnv1a64(b: bytes) -> int:
    h = 0xcbf29ce484222325
    for x in b:
        h = ((h ^ x) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _write(path, *, ch=(64, 128, 256), blocks=1, levels=(8, 8, 8, 5, 5, 5), nlevels=None, n=None, magic=MAGIC,
           version=VERSION, t_stem=1, truncate=0, payload=None):
    nlevels = len(ch) if nlevels is None else nlevels
    count = _count(Arch(ch=ch, blocks=blocks, t_stem=t_stem)) if n is None else n
    h = bytearray(104)
    h[0:4] = magic
    struct.pack_into("<I", h, 4, version)
    struct.pack_into("<iii", h, 8, 0, 3, nlevels)
    struct.pack_into("<4i", h, 20, *(list(ch) + [0] * (4 - len(ch))))
    struct.pack_into("<ii", h, 36, blocks, len(levels))
    struct.pack_into("<8i", h, 44, *(list(levels) + [0] * (8 - len(levels))))
    struct.pack_into("<ifii", h, 76, 32, 1e-6, 0, t_stem)
    struct.pack_into("<q", h, 96, count)
    p = (np.arange(max(count, 0), dtype=np.float32) * 1e-3).tobytes() if payload is None else payload
    data = bytes(h) + p + struct.pack("<Q", _fnv1a64(p) if len(p) < 1 << 16 else 0)
    path.write_bytes(data[:len(data) - truncate] if truncate else data)
    return count


@pytest.fixture(scope="module")
def L():
    from paper_2602_03529_b300 import _lib as L
    L.load()
    return L


def test_header_round_trip(L, tmp_path):
    f = tmp_path / "w.tokw"
    n = _write(f)
    a, m = L.tok_read_weights_header(str(f))
    assert m == n
    assert (a.kind, a.in_ch, a.nlevels, list(a.ch[:3]), a.blocks, a.nlev) == (0, 3, 3, [64, 128, 256], 1, 6)
    assert list(a.levels[:6]) == [8, 8, 8, 5, 5, 5] and a.gn_groups == 32 and a.t_stem == 1
    assert abs(a.gn_eps - 1e-6) < 1e-12


def test_header_eight_by_eight_by_eight(L, tmp_path):
    f = tmp_path / "w.tokw"
    n = _write(f, t_stem=2)
    a, m = L.tok_read_weights_header(str(f))
    assert (m, a.t_stem) == (n, 2)


@pytest.mark.parametrize("bad", ["magic", "version", "count", "levels", "nlevels", "truncated", "longer",
                                 "missing"])
def test_malformed_files_are_refused(L, tmp_path, bad):
    f = tmp_path / "w.tokw"
    if bad == "magic":
        _write(f, magic=b"TOKX")
    elif bad == "version":
        _write(f, version=2)
    elif bad == "count":
        n = _count(Arch(ch=(64, 128, 256), blocks=1))
        _write(f, n=n + 1)
    elif bad == "levels":
        _write(f, levels=(8, 8, 1))
    elif bad == "nlevels":
        _write(f, nlevels=5)
    elif bad == "truncated":
        _write(f, truncate=1)
    elif bad == "longer":
        n = _write(f)
        f.write_bytes(f.read_bytes() + b"\0")
    else:
        f = tmp_path / "absent.tokw"
    with pytest.raises(L.TokError) as e:
        L.tok_read_weights_header(str(f))
    assert e.value.code == L.TOK_EFILE
