"""ORACLE -- test infrastructure only.

Python access to the plain sequential CPU implementation in ``ace_oracle.c``
(encoder, decoder, dependency levels, seek closure, FNV-1a).  Only the test
suite, the smoke check and the benchmark's CPU-baseline leg use it; the GPU
library never imports it.  See ``ace_oracle.h`` for which parts are pinned
and how.
"""
import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "ace_oracle.c")
_HDR = os.path.join(_DIR, "ace_oracle.h")
_LIB = os.path.join(_DIR, "liboracle.so")

OK, E_INVAL, E_CORRUPT, E_RANGE, E_NOMEM = 0, -1, -2, -3, -4


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__("oracle %s failed: %d" % (what, rc))
        self.rc = rc


def build(force=False):
    """Compile the oracle with plain gcc (no architecture-specific flags)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        lib.oracle_fnv1a64.argtypes = [vp, u64]
        lib.oracle_fnv1a64.restype = u64
        lib.oracle_fnv1a32.argtypes = [vp, u64]
        lib.oracle_fnv1a32.restype = u32
        lib.oracle_rans_freqs.argtypes = [vp, u32, vp]
        lib.oracle_rans_encode.argtypes = [vp, u32, vp, vp, vp, u32, vp]
        lib.oracle_rans_decode.argtypes = [vp, u32, vp, vp, u32, vp]
        lib.oracle_encode_bound.argtypes = [u64, u32]
        lib.oracle_encode_bound.restype = u64
        lib.oracle_encode.argtypes = [vp, u64, u32, u32, u32, vp, u64, vp]
        lib.oracle_encode_adaptive.argtypes = [vp, u64, u32, u32, u32, u32, vp, u64, vp]
        lib.oracle_info.argtypes = [vp, u64, vp, vp, vp, vp]
        lib.oracle_decode.argtypes = [vp, u64, vp, u64]
        lib.oracle_decode_block_tokens.argtypes = [vp, u64, u64, vp, vp, vp, u32, vp]
        lib.oracle_levels.argtypes = [vp, u64, vp]
        lib.oracle_closure.argtypes = [vp, u64, u64, u64, vp]
        lib.oracle_seek.argtypes = [vp, u64, u64, u64, vp]
        for f in ("oracle_rans_freqs", "oracle_rans_encode", "oracle_rans_decode", "oracle_encode",
                  "oracle_encode_adaptive",
                  "oracle_info", "oracle_decode", "oracle_decode_block_tokens", "oracle_levels",
                  "oracle_closure", "oracle_seek"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(data):
    if isinstance(data, (bytes, bytearray)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    a = np.ascontiguousarray(data, dtype=np.uint8)
    return a


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


def fnv1a64(data):
    a = _u8(data)
    return _L().oracle_fnv1a64(_p(a), a.size)


def fnv1a32(data):
    a = _u8(data)
    return _L().oracle_fnv1a32(_p(a), a.size)


def rans_freqs(sym):
    s = _u8(sym)
    f = np.zeros(256, np.uint16)
    _check(_L().oracle_rans_freqs(_p(s), s.size, _p(f)), "rans_freqs")
    return f


def rans_encode(sym, freq):
    """Encode one stream: returns (states[32] uint32, renorm bytes uint8)."""
    s = _u8(sym)
    f = np.ascontiguousarray(freq, dtype=np.uint16)
    st = np.zeros(32, np.uint32)
    cap = 2 * s.size + 64
    out = np.zeros(cap, np.uint8)
    n = ctypes.c_uint32(0)
    _check(_L().oracle_rans_encode(_p(s), s.size, _p(f), _p(st), _p(out), cap, ctypes.byref(n)),
           "rans_encode")
    return st, out[:n.value].copy()


def rans_decode(data, states, freq, n):
    d = _u8(data)
    st = np.ascontiguousarray(states, dtype=np.uint32)
    f = np.ascontiguousarray(freq, dtype=np.uint16)
    out = np.zeros(max(n, 1), np.uint8)
    _check(_L().oracle_rans_decode(_p(d), d.size, _p(st), _p(f), n, _p(out)), "rans_decode")
    return out[:n]


def encode(data, log2_block=14, min_match=4, max_chain=64, adaptive=False):
    """Encode bytes into an archive (uint8 array); adaptive stores each
    stream that rANS would not shrink."""
    a = _u8(data)
    cap = _L().oracle_encode_bound(a.size, log2_block)
    arc = np.zeros(cap, np.uint8)
    n = ctypes.c_uint64(0)
    _check(_L().oracle_encode_adaptive(_p(a), a.size, log2_block, min_match, max_chain, int(adaptive),
                                       _p(arc), cap, ctypes.byref(n)), "encode")
    return arc[:n.value].copy()


def info(arc):
    a = _u8(arc)
    total, bs, nb, w = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32()
    _check(_L().oracle_info(_p(a), a.size, ctypes.byref(total), ctypes.byref(bs), ctypes.byref(nb),
                            ctypes.byref(w)), "info")
    return {"total": total.value, "block_size": bs.value, "n_blocks": nb.value, "off_width": w.value}


def decode(arc):
    a = _u8(arc)
    total = info(a)["total"]
    out = np.zeros(max(total, 1), np.uint8)
    _check(_L().oracle_decode(_p(a), a.size, _p(out), total), "decode")
    return out[:total]


def block_tokens(arc, block):
    """(lit_run, match_len, src) arrays of one block's tokens."""
    a = _u8(arc)
    cap = info(a)["block_size"] + 2
    lr, ml, src = np.zeros(cap, np.uint32), np.zeros(cap, np.uint32), np.zeros(cap, np.uint64)
    n = ctypes.c_uint32(0)
    _check(_L().oracle_decode_block_tokens(_p(a), a.size, block, _p(lr), _p(ml), _p(src), cap,
                                           ctypes.byref(n)), "block_tokens")
    k = n.value
    return lr[:k].copy(), ml[:k].copy(), src[:k].copy()


def levels(arc):
    a = _u8(arc)
    nb = info(a)["n_blocks"]
    lv = np.zeros(max(nb, 1), np.uint32)
    _check(_L().oracle_levels(_p(a), a.size, _p(lv)), "levels")
    return lv[:nb]


def closure(arc, first, last):
    a = _u8(arc)
    nb = info(a)["n_blocks"]
    m = np.zeros(max(nb, 1), np.uint8)
    _check(_L().oracle_closure(_p(a), a.size, first, last, _p(m)), "closure")
    return np.nonzero(m[:nb])[0]


def seek(arc, coord, length):
    a = _u8(arc)
    out = np.zeros(max(length, 1), np.uint8)
    _check(_L().oracle_seek(_p(a), a.size, coord, length, _p(out)), "seek")
    return out[:length]


def deps(arc):
    """Per-block dependency intervals read straight from the archive bytes."""
    a = _u8(arc)
    hdr = info(a)
    nb = hdr["n_blocks"]
    deps_off = int(a[40:48].view(np.uint64)[0])
    ptr = a[deps_off:deps_off + 4 * (nb + 1)].view(np.uint32)
    ivs = a[deps_off + 4 * (nb + 1):deps_off + 4 * (nb + 1) + 8 * int(ptr[-1] if nb else 0)].view(np.uint32)
    return [[(int(ivs[2 * i]), int(ivs[2 * i + 1])) for i in range(ptr[b], ptr[b + 1])] for b in range(nb)]
