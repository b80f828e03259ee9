"""Thin ctypes binding of libace.so: the C ABI of include/ace.h under the
same names, doing argument marshalling only.  Every step of decoding runs in
the library's CUDA kernels; there is no Python or CPU fallback, and loading
fails loudly when the library has not been built.

Device buffers are passed as integers or as objects with ``data_ptr()``
(torch tensors); streams as integers or objects with ``cuda_stream``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ACE_OK, ACE_E_INVAL, ACE_E_CORRUPT, ACE_E_RANGE, ACE_E_NOMEM, ACE_E_TIMEOUT, ACE_E_CUDA = range(7)
ACE_PASS_TOKENS, ACE_PASS_LITERALS, ACE_PASS_MATCH = 0, 1, 2
ACE_SCHEDULE_AUTO, ACE_SCHEDULE_PASSES, ACE_SCHEDULE_FUSED = 0, 1, 2


class AceError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s: %s" % (what, ace_status_str(status)))
        self.status = status


class ace_encode_params(ctypes.Structure):
    _fields_ = [("log2_block", ctypes.c_uint32), ("min_match", ctypes.c_uint32),
                ("threads", ctypes.c_uint32), ("max_chain", ctypes.c_uint32),
                ("off_width", ctypes.c_uint32), ("adaptive", ctypes.c_uint32)]


class ace_encode_stats(ctypes.Structure):
    _fields_ = [("n_tokens", ctypes.c_uint64), ("n_matches", ctypes.c_uint64),
                ("literal_bytes", ctypes.c_uint64), ("match_bytes", ctypes.c_uint64),
                ("match_src_bytes", ctypes.c_uint64), ("n_dep_intervals", ctypes.c_uint64),
                ("n_levels", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ace_info(ctypes.Structure):
    _fields_ = [("total_size", ctypes.c_uint64), ("n_blocks", ctypes.c_uint64),
                ("archive_bytes", ctypes.c_uint64), ("n_dep_intervals", ctypes.c_uint64),
                ("block_size", ctypes.c_uint32), ("off_width", ctypes.c_uint32),
                ("n_levels", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ace_tune(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("chunk_tokens", ctypes.c_uint32), ("schedule", ctypes.c_uint32),
                ("wait_timeout_ns", ctypes.c_uint64), ("copy_width", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ace_verify_report(ctypes.Structure):
    _fields_ = [("fnv_before", ctypes.c_uint64), ("fnv_after", ctypes.c_uint64),
                ("guard_bad_before", ctypes.c_uint64), ("guard_bad_after", ctypes.c_uint64),
                ("phase1_ok", ctypes.c_int32), ("phase2_ok", ctypes.c_int32),
                ("phase3_ok", ctypes.c_int32), ("seek_status", ctypes.c_int32)]


_lib = None
_u64, _u32, _vp, _i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32
_P = ctypes.POINTER

_SIGS = {
    "ace_status_str": ([_i32], ctypes.c_char_p),
    "ace_encode_bound": ([_u64, _u32, _P(_u64)], _i32),
    "ace_encode": ([_vp, _u64, _P(ace_encode_params), _vp, _u64, _P(_u64)], _i32),
    "ace_encode_run": ([_vp, _u64, _P(ace_encode_params), _P(_vp), _P(_u64)], _i32),
    "ace_encode_write": ([_vp, _vp, _u64], _i32),
    "ace_encode_free": ([_vp], _i32),
    "ace_encode_get_stats": ([_vp, _P(ace_encode_stats)], _i32),
    "ace_encode_gpu_size": ([_u64, _P(ace_encode_params), _P(_u64), _P(_u64)], _i32),
    "ace_encode_gpu": ([_vp, _u64, _P(ace_encode_params), _vp, _u64, _vp, _u64, _P(_u64), _P(ace_encode_stats), _vp],
                       _i32),
    "ace_index_size": ([_vp, _u64, _P(_u64)], _i32),
    "ace_index_build": ([_vp, _u64, _vp, _u64, _vp, _u64, _vp, _P(_vp)], _i32),
    "ace_index_info": ([_vp, _P(ace_info)], _i32),
    "ace_index_levels": ([_vp, _P(_u32), _u32, _vp], _i32),
    "ace_index_free": ([_vp], _i32),
    "ace_index_export_size": ([_vp, _P(_u64)], _i32),
    "ace_index_export": ([_vp, _vp, _u64, _vp], _i32),
    "ace_index_import": ([_vp, _u64, _vp, _u64, _vp, _u64, _vp, _u64, _vp, _P(_vp)], _i32),
    "ace_host_register": ([_vp, _u64, _u32, _P(_vp)], _i32),
    "ace_host_unregister": ([_vp], _i32),
    "ace_scratch_size": ([_vp, _u64, _P(_u64)], _i32),
    "ace_scratch_init": ([_vp, _vp, _u64, _vp], _i32),
    "ace_decode_all": ([_vp, _vp, _u64, _vp, _u64, _P(ace_tune), _vp], _i32),
    "ace_decode_pass": ([_vp, _i32, _vp, _u64, _vp, _u64, _P(ace_tune), _vp], _i32),
    "ace_seek": ([_vp, _u64, _u64, _vp, _u64, _vp, _u64, _vp], _i32),
    "ace_sync": ([_vp, _vp, _vp], _i32),
    "ace_index_set_tune": ([_vp, _P(ace_tune)], _i32),
    "ace_verify": ([_vp, _u64, _u64, _vp, _u64, _u64, _u32, _vp, _u64, _P(ace_verify_report), _vp], _i32),
    "ace_fnv1a64": ([_vp, _u64, _vp, _vp], _i32),
    "ace_seek_noalloc": ([_vp, _u64, _u64, _vp, _u64, _vp], _i32),
    "ace_batch_scratch_size": ([_vp, _u32, _P(_u64)], _i32),
    "ace_batch_create": ([_vp, _u32, _vp, _vp, _vp, _u64, _P(ace_tune), _vp, _P(_vp)], _i32),
    "ace_decode_batch": ([_vp, _vp], _i32),
    "ace_batch_sync": ([_vp, _vp], _i32),
    "ace_batch_launch_shape": ([_vp, _P(_u32), _P(_u32), _P(_u32)], _i32),
    "ace_batch_free": ([_vp], _i32),
    "ace_archive_state_size": ([_vp, _P(_u64)], _i32),
    "ace_cache_size": ([_vp, _u32, _u64, _u32, _P(_u64)], _i32),
    "ace_cache_create": ([_vp, _u32, _vp, _u64, _u32, _vp, _u64, _P(ace_tune), _vp, _P(_vp)], _i32),
    "ace_seek_batch": ([_vp, _vp, _u32, _vp, _u64, _vp], _i32),
    "ace_seek_batch_host": ([_vp, _vp, _vp, _u32, _vp, _u64, _vp], _i32),
    "ace_cache_sync": ([_vp, _vp], _i32),
    "ace_cache_usage": ([_vp, _P(_u32), _P(_u32), _vp], _i32),
    "ace_cache_reset": ([_vp, _vp], _i32),
    "ace_cache_counters": ([_vp, _P(_u64), _P(_u64), _vp], _i32),
    "ace_cache_limits": ([_vp, _P(_u32), _P(_u32), _P(_u32)], _i32),
    "ace_cache_free": ([_vp], _i32),
}


def lib():
    """The loaded libace.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError("libace.so is not built (%s); run __graft_entry__.build()" % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take a device pointer of %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, what):
    if rc != ACE_OK:
        raise AceError(rc, what)


def ace_status_str(status):
    return lib().ace_status_str(int(status)).decode()


# ------------------------------------------------------------------ encoding

def ace_encode_bound(n, log2_block):
    out = _u64()
    _check(lib().ace_encode_bound(n, log2_block, ctypes.byref(out)), "ace_encode_bound")
    return out.value


def ace_encode(h_in, log2_block=14, min_match=4, threads=0, max_chain=16, stats=False, off_width=0, adaptive=False):
    """Encode host bytes (numpy uint8) into an archive (numpy uint8) on the
    CPU; with stats=True also return the parse statistics as a dict.
    off_width: absolute-offset bytes, 0 for the smallest that fits (4 up to
    2^32 bytes of input, else 5), or 5 to force five.  adaptive: store each
    block's stream verbatim when rANS would not shrink it."""
    a = np.ascontiguousarray(h_in, dtype=np.uint8)
    prm = ace_encode_params(log2_block, min_match, threads, max_chain, off_width, 1 if adaptive else 0)
    enc, n = _vp(), _u64()
    _check(lib().ace_encode_run(a.ctypes.data, a.size, ctypes.byref(prm), ctypes.byref(enc),
                                ctypes.byref(n)), "ace_encode_run")
    try:
        arc = np.empty(n.value, np.uint8)
        _check(lib().ace_encode_write(enc, arc.ctypes.data, arc.size), "ace_encode_write")
        st = ace_encode_stats()
        _check(lib().ace_encode_get_stats(enc, ctypes.byref(st)), "ace_encode_get_stats")
    finally:
        lib().ace_encode_free(enc)
    if stats:
        return arc, {k: getattr(st, k) for k, _ in ace_encode_stats._fields_ if k != "reserved"}
    return arc


def ace_encode_gpu(d_in, log2_block=14, min_match=4, max_chain=16, stats=False, off_width=0, adaptive=False,
                   chunk_blocks=0, stream=None):
    """Encode device bytes (a uint8 CUDA tensor) into an archive on the same
    device; returns the archive as a CUDA tensor view (and, with stats=True,
    the parse statistics).  Scratch and archive memory come from PyTorch:
    first a buffer for the archive at about the input's size plus the
    dependency table's room, and the bound when that is too small."""
    import torch

    n = d_in.numel()
    prm = ace_encode_params(log2_block, min_match, chunk_blocks, max_chain, off_width, 1 if adaptive else 0)
    sb, bound = _u64(), _u64()
    _check(lib().ace_encode_gpu_size(n, ctypes.byref(prm), ctypes.byref(sb), ctypes.byref(bound)),
           "ace_encode_gpu_size")
    scratch = torch.empty(sb.value, dtype=torch.uint8, device=d_in.device)
    nb = (n + (1 << log2_block) - 1) >> log2_block
    reserve = bound.value - _enc_payload_room(nb, log2_block, min_match)  # header, directory, dependency room
    guess = min(bound.value, reserve + n + n // 8 + nb * 2048 + (1 << 20))
    for cap in (guess, bound.value):
        arc = torch.empty(cap, dtype=torch.uint8, device=d_in.device)
        ln, st = _u64(), ace_encode_stats()
        rc = lib().ace_encode_gpu(_ptr(d_in), n, ctypes.byref(prm), _ptr(scratch), sb.value, _ptr(arc), cap,
                                  ctypes.byref(ln), ctypes.byref(st), _stream(stream))
        if rc == ACE_E_NOMEM and cap < bound.value:
            del arc
            continue
        _check(rc, "ace_encode_gpu")
        out = arc[:ln.value]
        if stats:
            return out, {k: getattr(st, k) for k, _ in ace_encode_stats._fields_ if k != "reserved"}
        return out
    raise AssertionError("unreachable")


def _enc_payload_room(nb, log2_block, min_match):
    """The part of the GPU encoder's archive bound that is payload room (the
    bound less the header, directory and dependency-table room)."""
    B = 1 << log2_block
    tok_cap = B // min_match + 2
    sym_cap = (B + 11 * tok_cap + 15) & ~15
    pay_cap = (3 * (160 + 512 + 16) + 2 * sym_cap + 64 + 15) & ~15
    return nb * pay_cap + 256


# --------------------------------------------------------------------- index

def ace_index_size(h_header):
    h = np.ascontiguousarray(h_header[:64], dtype=np.uint8)
    out = _u64()
    _check(lib().ace_index_size(h.ctypes.data, h.size, ctypes.byref(out)), "ace_index_size")
    return out.value


def ace_index_build(d_archive, archive_bytes, h_header, d_index_mem, index_bytes, stream=None):
    h = np.ascontiguousarray(h_header[:64], dtype=np.uint8)
    out = _vp()
    _check(lib().ace_index_build(_ptr(d_archive), archive_bytes, h.ctypes.data, h.size,
                                 _ptr(d_index_mem), index_bytes, _stream(stream), ctypes.byref(out)),
           "ace_index_build")
    return out


def ace_index_levels(idx, n_levels, stream=None):
    """Blocks per dependency level, as a numpy array of n_levels entries."""
    out = np.zeros(max(n_levels, 1), np.uint32)
    _check(lib().ace_index_levels(idx, out.ctypes.data_as(ctypes.POINTER(_u32)), n_levels, _stream(stream)),
           "ace_index_levels")
    return out[:n_levels]


def ace_index_info(idx):
    info = ace_info()
    _check(lib().ace_index_info(idx, ctypes.byref(info)), "ace_index_info")
    return {k: getattr(info, k) for k, _ in ace_info._fields_ if k != "reserved"}


def ace_index_free(idx):
    lib().ace_index_free(idx)


def ace_index_export(idx, stream=None):
    """The stored form of an index (numpy uint8), for a file."""
    n = _u64()
    _check(lib().ace_index_export_size(idx, ctypes.byref(n)), "ace_index_export_size")
    blob = np.empty(n.value, np.uint8)
    _check(lib().ace_index_export(idx, blob.ctypes.data, blob.size, _stream(stream)), "ace_index_export")
    return blob


def ace_index_import(d_archive, archive_bytes, h_header, h_blob, d_index_mem, index_bytes, stream=None):
    h = np.ascontiguousarray(h_header[:64], dtype=np.uint8)
    b = np.ascontiguousarray(h_blob, dtype=np.uint8)
    out = _vp()
    _check(lib().ace_index_import(_ptr(d_archive), archive_bytes, h.ctypes.data, h.size, b.ctypes.data, b.size,
                                  _ptr(d_index_mem), index_bytes, _stream(stream), ctypes.byref(out)),
           "ace_index_import")
    return out


def ace_host_register(h_array, read_only=True):
    """Pins and maps a host numpy array; returns the device address of it."""
    d = _vp()
    _check(lib().ace_host_register(h_array.ctypes.data, h_array.nbytes, 1 if read_only else 0, ctypes.byref(d)),
           "ace_host_register")
    return d.value


def ace_host_unregister(h_array):
    _check(lib().ace_host_unregister(h_array.ctypes.data), "ace_host_unregister")


def ace_scratch_size(idx, max_seek_blocks=0):
    out = _u64()
    _check(lib().ace_scratch_size(idx, max_seek_blocks, ctypes.byref(out)), "ace_scratch_size")
    return out.value


def ace_scratch_init(idx, d_scratch, scratch_bytes, stream=None):
    _check(lib().ace_scratch_init(idx, _ptr(d_scratch), scratch_bytes, _stream(stream)), "ace_scratch_init")


# ------------------------------------------------------------------ decoding

def make_tune(warps_per_cta=0, ctas_per_sm=0, chunk_tokens=0, wait_timeout_ns=0, schedule=0, copy_width=0):
    return ace_tune(warps_per_cta, ctas_per_sm, chunk_tokens, schedule, wait_timeout_ns, copy_width, 0)


def ace_decode_all(idx, d_out, out_bytes, d_scratch, scratch_bytes, tune=None, stream=None):
    t = ctypes.byref(tune) if tune is not None else None
    _check(lib().ace_decode_all(idx, _ptr(d_out), out_bytes, _ptr(d_scratch), scratch_bytes, t,
                                _stream(stream)), "ace_decode_all")


def ace_decode_pass(idx, pass_, d_out, out_bytes, d_scratch, scratch_bytes, tune=None, stream=None):
    t = ctypes.byref(tune) if tune is not None else None
    _check(lib().ace_decode_pass(idx, pass_, _ptr(d_out), out_bytes, _ptr(d_scratch), scratch_bytes, t,
                                 _stream(stream)), "ace_decode_pass")


def ace_seek(idx, coord, length, d_out, out_bytes, d_scratch, scratch_bytes, stream=None):
    _check(lib().ace_seek(idx, coord, length, _ptr(d_out), out_bytes, _ptr(d_scratch), scratch_bytes,
                          _stream(stream)), "ace_seek")


def ace_index_set_tune(idx, tune=None):
    t = ctypes.byref(tune) if tune is not None else None
    _check(lib().ace_index_set_tune(idx, t), "ace_index_set_tune")


def ace_sync(idx, d_scratch, stream=None):
    """Synchronise and return the first device-side status (does not raise)."""
    return lib().ace_sync(idx, _ptr(d_scratch), _stream(stream))


def ace_verify(idx, coord, length, d_buf, guard_bytes, expected_fnv1a64, canary_seed, d_scratch,
               scratch_bytes, stream=None):
    rep = ace_verify_report()
    _check(lib().ace_verify(idx, coord, length, _ptr(d_buf), guard_bytes, expected_fnv1a64, canary_seed,
                            _ptr(d_scratch), scratch_bytes, ctypes.byref(rep), _stream(stream)), "ace_verify")
    return {k: getattr(rep, k) for k, _ in ace_verify_report._fields_}


def ace_fnv1a64(d_p, n, d_result, stream=None):
    _check(lib().ace_fnv1a64(_ptr(d_p), n, _ptr(d_result), _stream(stream)), "ace_fnv1a64")


def ace_seek_noalloc(idx, coord, length, d_out, out_bytes, stream=None):
    """Seek with the library's fixed device scratch (no caller scratch);
    synchronous, returns the device-side status without raising."""
    return lib().ace_seek_noalloc(idx, coord, length, _ptr(d_out), out_bytes, _stream(stream))


# ------------------------------------------------------------------- batches

def _handles(idxs):
    arr = (ctypes.c_void_p * len(idxs))(*[i.value if isinstance(i, ctypes.c_void_p) else i for i in idxs])
    return arr


def ace_batch_scratch_size(idxs):
    out = _u64()
    _check(lib().ace_batch_scratch_size(_handles(idxs), len(idxs), ctypes.byref(out)), "ace_batch_scratch_size")
    return out.value


def ace_batch_create(idxs, d_outs, out_bytes, d_scratch, scratch_bytes, tune=None, stream=None):
    n = len(idxs)
    outs = (ctypes.c_void_p * n)(*[_ptr(o) for o in d_outs])
    sizes = (ctypes.c_uint64 * n)(*out_bytes)
    h = _vp()
    t = ctypes.byref(tune) if tune is not None else None
    _check(lib().ace_batch_create(_handles(idxs), n, outs, sizes, _ptr(d_scratch), scratch_bytes, t,
                                  _stream(stream), ctypes.byref(h)), "ace_batch_create")
    return h


def ace_decode_batch(batch, stream=None):
    _check(lib().ace_decode_batch(batch, _stream(stream)), "ace_decode_batch")


def ace_batch_sync(batch, stream=None):
    return lib().ace_batch_sync(batch, _stream(stream))


def ace_batch_launch_shape(batch):
    g, w, c = _u32(), _u32(), _u32()
    _check(lib().ace_batch_launch_shape(batch, ctypes.byref(g), ctypes.byref(w), ctypes.byref(c)),
           "ace_batch_launch_shape")
    return {"grid": g.value, "warps_per_cta": w.value, "window": c.value}


def ace_batch_free(batch):
    lib().ace_batch_free(batch)


# ------------------------------------------------------ seek batches (cache)

SEEK_REQ = np.dtype([("archive", np.uint32), ("reserved", np.uint32), ("coord", np.uint64),
                     ("len", np.uint64), ("out_off", np.uint64)])


def ace_archive_state_size(idx):
    out = _u64()
    _check(lib().ace_archive_state_size(idx, ctypes.byref(out)), "ace_archive_state_size")
    return out.value


def ace_cache_size(idxs, n_slots, max_reqs):
    out = _u64()
    _check(lib().ace_cache_size(_handles(idxs), len(idxs), n_slots, max_reqs, ctypes.byref(out)), "ace_cache_size")
    return out.value


def ace_cache_create(idxs, d_states, n_slots, max_reqs, d_mem, mem_bytes, tune=None, stream=None):
    n = len(idxs)
    st = (ctypes.c_void_p * n)(*[_ptr(x) for x in d_states])
    h = _vp()
    t = ctypes.byref(tune) if tune is not None else None
    _check(lib().ace_cache_create(_handles(idxs), n, st, n_slots, max_reqs, _ptr(d_mem), mem_bytes, t,
                                  _stream(stream), ctypes.byref(h)), "ace_cache_create")
    return h


def ace_seek_batch(cache, d_reqs, n, d_pool, pool_bytes, stream=None):
    _check(lib().ace_seek_batch(cache, _ptr(d_reqs), n, _ptr(d_pool), pool_bytes, _stream(stream)),
           "ace_seek_batch")


def ace_seek_batch_host(cache, h_reqs, h_totals, d_pool, pool_bytes, stream=None):
    """h_reqs: numpy array of SEEK_REQ; h_totals: numpy uint64 sizes or None."""
    r = np.ascontiguousarray(h_reqs, dtype=SEEK_REQ)
    tot = None if h_totals is None else np.ascontiguousarray(h_totals, dtype=np.uint64)
    _check(lib().ace_seek_batch_host(cache, r.ctypes.data, None if tot is None else tot.ctypes.data, r.size,
                                     _ptr(d_pool), pool_bytes, _stream(stream)), "ace_seek_batch_host")


def ace_cache_sync(cache, stream=None):
    return lib().ace_cache_sync(cache, _stream(stream))


def ace_cache_usage(cache, stream=None):
    u, n = _u32(), _u32()
    _check(lib().ace_cache_usage(cache, ctypes.byref(u), ctypes.byref(n), _stream(stream)), "ace_cache_usage")
    return u.value, n.value


def ace_cache_reset(cache, stream=None):
    _check(lib().ace_cache_reset(cache, _stream(stream)), "ace_cache_reset")


def ace_cache_counters(cache, stream=None):
    """(blocks evicted, blocks decoded) since the cache was created."""
    e, d = _u64(), _u64()
    _check(lib().ace_cache_counters(cache, ctypes.byref(e), ctypes.byref(d), _stream(stream)), "ace_cache_counters")
    return e.value, d.value


def ace_cache_limits(cache):
    """(slots, blocks one batch may decode, requests one batch may hold)."""
    a, b, c = _u32(), _u32(), _u32()
    _check(lib().ace_cache_limits(cache, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "ace_cache_limits")
    return a.value, b.value, c.value


def ace_cache_free(cache):
    lib().ace_cache_free(cache)
