"""Seeded synthetic inputs shared by the oracle tests and the GPU library's
benchmark.

Holds no codec arithmetic: it only generates original byte strings shaped
like the paper's four data profiles (Section 6, Table 1: FASTQ reads, a
repetitive genome, English text, mixed data) and the workload tables that
drive a run (object sizes, seek targets, request arrivals).  The C source is
``synth.c``; this module compiles it on first use with gcc.
"""
import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "synth.c")
_LIB = os.path.join(_DIR, "libsynth.so")

PROFILES = {"fastq": 0, "genome": 1, "text": 2, "mixed": 3}
PROFILE_NAMES = {v: k for k, v in PROFILES.items()}


def build(force=False):
    """Compile synth.c into libsynth.so (plain gcc, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, i32, u32, dbl, vp = (ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.synth_profile.argtypes = [i32, vp, u64, u64]
        lib.synth_profile.restype = u64
        lib.synth_mixed.argtypes = [vp, u64, u64, dbl]
        lib.synth_mixed.restype = u64
        lib.synth_objects.argtypes = [u64, u32, u64, u64, u64, vp, vp, vp, vp]
        lib.synth_uniform.argtypes = [u64, u32, u64, u64, vp]
        lib.synth_log_uniform.argtypes = [u64, u32, u64, u64, vp]
        lib.synth_requests.argtypes = [u64, u32, dbl, u32, vp, u64, u64, vp, vp, vp, vp]
        lib.synth_det_log.argtypes = [dbl]
        lib.synth_det_log.restype = dbl
        lib.synth_det_exp.argtypes = [dbl]
        lib.synth_det_exp.restype = dbl
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def generate(profile, n, seed, out=None):
    """Return (or fill) a uint8 array of n bytes of the named profile."""
    p = PROFILES[profile] if isinstance(profile, str) else int(profile)
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= n
    got = _L().synth_profile(p, _ptr(out), n, seed)
    if got != n:
        raise RuntimeError("synth: generator %r produced %d of %d bytes" % (profile, got, n))
    return out[:n]


def mixed(n, seed, copy_frac=0.4):
    out = np.empty(n, dtype=np.uint8)
    got = _L().synth_mixed(_ptr(out), n, seed, copy_frac)
    if got != n:
        raise RuntimeError("synth: mixed produced %d of %d bytes" % (got, n))
    return out


def objects(seed, count, min_size=4096, max_size=1 << 26, seed_base=1000):
    """The uneven-batch table: (sizes, profiles, block_sizes, seeds)."""
    sizes = np.empty(count, np.uint64)
    profiles = np.empty(count, np.int32)
    bsz = np.empty(count, np.uint32)
    seeds = np.empty(count, np.uint64)
    _L().synth_objects(seed, count, min_size, max_size, seed_base,
                       _ptr(sizes), _ptr(profiles), _ptr(bsz), _ptr(seeds))
    return sizes, profiles, bsz, seeds


def uniform(seed, count, lo, hi):
    out = np.empty(count, np.uint64)
    _L().synth_uniform(seed, count, lo, hi, _ptr(out))
    return out


def log_uniform(seed, count, lo, hi):
    out = np.empty(count, np.uint64)
    _L().synth_log_uniform(seed, count, lo, hi, _ptr(out))
    return out


def requests(seed, count, rate, sizes, len_lo=1 << 14, len_hi=1 << 20):
    """Poisson seek requests: (t_ns, archive, coord, len)."""
    sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
    t = np.empty(count, np.uint64)
    a = np.empty(count, np.uint32)
    c = np.empty(count, np.uint64)
    ln = np.empty(count, np.uint64)
    _L().synth_requests(seed, count, float(rate), sizes.size, _ptr(sizes), len_lo, len_hi,
                        _ptr(t), _ptr(a), _ptr(c), _ptr(ln))
    return t, a, c, ln


def det_log(x):
    return _L().synth_det_log(float(x))


def det_exp(x):
    return _L().synth_det_exp(float(x))
