"""Device residency for one archive: PyTorch allocates the archive, index,
scratch and output buffers; every operation is a call into libace.so."""
import os

import numpy as np
import torch

from . import ace


STREAM_NAMES = ("literals", "lengths", "offsets")


def stream_report(h_arc):
    """Per token stream, from the archive's directory: symbol bytes (raw),
    bytes as stored, raw / stored (below 1: the coding inflated the stream),
    and how many blocks store the stream verbatim (mode 1) -- the per-stream
    view of Section 4's finding that entropy coding pays only on some data."""
    a = np.ascontiguousarray(h_arc, dtype=np.uint8)
    hdr = a[:64].view(np.uint64)
    nb, dir_off = int(hdr[3]), int(hdr[4])
    d = a[dir_off:dir_off + 64 * nb].reshape(nb, 64)
    stored = d[:, 24:36].copy().view(np.uint32).astype(np.int64)
    raw = d[:, 36:48].copy().view(np.uint32).astype(np.int64)
    mode = d[:, 56:59]
    rep = {}
    for k, name in enumerate(STREAM_NAMES):
        r, st = int(raw[:, k].sum()), int(stored[:, k].sum())
        rep[name] = {"raw": r, "stored": st, "ratio": r / st if st else None,
                     "stored_verbatim_blocks": int((mode[:, k] == 1).sum())}
    return rep


class DeviceArchive:
    """An archive resident on one GPU with its block index built.

    ``max_seek_blocks`` sizes the seek scratch (blocks one seek may decode,
    including the blocks its matches read); 0 sizes it for whole decodes only.
    ``h_arc`` may be a file name; ``index`` a stored index (bytes or a file
    name, see save_index) loaded instead of built.
    """

    def __init__(self, h_arc, max_seek_blocks=0, device="cuda", stream=None, scratch=True, index=None):
        if isinstance(h_arc, str):
            h_arc = load_archive(h_arc)
        if isinstance(index, str):
            index = np.fromfile(index, dtype=np.uint8)
        h_arc = np.ascontiguousarray(h_arc, dtype=np.uint8)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h_header = h_arc[:64].copy()
        with torch.cuda.device(self.device):
            self.d_arc = torch.from_numpy(h_arc).to(self.device)
            self.index_bytes = ace.ace_index_size(self.h_header)
            self.d_index = torch.empty(self.index_bytes, dtype=torch.uint8, device=self.device)
            torch.cuda.current_stream(self.device).synchronize()
            if index is None:
                self.idx = ace.ace_index_build(self.d_arc, h_arc.size, self.h_header, self.d_index,
                                               self.index_bytes, self.stream)
            else:  # a stored index, checked against the archive instead of rebuilt
                self.idx = ace.ace_index_import(self.d_arc, h_arc.size, self.h_header, index, self.d_index,
                                                self.index_bytes, self.stream)
        self.info = ace.ace_index_info(self.idx)
        self.total = self.info["total_size"]
        self.block_size = self.info["block_size"]
        self.max_seek_blocks = max_seek_blocks
        self.scratch_bytes = 0
        self.d_scratch = None
        if scratch:
            self.scratch_bytes = ace.ace_scratch_size(self.idx, max_seek_blocks)
            self.d_scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=self.device)
            ace.ace_scratch_init(self.idx, self.d_scratch, self.scratch_bytes, self.stream)

    def new_scratch(self, max_seek_blocks):
        """A separate scratch buffer, for calls that overlap on the device."""
        nbytes = ace.ace_scratch_size(self.idx, max_seek_blocks)
        buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        ace.ace_scratch_init(self.idx, buf, nbytes, self.stream)
        return buf

    def decode_all(self, out=None, tune=None, scratch=None):
        if out is None:
            out = torch.empty(max(self.total, 1), dtype=torch.uint8, device=self.device)
        sc = self.d_scratch if scratch is None else scratch
        ace.ace_decode_all(self.idx, out, out.numel(), sc, sc.numel(), tune, self.stream)
        return out

    def seek(self, coord, length, out=None, scratch=None):
        if out is None:
            out = torch.empty(max(length, 1), dtype=torch.uint8, device=self.device)
        sc = self.d_scratch if scratch is None else scratch
        ace.ace_seek(self.idx, coord, length, out, out.numel(), sc, sc.numel(), self.stream)
        return out

    def sync(self, scratch=None):
        sc = self.d_scratch if scratch is None else scratch
        return ace.ace_sync(self.idx, sc, self.stream)

    def verify(self, coord, length, expected_fnv1a64, guard_bytes=None, canary_seed=12345):
        g = self.block_size if guard_bytes is None else guard_bytes
        buf = torch.empty(length + 2 * g, dtype=torch.uint8, device=self.device)
        rep = ace.ace_verify(self.idx, coord, length, buf, g, expected_fnv1a64, canary_seed,
                             self.d_scratch, self.scratch_bytes, self.stream)
        return rep, buf

    def close(self):
        if self.idx is not None:
            ace.ace_index_free(self.idx)
            self.idx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def save_archive(path, h_arc):
    """Writes an archive's bytes to a file (the archive is its own storage
    format)."""
    np.ascontiguousarray(h_arc, dtype=np.uint8).tofile(path)


def page_aligned(n, page=4096):
    """An uninitialised numpy uint8 array of n bytes starting on a page
    boundary (host memory the GPU is to read in place is pinned by pages)."""
    raw = np.empty(n + page, dtype=np.uint8)
    off = (-raw.ctypes.data) % page
    return raw[off:off + n]


def load_archive(path, aligned=False):
    """An archive file's bytes as a numpy uint8 array (page-aligned when
    aligned is set)."""
    if not aligned:
        return np.fromfile(path, dtype=np.uint8)
    n = os.path.getsize(path)
    out = page_aligned(n)
    with open(path, "rb") as f:
        f.readinto(memoryview(out))
    return out


def save_index(path, da):
    """Writes the stored form of a resident archive's index to a file."""
    ace.ace_index_export(da.idx, da.stream).tofile(path)


class HostArchive(DeviceArchive):
    """An archive that stays in host memory (for archives that, with their
    output, exceed device memory): its bytes are pinned and mapped so the GPU
    reads them in place, across the chip-to-chip link; the index and the
    seek scratch live on the device.  Built from the archive's bytes or a
    file, with an optional stored index (bytes or a file) loaded instead of
    rebuilt."""

    def __init__(self, h_arc, max_seek_blocks=4096, device="cuda", stream=None, index=None):
        if isinstance(h_arc, str):
            h_arc = load_archive(h_arc, aligned=True)
        h_arc = np.ascontiguousarray(h_arc, dtype=np.uint8)
        if h_arc.ctypes.data % 4096:
            a = page_aligned(h_arc.size)
            a[:] = h_arc
            h_arc = a
        self.h_arc = h_arc
        if isinstance(index, str):
            index = np.fromfile(index, dtype=np.uint8)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h_header = self.h_arc[:64].copy()
        self.idx = None
        with torch.cuda.device(self.device):
            self.d_arc_ptr = ace.ace_host_register(self.h_arc, read_only=True)
            self.d_arc = None
            self.index_bytes = ace.ace_index_size(self.h_header)
            self.d_index = torch.empty(self.index_bytes, dtype=torch.uint8, device=self.device)
            torch.cuda.current_stream(self.device).synchronize()
            if index is None:
                self.idx = ace.ace_index_build(self.d_arc_ptr, self.h_arc.size, self.h_header, self.d_index,
                                               self.index_bytes, self.stream)
            else:
                self.idx = ace.ace_index_import(self.d_arc_ptr, self.h_arc.size, self.h_header, index,
                                                self.d_index, self.index_bytes, self.stream)
        self.info = ace.ace_index_info(self.idx)
        self.total = self.info["total_size"]
        self.block_size = self.info["block_size"]
        self.max_seek_blocks = max_seek_blocks
        self.scratch_bytes = ace.ace_scratch_size(self.idx, max_seek_blocks)
        self.d_scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=self.device)
        ace.ace_scratch_init(self.idx, self.d_scratch, self.scratch_bytes, self.stream)

    def decode_range_to_host(self, coord, length, h_out=None, chunk_blocks=2048):
        """[coord, coord + length) decoded into host memory in sub-ranges of
        chunk_blocks blocks, two in flight: each is a seek (its blocks and
        the blocks they read, decoded from the host-resident archive into
        device scratch) followed by a device-to-host copy on its own stream.
        Returns the pinned host tensor holding the range."""
        B = self.block_size
        end = coord + length
        if h_out is None:
            h_out = torch.empty(length, dtype=torch.uint8).pin_memory()
        slack = min(self.info["n_blocks"], chunk_blocks + 8192)  # the closure's source blocks
        lanes = []
        for _ in range(2):
            st = torch.cuda.Stream(self.device)
            lanes.append({"stream": st, "buf": torch.empty(chunk_blocks * B, dtype=torch.uint8, device=self.device),
                          "scratch": self.new_scratch(slack), "event": None})
        torch.cuda.synchronize(self.device)
        pos, k = coord, 0
        while pos < end:
            n = min(chunk_blocks * B - (pos % B), end - pos)  # sub-ranges end on block boundaries
            ln = lanes[k % 2]
            if ln["event"] is not None:
                ln["event"].synchronize()
            sc = ln["scratch"]
            ace.ace_seek(self.idx, pos, n, ln["buf"], ln["buf"].numel(), sc, sc.numel(), ln["stream"])
            with torch.cuda.stream(ln["stream"]):
                h_out[pos - coord:pos - coord + n].copy_(ln["buf"][:n], non_blocking=True)
                ln["event"] = torch.cuda.Event()
                ln["event"].record(ln["stream"])
            pos += n
            k += 1
        for ln in lanes:
            st = ace.ace_sync(self.idx, ln["scratch"], ln["stream"])
            if st != ace.ACE_OK:
                raise ace.AceError(st, "range decode")
        return h_out

    def close(self):
        if self.idx is not None:
            ace.ace_index_free(self.idx)
            self.idx = None
        if getattr(self, "d_arc_ptr", None):
            torch.cuda.synchronize(self.device)
            ace.ace_host_unregister(self.h_arc)
            self.d_arc_ptr = None
