"""Device residency for one archive: PyTorch allocates the archive, index,
scratch and output buffers; every operation is a call into libace.so."""
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
    """

    def __init__(self, h_arc, max_seek_blocks=0, device="cuda", stream=None, scratch=True):
        h_arc = np.ascontiguousarray(h_arc, dtype=np.uint8)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h_header = h_arc[:64].copy()
        with torch.cuda.device(self.device):
            self.d_arc = torch.from_numpy(h_arc).to(self.device)
            self.index_bytes = ace.ace_index_size(self.h_header)
            self.d_index = torch.empty(self.index_bytes, dtype=torch.uint8, device=self.device)
            torch.cuda.current_stream(self.device).synchronize()
            self.idx = ace.ace_index_build(self.d_arc, h_arc.size, self.h_header, self.d_index,
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
