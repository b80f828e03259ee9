"""Batched decode of many independent archives in one persistent launch,
replayable as a CUDA graph, with an autotuner for the launch shape.

Device memory comes from PyTorch; every step runs in libace.so's kernels."""
import json
import os
import time

import numpy as np
import torch

from . import ace
from .archive import DeviceArchive


class DeviceBatch:
    """Archives resident on one GPU, their outputs packed in one buffer
    (each 256-byte aligned), and an ace_batch over them."""

    def __init__(self, archives, tune=None, device="cuda", stream=None):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.items = [DeviceArchive(a, device=self.device, stream=self.stream, scratch=False) for a in archives]
        self.sizes = [x.total for x in self.items]
        offs, o = [], 0
        for n in self.sizes:
            offs.append(o)
            o += (n + 255) & ~255
        self.offsets = offs
        self.out = torch.empty(max(o, 256), dtype=torch.uint8, device=self.device)
        self.scratch_bytes = ace.ace_batch_scratch_size([x.idx for x in self.items])
        self.d_scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=self.device)
        self.batch = None
        self.retune(tune)

    def retune(self, tune=None):
        if self.batch is not None:
            ace.ace_batch_free(self.batch)
        base = self.out.data_ptr()
        self.batch = ace.ace_batch_create([x.idx for x in self.items], [base + o for o in self.offsets],
                                          self.sizes, self.d_scratch, self.scratch_bytes, tune, self.stream)
        self.tune = tune
        return ace.ace_batch_launch_shape(self.batch)

    def decode(self):
        ace.ace_decode_batch(self.batch, self.stream)

    def sync(self):
        return ace.ace_batch_sync(self.batch, self.stream)

    def output(self, i):
        return self.out[self.offsets[i]: self.offsets[i] + self.sizes[i]]

    def capture(self):
        """A CUDA graph whose replay decodes the whole batch."""
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(g):
            ace.ace_decode_batch(self.batch, torch.cuda.current_stream(self.device))
        return g

    def close(self):
        if self.batch is not None:
            ace.ace_batch_free(self.batch)
            self.batch = None
        for x in self.items:
            x.close()


TUNE_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ace_gb300", "tune.json")


def autotune(db, candidates=None, reps=3, cache_key=None, cache_path=TUNE_CACHE):
    """Times each (warps per CTA, token window, schedule, copy width)
    candidate on the batch and keeps the fastest; results are cached by
    cache_key in a JSON file."""
    def tune_of(c):
        return ace.make_tune(c["warps_per_cta"], 0, c["window"], schedule=c.get("schedule", 0),
                             copy_width=c.get("copy_width", 0))

    if cache_key is not None and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                hit = json.load(f).get(cache_key)
            if hit:
                db.retune(tune_of(hit))
                return hit
        except (OSError, ValueError):
            pass
    if candidates is None:
        candidates = [(w, c, s, cw) for s in (ace.ACE_SCHEDULE_PASSES, ace.ACE_SCHEDULE_FUSED)
                      for w in (1, 2, 4, 8) for c in (64, 128, 256) for cw in (8, 16)]
    best = None
    results = []
    for cand in candidates:
        w, c = cand[0], cand[1]
        sch = cand[2] if len(cand) > 2 else ace.ACE_SCHEDULE_PASSES
        cw = cand[3] if len(cand) > 3 else 0
        try:
            db.retune(ace.make_tune(w, 0, c, schedule=sch, copy_width=cw))
        except ace.AceError:
            continue
        db.decode()
        if db.sync() != ace.ACE_OK:
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(reps):
            e0.record(db.stream)
            db.decode()
            e1.record(db.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        row = {"warps_per_cta": w, "window": c, "schedule": sch, "copy_width": cw, "ms": ms}
        results.append(row)
        if best is None or ms < best["ms"]:
            best = dict(row)
    db.retune(tune_of(best))
    best = dict(best, sweep=results)
    if cache_key is not None:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            data = {}
            if os.path.exists(cache_path):
                with open(cache_path) as f:
                    data = json.load(f)
            data[cache_key] = best
            with open(cache_path, "w") as f:
                json.dump(data, f, indent=1)
        except (OSError, ValueError):
            pass
    return best


def make_objects(count, seed=4, min_size=4096, max_size=1 << 26, seed_base=1000, workers=0, stats=False,
                 encoder="host", device="cuda"):
    """The uneven batch workload: (originals, archives[, parse statistics])
    for count objects with log-uniform sizes, a random profile and block size
    each (the synth module's object table).  Objects are generated on a
    thread pool (the native calls release the interpreter lock); encoder
    "host" encodes them there too, one encoder thread each, "gpu" with the
    GPU encoder as they come."""
    from concurrent.futures import ThreadPoolExecutor

    import synth

    sizes, profiles, bsz, seeds = synth.objects(seed, count, min_size, max_size, seed_base)
    mm = {0: 16, 1: 20, 2: 4, 3: 4}

    def one(k):
        d = synth.generate(int(profiles[k]), int(sizes[k]), int(seeds[k]))
        log2b = int(bsz[k]).bit_length() - 1
        if encoder == "gpu":
            return d, log2b
        arc, st = ace.ace_encode(d, log2b, mm[int(profiles[k])], threads=1, stats=True)
        return d, arc, st

    if encoder == "gpu":
        res = [None] * count
        with ThreadPoolExecutor(workers or os.cpu_count() or 4) as ex:
            for k, (d, log2b) in enumerate(ex.map(one, range(count))):
                arc, st = ace.ace_encode_gpu(torch.from_numpy(d).to(device), log2b, mm[int(profiles[k])], stats=True)
                res[k] = (d, arc.cpu().numpy(), st)
        if stats:
            return [r[0] for r in res], [r[1] for r in res], [r[2] for r in res]
        return [r[0] for r in res], [r[1] for r in res]

    # the largest objects first, so the pool ends on small ones
    order = sorted(range(count), key=lambda k: -int(sizes[k]))
    res = [None] * count
    with ThreadPoolExecutor(workers or os.cpu_count() or 4) as ex:
        for k, r in zip(order, ex.map(one, order)):
            res[k] = r
    if stats:
        return [r[0] for r in res], [r[1] for r in res], [r[2] for r in res]
    return [r[0] for r in res], [r[1] for r in res]


def time_per_object(items, out_views, reps=1):
    """The plain alternative: one ace_decode_all launch sequence per object,
    on one stream; returns the total device time in ms (events around the
    whole sequence).  One scratch buffer, sized for the largest object,
    serves every call: calls on one stream run in order, and a whole decode
    of these archives (at most 32 dependency levels) uses only the scratch
    header and its match records, both rewritten by the call."""
    st = torch.cuda.current_stream()
    nbytes = max(ace.ace_scratch_size(x.idx, 0) for x in items)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=items[0].device)
    assert all(x.info["n_levels"] <= 32 for x in items)
    for x in items:
        ace.ace_scratch_init(x.idx, scratch, nbytes, st)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for x, o in zip(items, out_views):
            ace.ace_decode_all(x.idx, o, o.numel(), scratch, nbytes, None, st)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    assert ace.ace_sync(items[0].idx, scratch, st) == ace.ACE_OK
    return best
