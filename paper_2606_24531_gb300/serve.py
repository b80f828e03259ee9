"""Seek serving over resident archives: a decoded-block cache per in-flight
stream, and a continuous-batching request loop.

Requests that arrive while earlier batches are on the GPU are admitted as
soon as a cache (its slots and output pool) is free, so batches on several
streams overlap on the device.  The device working set -- caches, output
pools and per-archive seek state -- is fixed up front against a byte budget.
Every decode runs in libace.so; PyTorch provides memory, streams and events.
"""
import collections
import time

import numpy as np
import torch

from . import ace


class SeekCache:
    """A decoded-block cache over archives sharing one block size, with its
    own stream and output pool."""

    def __init__(self, archives, n_slots, max_reqs, pool_bytes, device="cuda", stream=None, tune=None):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.archives = archives
        idxs = [a.idx for a in archives]
        self.states = [torch.empty(ace.ace_archive_state_size(a.idx), dtype=torch.uint8, device=self.device)
                       for a in archives]
        self.mem_bytes = ace.ace_cache_size(idxs, n_slots, max_reqs)
        self.mem = torch.empty(self.mem_bytes, dtype=torch.uint8, device=self.device)
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=self.device)
        self.cache = ace.ace_cache_create(idxs, self.states, n_slots, max_reqs, self.mem, self.mem_bytes, tune,
                                          self.stream)
        self.totals = np.array([a.total for a in archives], np.uint64)
        self.n_slots, self.max_reqs, self.pool_bytes = n_slots, max_reqs, pool_bytes
        self.status_host = torch.zeros(4, dtype=torch.uint8).pin_memory()
        self.done = torch.cuda.Event()

    def working_set_bytes(self):
        return self.mem_bytes + self.pool_bytes + sum(s.numel() for s in self.states)

    def plan(self, reqs):
        """Request array for [(archive, coord, len)], results packed 16-byte
        aligned in the pool; None if they do not fit one batch."""
        if not len(reqs):
            return np.zeros(0, ace.SEEK_REQ)
        a, c, n = (np.asarray(x, np.uint64) for x in zip(*reqs))
        return self.plan_arrays(a, c, n)

    def plan_arrays(self, archive, coord, length):
        """plan() for parallel arrays of archive ids, coordinates and lengths."""
        n = len(coord)
        r = np.zeros(n, ace.SEEK_REQ)
        r["archive"] = archive
        r["coord"] = coord
        r["len"] = length
        aligned = (np.asarray(length, np.uint64) + np.uint64(15)) & ~np.uint64(15)
        ends = np.cumsum(aligned, dtype=np.uint64)
        r["out_off"][1:] = ends[:-1]
        if (n and int(ends[-1]) > self.pool_bytes) or n > self.max_reqs:
            return None
        return r

    def submit(self, r):
        """Enqueue a batch (asynchronous) and the copy of its status word."""
        ace.ace_seek_batch_host(self.cache, r, self.totals, self.pool, self.pool_bytes, self.stream)
        with torch.cuda.stream(self.stream):
            self.status_host.copy_(self.mem[:4], non_blocking=True)
            self.done.record(self.stream)

    def status(self):
        """Device status of the last batch, once self.done has completed."""
        return int.from_bytes(bytes(self.status_host.numpy()), "little")

    def sync(self):
        return ace.ace_cache_sync(self.cache, self.stream)

    def reset(self):
        ace.ace_cache_reset(self.cache, self.stream)

    def run_batch(self, r):
        """Blocking: runs the planned batch r (resetting the cache once if it
        ran out of slots); the results are in the pool at r["out_off"]."""
        for attempt in range(2):
            self.submit(r)
            st = self.sync()
            if st == ace.ACE_OK:
                return r
            if st != ace.ACE_E_NOMEM or attempt:
                raise ace.AceError(st, "seek batch")
            self.reset()
        raise AssertionError("unreachable")

    def seek_many(self, reqs):
        """Blocking convenience: results of [(archive, coord, len)] as pool views."""
        r = self.plan(reqs)
        assert r is not None, "batch larger than the pool"
        self.run_batch(r)
        return [self.pool[int(q["out_off"]): int(q["out_off"]) + int(q["len"])] for q in r]

    def close(self):
        if self.cache is not None:
            ace.ace_cache_free(self.cache)
            self.cache = None


class Server:
    """Continuous batching of seeks under a device working-set budget."""

    def __init__(self, archives, budget_bytes, n_streams=2, max_batch=256, pool_bytes=64 << 20, device="cuda",
                 tune=None):
        self.archives = archives
        state = sum(ace.ace_archive_state_size(a.idx) for a in archives)
        per = budget_bytes // n_streams - pool_bytes - state
        idxs = [a.idx for a in archives]
        lo, hi = 1, max(1, per // archives[0].block_size)
        if ace.ace_cache_size(idxs, lo, max_batch) > per:
            raise ace.AceError(ace.ACE_E_NOMEM, "serving budget below one cache slot per stream")
        while lo < hi:  # the most slots whose cache fits the per-stream share
            mid = (lo + hi + 1) // 2
            if ace.ace_cache_size(idxs, mid, max_batch) <= per:
                lo = mid
            else:
                hi = mid - 1
        n_slots = lo
        self.caches = []
        for _ in range(n_streams):
            self.caches.append(SeekCache(archives, n_slots, max_batch, pool_bytes, device=device, tune=tune))
        self.budget = budget_bytes
        self.max_batch = max_batch

    def working_set_bytes(self):
        return sum(c.working_set_bytes() for c in self.caches)

    def run(self, t_ns, archive, coord, length, keep=None, time_limit_s=None):
        """Serves requests arriving at t_ns (ns from the start) in real time.
        Returns latencies (ns, -1 for requests not served), bytes served,
        elapsed seconds, batches, resets and, for ids in keep, their bytes."""
        n = len(t_ns)
        lat = np.full(n, -1, np.int64)
        kept = {}
        queue = collections.deque()
        busy = {}
        nxt = 0
        served = 0
        resets = 0
        batches = 0
        bytes_out = 0
        start = time.perf_counter_ns()
        deadline = None if time_limit_s is None else start + int(time_limit_s * 1e9)
        while served < n:
            now = time.perf_counter_ns()
            if deadline is not None and now > deadline and not busy:
                break
            while nxt < n and t_ns[nxt] <= now - start and (deadline is None or now <= deadline):
                queue.append(nxt)
                nxt += 1
            for ci in list(busy):
                c = self.caches[ci]
                if not c.done.query():
                    continue
                ids, r = busy.pop(ci)
                st = c.status()
                if st == ace.ACE_E_NOMEM:  # out of slots: forget the cache, run the batch again
                    c.sync()
                    c.reset()
                    resets += 1
                    c.submit(r)
                    busy[ci] = (ids, r)
                    continue
                if st != ace.ACE_OK:
                    raise ace.AceError(st, "seek batch")
                t_done = time.perf_counter_ns() - start
                for k, rid in enumerate(ids):
                    lat[rid] = t_done - int(t_ns[rid])
                    if keep is not None and rid in keep:
                        o, ln = int(r[k]["out_off"]), int(r[k]["len"])
                        kept[rid] = c.pool[o:o + ln].cpu().numpy().copy()
                served += len(ids)
                bytes_out += int(r["len"].sum())
            for ci, c in enumerate(self.caches):
                if ci in busy or not queue:
                    continue
                ids, reqs, used = [], [], 0
                while queue and len(ids) < self.max_batch:
                    rid = queue[0]
                    ln = int(length[rid])
                    if used + ((ln + 15) & ~15) > c.pool_bytes:
                        break
                    queue.popleft()
                    ids.append(rid)
                    reqs.append((int(archive[rid]), int(coord[rid]), ln))
                    used += (ln + 15) & ~15
                r = c.plan(reqs)
                c.submit(r)
                busy[ci] = (ids, r)
                batches += 1
            if not busy and not queue and nxt < n:
                wait = int(t_ns[nxt]) - (time.perf_counter_ns() - start)
                if wait > 50_000:
                    time.sleep(wait / 1e9 * 0.5)
        elapsed = (time.perf_counter_ns() - start) / 1e9
        return {"latency_ns": lat, "bytes": bytes_out, "seconds": elapsed, "batches": batches, "resets": resets,
                "served": int((lat >= 0).sum()), "kept": kept}

    def close(self):
        for c in self.caches:
            c.close()


def plain_latencies(archives, scratches, archive, coord, length, limit=None):
    """The plain path: one ace_seek and one ace_sync per request, in order;
    per-request wall-clock latency in ns."""
    st = torch.cuda.current_stream()
    out = torch.empty(int(max(length)), dtype=torch.uint8, device=archives[0].device)
    m = len(coord) if limit is None else min(limit, len(coord))
    lat = np.zeros(m, np.int64)
    for k in range(m):
        a = archives[int(archive[k])]
        sc = scratches[int(archive[k])]
        t0 = time.perf_counter_ns()
        ace.ace_seek(a.idx, int(coord[k]), int(length[k]), out, out.numel(), sc, sc.numel(), st)
        s = ace.ace_sync(a.idx, sc, st)
        lat[k] = time.perf_counter_ns() - t0
        assert s == ace.ACE_OK, ace.ace_status_str(s)
    return lat
