"""Seek serving over resident archives: decoded-block caches, one per
in-flight stream, and a continuous-batching request loop.

The archives are partitioned over the streams (archive i is served by cache
i mod the stream count), so no block is ever held by two caches, and each
cache is driven by one stream, so its batches are ordered.  Requests that
arrive while batches are on the GPU wait in their cache's queue and are
admitted as soon as that cache's previous batch completes, so the batches of
different caches overlap on the device.  Inside a cache, a clock evicts the
blocks least recently used when new ones need slots (the library's cache
kernels).  The device working set -- caches, output pools and per-archive
seek state -- is fixed up front against a byte budget.

Admission: a request longer than its cache's output pool, or covering more
blocks than one batch may decode, is rejected at once (ACE_E_NOMEM).  A
batch the device refuses for want of slots is split in half and both halves
served in turn; a single request refused on its own is rejected.  No batch
is ever empty.  Every decode runs in libace.so; PyTorch provides memory,
streams and events.
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
        self.max_work = ace.ace_cache_limits(self.cache)[1]
        self.block_size = archives[0].block_size
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
        assert len(r) > 0, "an empty batch"
        ace.ace_seek_batch_host(self.cache, r, self.totals, self.pool, self.pool_bytes, self.stream)
        with torch.cuda.stream(self.stream):
            self.status_host.copy_(self.mem[:4], non_blocking=True)
            self.done.record(self.stream)

    def query(self):
        return self.done.query()

    def status(self):
        """Device status of the last batch, once self.done has completed."""
        return int.from_bytes(bytes(self.status_host.numpy()), "little")

    def clear_status(self):
        """Reads and clears the device status (after a refused batch)."""
        return ace.ace_cache_sync(self.cache, self.stream)

    def result(self, r, k):
        o, ln = int(r[k]["out_off"]), int(r[k]["len"])
        return self.pool[o:o + ln]

    def sync(self):
        return ace.ace_cache_sync(self.cache, self.stream)

    def reset(self):
        ace.ace_cache_reset(self.cache, self.stream)

    def counters(self):
        """(blocks evicted, blocks decoded) since creation."""
        return ace.ace_cache_counters(self.cache, self.stream)

    def run_batch(self, r):
        """Blocking: runs the planned batch r; a batch refused for want of
        slots is served in halves.  The results are in the pool at
        r["out_off"] (halves are planned into the same places)."""
        self.submit(r)
        st = self.sync()
        if st == ace.ACE_OK:
            return r
        if st != ace.ACE_E_NOMEM or len(r) == 1:
            raise ace.AceError(st, "seek batch")
        h = len(r) // 2
        self.run_batch(r[:h])
        self.run_batch(r[h:])
        return r

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


def serve_loop(caches, route, t_ns, archive, coord, length, keep=None, time_limit_s=None, clock=None,
               idle=None):
    """Continuous batching over caches, in real time.

    caches: objects with plan_arrays, submit, query, status, clear_status,
    result, pool_bytes, max_reqs, max_work, block_size.  route[a] = (cache,
    archive's place in that cache).  Requests arrive at t_ns (ns from the
    start); each waits in its cache's queue until that cache is idle, then
    joins the next batch (up to max_reqs requests and the pool).  Returns
    latencies (ns, -1 for requests not served), the status per request
    (ACE_OK served, ACE_E_NOMEM rejected, -1 not reached in time), bytes
    served, elapsed seconds, batch and split counts, and for ids in keep
    their bytes."""
    clock = clock or time.perf_counter_ns
    n = len(t_ns)
    lat = np.full(n, -1, np.int64)
    status = np.full(n, -1, np.int32)
    kept = {}
    queues = [collections.deque() for _ in caches]
    busy = {}  # cache -> (request ids, planned batch)
    nxt = 0
    done = 0
    batches = splits = 0
    bytes_out = 0
    start = clock()
    deadline = None if time_limit_s is None else start + int(time_limit_s * 1e9)

    def blocks_of(rid, c):
        B = c.block_size
        return (int(coord[rid]) + int(length[rid]) - 1) // B - int(coord[rid]) // B + 1

    def plan(c, ids):
        ci = caches.index(c)
        a = np.array([route[int(archive[i])][1] for i in ids], np.uint32)
        r = c.plan_arrays(a, np.asarray([coord[i] for i in ids], np.uint64),
                          np.asarray([length[i] for i in ids], np.uint64))
        assert r is not None, "batch planned beyond cache %d's pool" % ci
        return r

    while done < n:
        now = clock()
        if deadline is not None and now > deadline and not busy:
            break
        while nxt < n and t_ns[nxt] <= now - start and (deadline is None or now <= deadline):
            ci = route[int(archive[nxt])][0]
            c = caches[ci]
            ln = int(length[nxt])
            if ((ln + 15) & ~15) > c.pool_bytes or blocks_of(nxt, c) > c.max_work:
                status[nxt] = ace.ACE_E_NOMEM  # can never fit this cache
                done += 1
            else:
                queues[ci].append(nxt)
            nxt += 1
        for ci in list(busy):
            c = caches[ci]
            if not c.query():
                continue
            ids, r = busy.pop(ci)
            st = c.status()
            if st == ace.ACE_E_NOMEM:  # the batch's new blocks do not fit the free slots
                c.clear_status()
                if len(ids) == 1:
                    status[ids[0]] = ace.ACE_E_NOMEM
                    done += 1
                else:
                    h = len(ids) // 2
                    queues[ci].extendleft(reversed(ids[h:]))
                    first = ids[:h]
                    r1 = plan(c, first)
                    c.submit(r1)
                    busy[ci] = (first, r1)
                    splits += 1
                    batches += 1
                continue
            if st != ace.ACE_OK:
                raise ace.AceError(st, "seek batch")
            t_done = clock() - start
            for k, rid in enumerate(ids):
                lat[rid] = t_done - int(t_ns[rid])
                status[rid] = ace.ACE_OK
                if keep is not None and rid in keep:
                    kept[rid] = c.result(r, k).cpu().numpy().copy()
            done += len(ids)
            bytes_out += int(r["len"].sum())
        for ci, c in enumerate(caches):
            q = queues[ci]
            if ci in busy or not q:
                continue
            ids, used = [], 0
            while q and len(ids) < c.max_reqs:
                ln = (int(length[q[0]]) + 15) & ~15
                if used + ln > c.pool_bytes:
                    break
                ids.append(q.popleft())
                used += ln
            r = plan(c, ids)
            c.submit(r)
            busy[ci] = (ids, r)
            batches += 1
        if not busy and nxt < n and not any(queues):
            wait = int(t_ns[nxt]) - (clock() - start)
            if wait > 50_000:
                (idle or time.sleep)(wait / 1e9 * 0.5)
    elapsed = (clock() - start) / 1e9
    return {"latency_ns": lat, "status": status, "bytes": bytes_out, "seconds": elapsed, "batches": batches,
            "splits": splits, "served": int((status == ace.ACE_OK).sum()),
            "rejected": int((status == ace.ACE_E_NOMEM).sum()), "kept": kept}


class Server:
    """Continuous batching of seeks under a device working-set budget.

    The archives are split over n_streams caches (archive i to cache i mod
    n_streams); each cache's share of the budget follows the decompressed
    bytes of its archives."""

    def __init__(self, archives, budget_bytes, n_streams=4, max_batch=256, pool_bytes=96 << 20, device="cuda",
                 tune=None):
        self.archives = archives
        self.n_streams = max(1, min(n_streams, len(archives)))
        groups = [[i for i in range(len(archives)) if i % self.n_streams == k] for k in range(self.n_streams)]
        state = sum(ace.ace_archive_state_size(a.idx) for a in archives)
        total = float(sum(a.total for a in archives))
        free = budget_bytes - state - self.n_streams * pool_bytes
        self.caches, self.route = [], {}
        for k, g in enumerate(groups):
            share = int(free * sum(archives[i].total for i in g) / total)
            idxs = [archives[i].idx for i in g]
            lo, hi = 1, max(1, share // archives[g[0]].block_size)
            if ace.ace_cache_size(idxs, lo, max_batch) > share:
                raise ace.AceError(ace.ACE_E_NOMEM, "serving budget below one cache slot per stream")
            while lo < hi:  # the most slots whose cache fits the share
                mid = (lo + hi + 1) // 2
                if ace.ace_cache_size(idxs, mid, max_batch) <= share:
                    lo = mid
                else:
                    hi = mid - 1
            self.caches.append(SeekCache([archives[i] for i in g], lo, max_batch, pool_bytes, device=device,
                                         tune=tune))
            for j, i in enumerate(g):
                self.route[i] = (k, j)
        self.budget = budget_bytes
        self.max_batch = max_batch

    def working_set_bytes(self):
        return sum(c.working_set_bytes() for c in self.caches)

    def run(self, t_ns, archive, coord, length, keep=None, time_limit_s=None):
        """Serves requests arriving at t_ns (ns from the start) in real time;
        see serve_loop.  Adds the blocks the caches evicted meanwhile."""
        before = [c.counters()[0] for c in self.caches]
        res = serve_loop(self.caches, self.route, t_ns, archive, coord, length, keep, time_limit_s)
        res["evicted"] = int(sum(c.counters()[0] - b for c, b in zip(self.caches, before)))
        return res

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
