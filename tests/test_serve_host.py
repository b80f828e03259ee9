"""Host-side planning of seek batches (no GPU): results packed 16-byte
aligned in the output pool in request order, and batches that do not fit
the pool or the request table refused."""
import types

import numpy as np

from paper_2606_24531_gb300 import ace
from paper_2606_24531_gb300.serve import SeekCache, serve_loop


def _cache(pool_bytes, max_reqs):
    c = types.SimpleNamespace(pool_bytes=pool_bytes, max_reqs=max_reqs)
    c.plan_arrays = lambda a, co, n: SeekCache.plan_arrays(c, a, co, n)
    return c


def test_results_packed_16_byte_aligned_in_order():
    c = _cache(1 << 20, 256)
    reqs = [(0, 5, 1), (1, 100, 16), (0, 0, 17), (2, 7, 300)]
    r = SeekCache.plan(c, reqs)
    assert r.dtype == ace.SEEK_REQ
    assert list(r["archive"]) == [0, 1, 0, 2]
    assert list(r["coord"]) == [5, 100, 0, 7]
    assert list(r["len"]) == [1, 16, 17, 300]
    assert list(r["out_off"]) == [0, 16, 32, 64]
    assert all(int(o) % 16 == 0 for o in r["out_off"])
    # arrays give the same plan
    a, co, n = (np.array(x, np.uint64) for x in zip(*reqs))
    assert np.array_equal(SeekCache.plan_arrays(c, a, co, n), r)


def test_batches_that_do_not_fit_are_refused():
    assert SeekCache.plan(_cache(64, 256), [(0, 0, 48), (0, 0, 16)]) is not None  # exactly full
    assert SeekCache.plan(_cache(64, 256), [(0, 0, 48), (0, 0, 17)]) is None  # 48 + 32 > 64
    assert SeekCache.plan(_cache(1 << 20, 2), [(0, 0, 1)] * 3) is None
    assert SeekCache.plan(_cache(1 << 20, 2), []).size == 0


class FakeCache:
    """A stand-in for SeekCache on the host: a batch is refused (ACE_E_NOMEM)
    when the blocks its requests cover exceed slot_limit, as the device cache
    refuses a batch whose new blocks exceed its free slots."""

    def __init__(self, pool_bytes=1 << 20, max_reqs=8, max_work=64, block_size=4096, slot_limit=16):
        self.pool_bytes, self.max_reqs, self.max_work, self.block_size = pool_bytes, max_reqs, max_work, block_size
        self.slot_limit = slot_limit
        self.submitted = []
        self.st = ace.ACE_OK

    def plan_arrays(self, a, co, n):
        return SeekCache.plan_arrays(self, a, co, n)

    def submit(self, r):
        assert len(r) > 0, "an empty batch was submitted"
        self.submitted.append(len(r))
        blocks = set()
        for q in r:
            for b in range(int(q["coord"]) // self.block_size, (int(q["coord"]) + int(q["len"]) - 1) // self.block_size + 1):
                blocks.add((int(q["archive"]), b))
        self.st = ace.ACE_E_NOMEM if len(blocks) > self.slot_limit else ace.ACE_OK

    def query(self):
        return True

    def status(self):
        return self.st

    def clear_status(self):
        st, self.st = self.st, ace.ACE_OK
        return st

    def result(self, r, k):
        import torch
        return torch.zeros(int(r[k]["len"]), dtype=torch.uint8)


class Clock:
    def __init__(self):
        self.t = 0

    def __call__(self):
        self.t += 1000
        return self.t


def _loop(caches, route, reqs, **kw):
    t = np.zeros(len(reqs), np.uint64)
    a, c, n = (np.array(x, np.uint64) for x in zip(*reqs))
    return serve_loop(caches, route, t, a.astype(np.uint32), c, n, clock=Clock(), idle=lambda s: None, **kw)


def test_oversize_requests_are_rejected_not_left_queued():
    """A request longer than the output pool, or covering more blocks than a
    batch may decode, can never be served: it is rejected at admission and
    the loop ends (it used to stay queued forever while empty batches went
    out)."""
    c = FakeCache(pool_bytes=64 << 10, max_work=8)
    res = _loop([c], {0: (0, 0)}, [(0, 0, 100), (0, 0, 200 << 10), (0, 0, 40 << 10), (0, 4096, 50)])
    assert list(res["status"]) == [ace.ACE_OK, ace.ACE_E_NOMEM, ace.ACE_E_NOMEM, ace.ACE_OK]
    assert res["served"] == 2 and res["rejected"] == 2
    assert all(k > 0 for k in c.submitted)


def test_refused_batches_are_split_and_single_refusals_rejected():
    """A batch refused for want of slots is served in halves; a request
    refused on its own is rejected; every other request is served."""
    c = FakeCache(max_reqs=8, slot_limit=4, max_work=64)
    reqs = [(0, 4096 * k, 10) for k in range(8)]  # 8 blocks: refused, split into 4 + 4
    reqs.append((0, 0, 5 * 4096))  # 5 blocks alone: more than 4 slots
    res = _loop([c], {0: (0, 0)}, reqs)
    assert res["served"] == 8 and res["rejected"] == 1
    assert res["status"][8] == ace.ACE_E_NOMEM
    assert res["splits"] >= 1
    assert all(k > 0 for k in c.submitted)


def test_archives_routed_to_their_caches():
    """Each request goes to the cache holding its archive, with the
    archive's place in that cache."""
    c0, c1 = FakeCache(), FakeCache()
    route = {0: (0, 0), 1: (1, 0), 2: (0, 1)}
    res = _loop([c0, c1], route, [(0, 0, 10), (1, 0, 10), (2, 0, 10), (1, 4096, 10)])
    assert res["served"] == 4
    assert sum(c0.submitted) == 2 and sum(c1.submitted) == 2
