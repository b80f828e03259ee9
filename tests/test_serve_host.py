"""Host-side planning of seek batches (no GPU): results packed 16-byte
aligned in the output pool in request order, and batches that do not fit
the pool or the request table refused."""
import types

import numpy as np

from paper_2606_24531_gb300 import ace
from paper_2606_24531_gb300.serve import SeekCache


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
