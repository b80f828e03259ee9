"""Seek batches through the decoded-block cache, and the serving loop: each
request's result is the same alone and in the mix (tolerance 0 bytes),
cache exhaustion is recovered, and overlapping batches on two streams do
not interfere."""
import os

import numpy as np
import pytest

import synth
import __graft_entry__

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_24531_gb300 import ace  # noqa: E402
from paper_2606_24531_gb300.archive import DeviceArchive  # noqa: E402
from paper_2606_24531_gb300.serve import SeekCache, Server, plain_latencies  # noqa: E402

MM = {"fastq": 16, "genome": 20, "text": 4, "mixed": 4}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _archives(size, profiles=("fastq", "genome", "text", "mixed"), seed0=10):
    datas, das = [], []
    for k, p in enumerate(profiles):
        d = synth.generate(p, size, seed0 + k)
        datas.append(d)
        das.append(DeviceArchive(ace.ace_encode(d, 14, MM[p]), max_seek_blocks=4096))
    return datas, das


def test_seek_batch_equals_originals_and_single_seeks():
    datas, das = _archives(3_000_000)
    c = SeekCache(das, n_slots=2048, max_reqs=512, pool_bytes=64 << 20)
    rng = np.random.default_rng(0)
    reqs = []
    for _ in range(300):
        a = int(rng.integers(0, len(das)))
        n = int(rng.integers(1, 300_000))
        co = int(rng.integers(0, len(datas[a]) - n))
        reqs.append((a, co, n))
    reqs += [(0, 0, 1), (1, len(datas[1]) - 1, 1), (2, 16384 * 5, 16384)]
    outs = c.seek_many(reqs)
    for (a, co, n), o in zip(reqs, outs):
        assert np.array_equal(o.cpu().numpy(), datas[a][co:co + n])
    # the same requests again: now mostly from the cache
    used_before = ace.ace_cache_usage(c.cache)[0]
    outs = c.seek_many(reqs[:50])
    for (a, co, n), o in zip(reqs[:50], outs):
        assert np.array_equal(o.cpu().numpy(), datas[a][co:co + n])
    assert ace.ace_cache_usage(c.cache)[0] == used_before
    # alone (plain ace_seek) equals in the mix
    for a, co, n in reqs[:20]:
        s = das[a].seek(co, n)
        assert das[a].sync() == ace.ACE_OK
        assert np.array_equal(s.cpu().numpy(), datas[a][co:co + n])
    c.close()


def test_cache_exhaustion_reports_nomem_and_stays_valid():
    """A batch whose new blocks exceed the slots is refused with ACE_E_NOMEM
    and copies nothing; the cache stays valid without a reset, and
    run_batch serves a refused batch in halves."""
    datas, das = _archives(2_000_000, profiles=("mixed", "text"))
    c = SeekCache(das, n_slots=40, max_reqs=64, pool_bytes=8 << 20)
    r = c.plan([(0, 0, 30 * 16384), (1, 0, 30 * 16384)])  # 60 target blocks > 40 slots
    c.submit(r)
    assert c.sync() == ace.ACE_E_NOMEM
    outs = c.seek_many([(0, 16384 * 3, 20000), (1, 5, 16384 * 10)])
    assert np.array_equal(outs[0].cpu().numpy(), datas[0][16384 * 3:16384 * 3 + 20000])
    assert np.array_equal(outs[1].cpu().numpy(), datas[1][5:5 + 16384 * 10])
    reqs = [(0, 16384 * 20, 16384 * 16), (1, 16384 * 40, 16384 * 16), (0, 16384 * 40, 16384 * 16)]
    r = c.plan(reqs)
    c.submit(r)  # 48 new blocks in one batch: more than the 40 slots
    assert c.sync() == ace.ACE_E_NOMEM
    c.run_batch(r)  # refused whole, served in halves (16 blocks, then 32)
    for q, (a, co, n) in zip(r, reqs):
        o = int(q["out_off"])
        assert np.array_equal(c.pool[o:o + n].cpu().numpy(), datas[a][co:co + n])
    c.close()


def test_cache_evicts_least_recently_used_blocks():
    """Many batches over more distinct blocks than the cache holds: blocks
    are evicted by the clock (no reset), every result stays exact, and the
    slots a batch reads from are never taken by its own new blocks."""
    datas, das = _archives(3_000_000, profiles=("fastq", "text", "genome"))
    c = SeekCache(das, n_slots=400, max_reqs=64, pool_bytes=16 << 20)
    rng = np.random.default_rng(1)
    for it in range(60):
        reqs = []
        for _ in range(int(rng.integers(1, 12))):
            a = int(rng.integers(0, len(das)))
            n = int(rng.integers(1, 120_000))
            co = int(rng.integers(0, len(datas[a]) - n))
            reqs.append((a, co, n))
        outs = c.seek_many(reqs)
        for (a, co, n), o in zip(reqs, outs):
            assert np.array_equal(o.cpu().numpy(), datas[a][co:co + n]), (it, a, co, n)
    evicted, decoded = c.counters()
    used, n_slots = ace.ace_cache_usage(c.cache)
    assert evicted > 0 and decoded > n_slots
    assert used == n_slots == 400
    c.close()


def test_server_results_same_alone_and_in_the_mix():
    """Poisson arrivals, continuous batching on two streams; sampled
    requests' bytes equal the original and a lone ace_seek."""
    datas, das = _archives(4_000_000)
    sizes = np.array([len(d) for d in datas], np.uint64)
    t, a, co, ln = synth.requests(5, 3000, 2e5, sizes, 1 << 14, 1 << 18)
    srv = Server(das, budget_bytes=1 << 30, n_streams=2, max_batch=128, pool_bytes=48 << 20)
    assert srv.working_set_bytes() <= 1 << 30
    keep = set(range(0, 3000, 97))
    res = srv.run(t, a, co, ln, keep=keep)
    assert res["served"] == 3000
    assert (res["latency_ns"] > 0).all()
    for rid in keep:
        i = int(a[rid])
        want = datas[i][int(co[rid]): int(co[rid]) + int(ln[rid])]
        assert np.array_equal(res["kept"][rid], want)
        alone = das[i].seek(int(co[rid]), int(ln[rid]))
        assert das[i].sync() == ace.ACE_OK
        assert np.array_equal(alone.cpu().numpy(), res["kept"][rid])
    srv.close()
    scr = [x.d_scratch for x in das]
    lat = plain_latencies(das, scr, a, co, ln, limit=200)
    assert (lat > 0).all()
