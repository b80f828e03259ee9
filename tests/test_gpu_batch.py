"""Batched decode: thousands of uneven independent archives (mixed profiles
and block sizes) in one persistent launch, replayed through a CUDA graph,
equal to their originals and to one launch per object, bit for bit."""
import os

import numpy as np
import pytest

import __graft_entry__

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_24531_gb300 import ace  # noqa: E402
from paper_2606_24531_gb300.batch import DeviceBatch, autotune, make_objects, time_per_object  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _check_all(db, datas):
    big = torch.cat([torch.from_numpy(d) for d in datas]).cuda() if datas else None
    o = 0
    for i, d in enumerate(datas):
        assert torch.equal(db.output(i), big[o:o + d.size]), i
        o += d.size


def test_batch_equals_originals_and_graph_replay():
    datas, arcs = make_objects(300, seed=4, max_size=1 << 20)
    db = DeviceBatch(arcs)
    db.decode()
    assert db.sync() == ace.ACE_OK
    _check_all(db, datas)
    db.out.zero_()
    g = db.capture()
    for _ in range(2):  # each replay decodes everything again
        db.out.zero_()
        g.replay()
        assert db.sync() == ace.ACE_OK
        _check_all(db, datas)
    # one launch per object gives the same bytes
    views = [db.output(i) for i in range(len(datas))]
    db.out.zero_()
    time_per_object(db.items, views)
    _check_all(db, datas)
    db.close()


def test_batch_tunings_agree_and_autotune():
    datas, arcs = make_objects(120, seed=7, max_size=1 << 19)
    db = DeviceBatch(arcs)
    best = autotune(db, candidates=[(1, 64), (2, 128), (4, 128), (8, 256)], reps=1, cache_key=None)
    assert best["warps_per_cta"] in (1, 2, 4, 8)
    for w, c in [(1, 64), (8, 256)]:
        db.retune(ace.make_tune(w, 0, c))
        db.out.zero_()
        db.decode()
        assert db.sync() == ace.ACE_OK
        _check_all(db, datas)
    db.close()


def test_uneven_batch_4096_objects():
    """4,096 objects, log-uniform sizes, random profile and block size each;
    sizes capped at 2 MiB here (ACE_FULL_CONFIGS=1 takes the 64 MiB cap of
    the full workload, about 28 GB)."""
    cap = 1 << 26 if os.environ.get("ACE_FULL_CONFIGS") == "1" else 1 << 21
    datas, arcs = make_objects(4096, seed=4, max_size=cap)
    db = DeviceBatch(arcs)
    g = db.capture()
    g.replay()
    assert db.sync() == ace.ACE_OK
    _check_all(db, datas)
    db.close()


def test_batch_mixes_offset_widths():
    """Archives with 4- and 5-byte offsets side by side in one launch."""
    import synth
    datas = [synth.generate(p, n, s) for p, n, s in
             [("mixed", 300_000, 1), ("fastq", 200_000, 2), ("text", 150_001, 3), ("genome", 90_000, 4)]]
    arcs = [ace.ace_encode(d, 12, 4, off_width=5 if i % 2 else 0) for i, d in enumerate(datas)]
    db = DeviceBatch(arcs)
    db.decode()
    assert db.sync() == ace.ACE_OK
    _check_all(db, datas)
    db.close()


def test_batch_with_deep_chain_oracle_archives():
    """The batch decoder's match phase waits on ready flags.  Archives written
    by the oracle (most-recent-first sources: hundreds of dependency levels
    at small blocks) mixed with library archives in one batch: every output
    bit-exact, in a plain decode and in graph replays, with both schedules."""
    import oracle
    import synth
    datas, arcs = [], []
    for k, (p, n, log2b) in enumerate([("text", 300_000, 8), ("mixed", 250_000, 10), ("fastq", 200_000, 8),
                                       ("genome", 180_000, 9), ("text", 120_000, 12), ("mixed", 90_000, 8)]):
        d = synth.generate(p, n, 40 + k)
        datas.append(d)
        arcs.append(oracle.encode(d, log2b, 4, 16))
        d2 = synth.generate(p, n // 2 + 777, 60 + k)
        datas.append(d2)
        arcs.append(ace.ace_encode(d2, 12, 4))
    assert max(oracle.levels(a).max() for a in arcs[::2]) > 32
    for schedule in (ace.ACE_SCHEDULE_FUSED, ace.ACE_SCHEDULE_PASSES):
        db = DeviceBatch(arcs, tune=ace.make_tune(schedule=schedule))
        db.decode()
        assert db.sync() == ace.ACE_OK
        _check_all(db, datas)
        g = db.capture()
        for _ in range(2):
            db.out.zero_()
            g.replay()
            assert db.sync() == ace.ACE_OK
            _check_all(db, datas)
        del g
        db.close()
