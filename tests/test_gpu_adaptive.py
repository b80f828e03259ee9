"""Stored streams (directory mode 1: entropy coding chosen per stream at
encode time, Section 6.1) through the GPU path: archives written adaptively
by the oracle and by the library's encoder decode bit-exact (tolerance 0
bytes) in whole decodes under both schedules, seeks, batches and seek
batches; a stored stream whose byte count differs from its symbol count,
or a third mode, is rejected when the index is built."""
import numpy as np
import pytest

import oracle
import synth
import __graft_entry__

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_24531_gb300 import ace  # noqa: E402
from paper_2606_24531_gb300.archive import DeviceArchive, stream_report  # noqa: E402

MM = {"mixed": 4, "text": 4, "fastq": 16, "genome": 20}
SCHEDULES = (ace.ACE_SCHEDULE_PASSES, ace.ACE_SCHEDULE_FUSED)


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _decode(arc, schedule):
    da = DeviceArchive(arc)
    out = da.decode_all(tune=ace.make_tune(schedule=schedule))
    st = da.sync()
    res = out.cpu().numpy()[: da.total]
    da.close()
    return st, res


def _modes(arc):
    hdr = arc[:64].view(np.uint64)
    nb, dir_off = int(hdr[3]), int(hdr[4])
    return arc[dir_off:dir_off + 64 * nb].reshape(nb, 64)[:, 56:59]


@pytest.mark.parametrize("profile", ["genome", "fastq", "mixed", "text"])
@pytest.mark.parametrize("log2b", [8, 10, 14])
def test_oracle_adaptive_archives(profile, log2b):
    data = synth.generate(profile, 400_000, 50 + log2b)
    arc = oracle.encode(data, log2b, 4, 16, adaptive=True)
    ref = oracle.decode(arc)
    assert np.array_equal(ref, data)
    for schedule in SCHEDULES:
        st, out = _decode(arc, schedule)
        assert st == ace.ACE_OK, ace.ace_status_str(st)
        assert np.array_equal(out, ref)


@pytest.mark.parametrize("profile", ["genome", "fastq", "mixed", "text"])
def test_library_adaptive_archives_decode_and_seek(profile):
    data = synth.generate(profile, 3_000_000 + 999, 60)
    arc = ace.ace_encode(data, 14, MM[profile], adaptive=True)
    if profile in ("genome", "fastq"):
        assert (_modes(arc) == 1).any()
    for schedule in SCHEDULES:
        st, out = _decode(arc, schedule)
        assert st == ace.ACE_OK, ace.ace_status_str(st)
        assert np.array_equal(out, data)
    da = DeviceArchive(arc, max_seek_blocks=512)
    rng = np.random.default_rng(4)
    n = data.size
    for coord, length in [(0, 1), (n - 1, 1), (n // 2, 70_000)] + [
            (int(c), int(rng.integers(1, 200_000))) for c in rng.integers(0, n - 200_000, 8)]:
        s = da.seek(coord, length)
        assert da.sync() == ace.ACE_OK
        assert np.array_equal(s.cpu().numpy(), data[coord:coord + length]), (coord, length)
    da.close()


def test_adaptive_archives_in_batches_and_seek_batches():
    from paper_2606_24531_gb300.batch import DeviceBatch
    from paper_2606_24531_gb300.serve import SeekCache

    datas, arcs = [], []
    for k, p in enumerate(["genome", "fastq", "text", "mixed", "genome", "fastq"]):
        d = synth.generate(p, 700_000 + 1111 * k, 70 + k)
        datas.append(d)
        arcs.append(ace.ace_encode(d, 12 if k % 2 else 14, MM[p], adaptive=k % 3 != 2))
    arcs[4] = oracle.encode(datas[4], 12, 4, 16, adaptive=True)  # deep chains with stored streams
    for schedule in SCHEDULES:
        db = DeviceBatch(arcs, tune=ace.make_tune(schedule=schedule))
        db.decode()
        assert db.sync() == ace.ACE_OK
        for i, d in enumerate(datas):
            assert np.array_equal(db.output(i).cpu().numpy(), d), (schedule, i)
        db.close()
    same_b = [0, 2]  # 16 KiB blocks both: one block size per cache
    das = [DeviceArchive(arcs[i], max_seek_blocks=256) for i in same_b]
    c = SeekCache(das, n_slots=1024, max_reqs=64, pool_bytes=16 << 20)
    rng = np.random.default_rng(5)
    reqs = []
    for _ in range(40):
        j = int(rng.integers(0, len(das)))
        n = int(rng.integers(1, 100_000))
        reqs.append((j, int(rng.integers(0, datas[same_b[j]].size - n)), n))
    outs = c.seek_many(reqs)
    for (j, co, n), o in zip(reqs, outs):
        assert np.array_equal(o.cpu().numpy(), datas[same_b[j]][co:co + n])
    c.close()


def test_stored_stream_checks_at_index_build():
    data = synth.generate("genome", 300_000, 8)
    arc = ace.ace_encode(data, 10, 20, adaptive=True)
    m = _modes(arc)
    b, k = map(int, np.argwhere(m == 1)[0])
    dir_off = int(arc[32:40].view(np.uint64)[0])
    e = dir_off + 64 * b
    nsym = int(arc[e + 36 + 4 * k:e + 40 + 4 * k].view(np.uint32)[0])
    bad = arc.copy()
    bad[e + 24 + 4 * k:e + 28 + 4 * k] = np.array([nsym + 1], np.uint32).view(np.uint8)
    with pytest.raises(ace.AceError) as err:
        DeviceArchive(bad)
    assert err.value.status == ace.ACE_E_CORRUPT
    bad = arc.copy()
    bad[e + 56 + k] = 2
    with pytest.raises(ace.AceError) as err:
        DeviceArchive(bad)
    assert err.value.status == ace.ACE_E_CORRUPT


def test_adaptive_genome_is_smaller_and_decodes():
    """The per-stream choice on repetitive genomic data (Table 2's finding):
    the structural streams are stored, the archive shrinks, the decode is
    exact."""
    data = synth.generate("genome", 32 << 20, 3)
    a0 = ace.ace_encode(data, 14, 20)
    a1 = ace.ace_encode(data, 14, 20, adaptive=True)
    rep = stream_report(a1)
    assert rep["lengths"]["stored_verbatim_blocks"] > 0
    assert a1.size < a0.size
    st, out = _decode(a1, ace.ACE_SCHEDULE_PASSES)
    assert st == ace.ACE_OK and np.array_equal(out, data)


def test_source_not_before_its_destination_is_reported():
    """A match whose absolute source lies at or after its own destination
    breaks the rule of the sequential copy (Section 2).  Patched into a
    stored offset stream, where no rANS end-of-stream check can catch it,
    it must come back as ACE_E_CORRUPT from whole decodes under both
    schedules and from a seek of its block, as the oracle rejects it too."""
    data = synth.generate("genome", 2_000_000, 9)
    arc = ace.ace_encode(data, 14, 20, adaptive=True)
    hdr = arc[:64].view(np.uint64)
    total, nb, dir_off, payload_off = (int(hdr[i]) for i in (2, 3, 4, 6))
    w = int(arc[9])  # off_width
    d = arc[dir_off:dir_off + 64 * nb].reshape(nb, 64)
    stored_off = [b for b in range(1, nb - 1)
                  if d[b, 58] == 1 and int(d[b, 44:48].copy().view(np.uint32)[0]) >= w]
    assert stored_off, "no block with a stored offset stream"
    b = stored_off[len(stored_off) // 2]
    off = payload_off + int(d[b, 16:24].copy().view(np.uint64)[0])  # the block's first match source
    bad = arc.copy()
    bad[off:off + w] = np.frombuffer(np.uint64(total - 1).tobytes()[:w], np.uint8)  # the data's last byte
    with pytest.raises(oracle.OracleError):
        oracle.decode(bad)
    for schedule in SCHEDULES:
        st, _ = _decode(bad, schedule)
        assert st == ace.ACE_E_CORRUPT, ace.ace_status_str(st)
    da = DeviceArchive(bad, max_seek_blocks=1024)
    B = 1 << 14
    da.seek(b * B, B)
    assert da.sync() == ace.ACE_E_CORRUPT
    da.close()
