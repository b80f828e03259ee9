"""GPU parity: the sm_103a decoder, called through the C ABI, against the
oracle and the original bytes.  Decoded output has exactly one correct
value, so every comparison is bit-exact (tolerance 0 bytes)."""
import time

import numpy as np
import pytest

import oracle
import synth
import __graft_entry__
from conftest import with_dep_removed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_24531_gb300 import ace  # noqa: E402
from paper_2606_24531_gb300.archive import DeviceArchive  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def gpu_decode(arc, tune=None):
    da = DeviceArchive(arc)
    out = da.decode_all(tune=tune)
    st = da.sync()
    res = out.cpu().numpy()[: da.total]
    da.close()
    return st, res


MIN_MATCH = {"mixed": 4, "text": 4, "fastq": 16, "genome": 20}


SCHEDULES = {"fused": ace.ACE_SCHEDULE_FUSED, "passes": ace.ACE_SCHEDULE_PASSES}


@pytest.mark.parametrize("schedule", sorted(SCHEDULES))
@pytest.mark.parametrize("profile", ["mixed", "fastq", "genome", "text"])
@pytest.mark.parametrize("log2b", [8, 12, 14, 16])
def test_decode_all_library_archives(profile, log2b, schedule):
    """Both decode schedules (one fused launch; three passes with the match
    pass by level) give the original bytes."""
    data = synth.generate(profile, 3_000_000 + 12345, 100 + log2b)
    arc = ace.ace_encode(data, log2b, MIN_MATCH[profile])
    st, out = gpu_decode(arc, ace.make_tune(schedule=SCHEDULES[schedule]))
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert np.array_equal(out, data)


@pytest.mark.parametrize("profile", ["text", "fastq"])
def test_decode_all_32k_blocks(profile):
    """32 KiB blocks: the largest that levels of few blocks resolve a block
    per CTA (15-bit positions, shared memory above the default limit)."""
    data = synth.generate(profile, 3_000_000 + 999, 77)
    arc = ace.ace_encode(data, 15, MIN_MATCH[profile])
    st, out = gpu_decode(arc)
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert np.array_equal(out, data)


@pytest.mark.parametrize("schedule", sorted(SCHEDULES))
@pytest.mark.parametrize("profile", ["mixed", "fastq", "genome", "text"])
@pytest.mark.parametrize("log2b", [8, 14])
def test_decode_all_oracle_archives(profile, log2b, schedule):
    """Archives written by the oracle (most-recent-first sources, deep
    dependency chains) decode to the oracle's own output."""
    data = synth.generate(profile, 400_000, 7)
    arc = oracle.encode(data, log2b, 4, 16)
    ref = oracle.decode(arc)
    assert np.array_equal(ref, data)
    st, out = gpu_decode(arc, ace.make_tune(schedule=SCHEDULES[schedule]))
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("schedule", sorted(SCHEDULES))
def test_seeks_under_both_schedules(schedule):
    """Seeks through the fused launch and through the three passes, on a
    library archive and on a deep-chain oracle archive, equal the original."""
    for arc_of, n in ((lambda d: ace.ace_encode(d, 12, 4), 2_000_000), (lambda d: oracle.encode(d, 10, 4, 16), 300_000)):
        data = synth.generate("text", n, 33)
        arc = arc_of(data)
        da = DeviceArchive(arc, max_seek_blocks=n // 1024 + 8)
        ace.ace_index_set_tune(da.idx, ace.make_tune(schedule=SCHEDULES[schedule]))
        rng = np.random.default_rng(8)
        cases = [(0, 1), (n - 1, 1), (n // 2, 5000)] + [(int(c), int(rng.integers(1, 60_000)))
                                                        for c in rng.integers(0, n - 60_000, 10)]
        for coord, length in cases:
            out = da.seek(coord, length)
            st = da.sync()
            assert st == ace.ACE_OK, (coord, length, ace.ace_status_str(st))
            assert np.array_equal(out.cpu().numpy(), data[coord:coord + length]), (coord, length)
        da.close()


def test_plain_small_config_decode_seek_and_three_phase():
    """1 MiB mixed data (seed 0), 16 KiB blocks, min match 4: full decode,
    seek of block 37, and the three-phase check (Section 5)."""
    data = synth.generate("mixed", 1 << 20, 0)
    B = 1 << 14
    for arc in (ace.ace_encode(data, 14, 4), oracle.encode(data, 14, 4, 64)):
        da = DeviceArchive(arc, max_seek_blocks=64)
        out = da.decode_all()
        assert da.sync() == ace.ACE_OK
        assert np.array_equal(out.cpu().numpy(), data)
        s = da.seek(37 * B, B)
        assert da.sync() == ace.ACE_OK
        assert np.array_equal(s.cpu().numpy(), oracle.seek(arc, 37 * B, B))
        want = oracle.fnv1a64(data[37 * B: 38 * B])
        rep, buf = da.verify(37 * B, B, want)
        assert rep["phase1_ok"] == 1 and rep["phase2_ok"] == 1 and rep["phase3_ok"] == 1, rep
        assert rep["fnv_after"] == want and rep["fnv_before"] != want
        assert np.array_equal(buf[B:2 * B].cpu().numpy(), data[37 * B: 38 * B])
        da.close()


def test_edge_sizes_and_empty():
    rng = np.random.default_rng(5)
    B = 256
    for n in [1, 2, 7, B - 1, B, B + 1, 3 * B + 7, 200 * B + 3]:
        for alpha in (1, 2, 256):
            data = rng.integers(0, alpha, n).astype(np.uint8)
            for arc in (ace.ace_encode(data, 8, 4), oracle.encode(data, 8, 4, 16)):
                st, out = gpu_decode(arc)
                assert st == ace.ACE_OK
                assert np.array_equal(out, data), (n, alpha)
    arc = ace.ace_encode(np.zeros(0, np.uint8), 12, 4)
    da = DeviceArchive(arc)
    assert da.total == 0
    da.decode_all()
    assert da.sync() == ace.ACE_OK
    da.close()


def test_separate_passes_equal_decode_all():
    """ace_decode_pass(TOKENS), (LITERALS), then (MATCH) on one stream is
    ace_decode_all; a pass number outside the three is rejected."""
    data = synth.generate("text", 1_500_000, 21)
    arc = ace.ace_encode(data, 14, 4)
    da = DeviceArchive(arc)
    out = torch.zeros(da.total, dtype=torch.uint8, device="cuda")
    for p in (ace.ACE_PASS_TOKENS, ace.ACE_PASS_LITERALS, ace.ACE_PASS_MATCH):
        ace.ace_decode_pass(da.idx, p, out, da.total, da.d_scratch, da.scratch_bytes, None, da.stream)
    assert da.sync() == ace.ACE_OK
    assert np.array_equal(out.cpu().numpy(), data)
    with pytest.raises(ace.AceError) as e:
        ace.ace_decode_pass(da.idx, 3, out, da.total, da.d_scratch, da.scratch_bytes, None, da.stream)
    assert e.value.status == ace.ACE_E_INVAL
    da.close()


def test_tunings_agree():
    data = synth.generate("text", 2_000_000, 9)
    arc = ace.ace_encode(data, 14, 4)
    ran = 0
    for warps in (1, 2, 4, 8, 16):
        for chunk in (32, 64, 128, 256):
            try:
                st, out = gpu_decode(arc, ace.make_tune(warps, 0, chunk))
            except ace.AceError as e:
                # more than 8 warps per CTA is outside the kernel's launch bounds
                assert e.status == ace.ACE_E_INVAL and warps > 8, (warps, chunk)
                continue
            ran += 1
            assert st == ace.ACE_OK
            assert np.array_equal(out, data), (warps, chunk)
    assert ran == 16


def test_overlap_rule():
    """Matches whose source overlaps the destination (distance d < length)
    reproduce the sequential bytewise copy, for d = 1..64."""
    rng = np.random.default_rng(2)
    parts = []
    for d in range(1, 65):
        for ln in (4, 5, 17, 31, 32, 33, 63, 64, 65, 100, 200, 300):
            parts.append(rng.integers(0, 256, 24).astype(np.uint8))  # separator
            unit = rng.integers(0, 256, d).astype(np.uint8)
            parts.append(np.resize(unit, d + ln))
    data = np.concatenate(parts)
    for arc in (ace.ace_encode(data, 12, 4), oracle.encode(data, 12, 4, 16)):
        dists = set()
        for b in range(oracle.info(arc)["n_blocks"]):
            lr, ml, src = oracle.block_tokens(arc, b)
            dst = b * 4096
            for t in range(len(lr)):
                dst += int(lr[t])
                if ml[t] and dst - int(src[t]) < ml[t]:
                    dists.add(dst - int(src[t]))
                dst += int(ml[t])
        assert set(range(1, 65)) <= dists  # every distance 1..64 occurs overlapped
        st, out = gpu_decode(arc)
        assert st == ace.ACE_OK
        assert np.array_equal(out, data)


def test_seek_random_ranges():
    data = synth.generate("mixed", 3_000_000, 11)
    arc = ace.ace_encode(data, 12, 4)
    da = DeviceArchive(arc, max_seek_blocks=1024)
    rng = np.random.default_rng(3)
    n = data.size
    cases = [(0, 1), (n - 1, 1), (0, n), (4096 * 37, 4096), (4095, 2), (n - 5000, 5000)]
    cases += [(int(c), int(rng.integers(1, 300_000))) for c in rng.integers(0, n - 300_000, 40)]
    for coord, length in cases:
        out = da.seek(coord, length)
        st = da.sync()
        assert st == ace.ACE_OK, (coord, length, ace.ace_status_str(st))
        assert np.array_equal(out.cpu().numpy(), data[coord:coord + length]), (coord, length)
    # the seek writes exactly len bytes of the caller's buffer
    buf = torch.full((10000,), 7, dtype=torch.uint8, device="cuda")
    ace.ace_seek(da.idx, 5000, 3000, buf[1000:].data_ptr(), 3000, da.d_scratch, da.scratch_bytes)
    assert da.sync() == ace.ACE_OK
    h = buf.cpu().numpy()
    assert (h[:1000] == 7).all() and (h[4000:] == 7).all()
    assert np.array_equal(h[1000:4000], data[5000:8000])
    for coord, length in [(n, 1), (0, 0), (1, n)]:
        with pytest.raises(ace.AceError) as e:
            da.seek(coord, max(length, 1) if length else 0, out=torch.empty(8, dtype=torch.uint8, device="cuda"))
        assert e.value.status in (ace.ACE_E_RANGE, ace.ACE_E_NOMEM)
    da.close()


@pytest.mark.parametrize("log2b", [8, 12])
def test_five_byte_offsets_decode_and_seek(log2b):
    """5-byte absolute offsets (the width above 2^32 bytes), forced on a small
    input: whole decode, separate passes, batched and plain seeks."""
    data = synth.generate("mixed", 2_000_000 + 77, 40 + log2b)
    arc = ace.ace_encode(data, log2b, 4, off_width=5)
    assert oracle.info(arc)["off_width"] == 5
    st, out = gpu_decode(arc)
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert np.array_equal(out, data)
    da = DeviceArchive(arc, max_seek_blocks=4096)
    rng = np.random.default_rng(log2b)
    n = data.size
    cases = [(0, 1), (n - 1, 1), (n - 3000, 3000)]
    cases += [(int(c), int(rng.integers(1, 200_000))) for c in rng.integers(0, n - 200_000, 12)]
    for coord, length in cases:
        s = da.seek(coord, length)
        st = da.sync()
        assert st == ace.ACE_OK, (coord, length, ace.ace_status_str(st))
        assert np.array_equal(s.cpu().numpy(), data[coord:coord + length]), (coord, length)
    da.close()


def test_seek_closure_larger_than_scratch_reports_nomem():
    data = synth.generate("genome", 2_000_000, 4)
    arc = oracle.encode(data, 12, 4, 16)  # deep chains: long closures
    cl = oracle.closure(arc, 400, 400)
    assert len(cl) > 4
    da = DeviceArchive(arc, max_seek_blocks=2)
    da.seek(400 * 4096, 10)
    assert da.sync() == ace.ACE_E_NOMEM
    # the scratch stays usable afterwards
    da2 = DeviceArchive(arc, max_seek_blocks=len(cl))
    out = da2.seek(400 * 4096, 10)
    assert da2.sync() == ace.ACE_OK
    assert np.array_equal(out.cpu().numpy(), data[400 * 4096: 400 * 4096 + 10])
    da.close()
    da2.close()


def test_seek_outside_its_closure_is_reported_at_once():
    """A seek whose closure misses a source block (its dependency list was
    emptied on the host) finds the block's flag unmarked by the closure and
    reports the archive corrupt without waiting; the context stays usable."""
    data = synth.generate("text", 200_000, 12)
    arc = oracle.encode(data, 12, 4, 16)
    b = 30
    deps = oracle.deps(arc)[b]
    assert deps and deps != [(0, 0)]
    bad = with_dep_removed(arc, b)
    da = DeviceArchive(bad, max_seek_blocks=64)
    ace.ace_index_set_tune(da.idx, ace.make_tune(wait_timeout_ns=2_000_000_000))
    t0 = time.perf_counter()
    da.seek(b * 4096, 100)
    assert da.sync() == ace.ACE_E_CORRUPT
    assert time.perf_counter() - t0 < 1.0  # no wait ran out
    # a clean seek on the same scratch still works
    out = da.seek(0, 4096)
    assert da.sync() == ace.ACE_OK
    assert np.array_equal(out.cpu().numpy(), data[:4096])
    da.close()


def test_wait_gives_up_with_timeout_status():
    """A seek batch through the block cache whose closure misses a source
    block waits on a flag nothing sets; the bounded wait ends with
    ACE_E_TIMEOUT and the cache stays usable after a reset."""
    from paper_2606_24531_gb300.serve import SeekCache

    data = synth.generate("text", 200_000, 12)
    arc = oracle.encode(data, 12, 4, 16)
    b = 30
    bad = with_dep_removed(arc, b)
    da = DeviceArchive(bad, max_seek_blocks=64)
    c = SeekCache([da], n_slots=64, max_reqs=4, pool_bytes=1 << 16,
                  tune=ace.make_tune(wait_timeout_ns=2_000_000))
    c.submit(c.plan([(0, b * 4096, 100)]))
    assert c.sync() == ace.ACE_E_TIMEOUT
    c.reset()
    out = c.seek_many([(0, 0, 4096)])
    assert np.array_equal(out[0].cpu().numpy(), data[:4096])
    c.close()
    da.close()


def test_library_archive_seek_with_a_dependency_removed():
    """A library archive (few dependency levels) whose block lost its
    dependency list: the seek's closure misses the blocks its matches read,
    which is reported as corrupt rather than read from other blocks' slots;
    a clean seek still works."""
    data = synth.generate("fastq", 3_000_000, 31)
    arc = ace.ace_encode(data, 14, 16)
    deps = oracle.deps(arc)
    b = next(k for k in range(len(deps)) if deps[k] and deps[k] != [(0, 0)] and k > 70)
    bad = with_dep_removed(arc, b)
    da = DeviceArchive(bad, max_seek_blocks=256)
    assert da.info["n_levels"] <= 32
    s = da.seek(b * 16384, 16384)
    st = da.sync()
    if st == ace.ACE_OK:  # only if block 0 happens to hold every source
        assert np.array_equal(s.cpu().numpy(), data[b * 16384:(b + 1) * 16384])
    else:
        assert st == ace.ACE_E_CORRUPT, ace.ace_status_str(st)
    out = da.seek(0, 16384)
    assert da.sync() == ace.ACE_OK
    assert np.array_equal(out.cpu().numpy(), data[:16384])
    da.close()


def test_decode_all_with_a_dependency_removed():
    """Whole decodes resolve matches one dependency level per launch; a
    dependency list that no longer covers a block's sources either leaves
    its levels valid (exact output) or is reported as corrupt."""
    data = synth.generate("text", 200_000, 12)
    for log2b, b in ((12, 30), (14, 9)):
        arc = oracle.encode(data, log2b, 4, 16)
        deps = oracle.deps(arc)[b]
        assert deps and deps != [(0, 0)]
        bad = with_dep_removed(arc, b)
        da = DeviceArchive(bad)
        ace.ace_index_set_tune(da.idx, ace.make_tune(wait_timeout_ns=20_000_000))
        out = da.decode_all()
        st = da.sync()
        assert st in (ace.ACE_OK, ace.ACE_E_CORRUPT, ace.ACE_E_TIMEOUT), ace.ace_status_str(st)
        if st == ace.ACE_OK:
            assert np.array_equal(out.cpu().numpy(), data)
        da.close()


def test_corrupt_payloads_are_reported_not_faulted():
    data = synth.generate("mixed", 300_000, 13)
    arc = ace.ace_encode(data, 12, 4)
    payload_off = int(arc[48:56].view(np.uint64)[0])
    rng = np.random.default_rng(1)
    seen = set()
    for trial in range(40):
        bad = arc.copy()
        k = int(rng.integers(payload_off, bad.size))
        bad[k] ^= np.uint8(1 << int(rng.integers(0, 8)))
        da = DeviceArchive(bad)
        ace.ace_index_set_tune(da.idx, ace.make_tune(wait_timeout_ns=50_000_000))
        out = da.decode_all()
        st = da.sync()
        assert st in (ace.ACE_OK, ace.ACE_E_CORRUPT), ace.ace_status_str(st)
        seen.add(st)
        if st == ace.ACE_OK:
            # a flip in padding leaves the archive valid; a payload flip the
            # end-of-stream checks miss (rANS has no checksum) decodes to the
            # same bytes the oracle decodes from the same corrupted archive
            ref = oracle.decode(bad)
            assert np.array_equal(out.cpu().numpy()[: data.size], ref)
        da.close()
    assert ace.ACE_E_CORRUPT in seen
    torch.cuda.synchronize()


def test_corrupt_directory_rejected_at_index_build():
    data = synth.generate("text", 100_000, 14)
    arc = ace.ace_encode(data, 10, 4)
    dir_off = int(arc[32:40].view(np.uint64)[0])
    bad = arc.copy()
    bad[dir_off + 24: dir_off + 28] = np.frombuffer(np.uint32(0xFFFFFFF0).tobytes(), np.uint8)  # stream_bytes
    with pytest.raises(ace.AceError) as e:
        DeviceArchive(bad)
    assert e.value.status == ace.ACE_E_CORRUPT


def test_device_fnv_matches_oracle():
    """Whole buffers and slices at every start alignment, with lengths around
    the 16-byte vectors and 128-byte batches the kernel reads."""
    data = synth.generate("fastq", 100_000, 15)
    d = torch.from_numpy(data).cuda()
    res = torch.zeros(1, dtype=torch.int64, device="cuda")
    cases = [(0, data.size), (0, 0)] + [(o, n) for o in range(0, 18) for n in (1, 15, 16, 127, 128, 129, 300, 4099)]
    for off, n in cases:
        ace.ace_fnv1a64(d[off:], n, res)
        torch.cuda.synchronize()
        assert int(res.cpu().numpy().view(np.uint64)[0]) == oracle.fnv1a64(data[off:off + n]), (off, n)


def test_levels_match_oracle():
    data = synth.generate("mixed", 1_000_000, 16)
    for arc in (ace.ace_encode(data, 12, 4), oracle.encode(data, 12, 4, 16)):
        da = DeviceArchive(arc)
        lv = oracle.levels(arc)
        assert da.info["n_levels"] == int(lv.max()) + 1
        nb = da.info["n_blocks"]
        level = da.d_index[256:256 + 4 * nb].cpu().numpy().view(np.uint32)
        assert np.array_equal(level, lv)
        n_lv = da.info["n_levels"]
        counts = ace.ace_index_levels(da.idx, n_lv)
        assert np.array_equal(counts, np.bincount(lv, minlength=n_lv)[:n_lv])
        da.close()


@pytest.mark.parametrize("copy_width", [8, 16])
def test_copy_widths_decode_and_seek(copy_width):
    """Both copy widths (16-byte pieces from 33 bytes, or from 512 with
    bytewise copies below) give the original bytes in whole decodes, seeks
    (which now take the piece copies too) and every overlap distance."""
    rng = np.random.default_rng(12)
    parts = []
    for d in range(1, 80, 3):
        for ln in (33, 47, 64, 100, 200, 511, 512, 700):
            parts.append(rng.integers(0, 256, 40).astype(np.uint8))
            unit = rng.integers(0, 256, max(d, 1)).astype(np.uint8)
            parts.append(np.resize(unit, d + ln))
            parts.append(parts[-1][: ln // 2])  # a non-overlapping repeat of part of it
    data = np.concatenate(parts + [synth.generate("genome", 600_000, 13)])
    tune = ace.make_tune(copy_width=copy_width)
    for arc in (ace.ace_encode(data, 12, 4), oracle.encode(data, 12, 4, 16)):
        for schedule in (ace.ACE_SCHEDULE_PASSES, ace.ACE_SCHEDULE_FUSED):
            st, out = gpu_decode(arc, ace.make_tune(schedule=schedule, copy_width=copy_width))
            assert st == ace.ACE_OK, ace.ace_status_str(st)
            assert np.array_equal(out, data)
        da = DeviceArchive(arc, max_seek_blocks=data.size // 4096 + 8)
        ace.ace_index_set_tune(da.idx, tune)
        n = data.size
        for coord, length in [(0, n), (n // 3, 80_000)] + [(int(c), int(rng.integers(1, 60_000)))
                                                           for c in rng.integers(0, n - 60_000, 6)]:
            s = da.seek(coord, length)
            assert da.sync() == ace.ACE_OK
            assert np.array_equal(s.cpu().numpy(), data[coord:coord + length]), (coord, length)
        da.close()
    with pytest.raises(ace.AceError):
        gpu_decode(ace.ace_encode(data[:5000], 12, 4), ace.make_tune(copy_width=4))
