"""ace_seek_noalloc, the seek for callers that cannot allocate device memory
(an application that owns all device memory through its own pool, a
plug-in inside one, a request thread that must never reach the allocator):
its output through the C ABI equals ace_seek's, bit for bit, on calls in a
row, and it refuses requests larger than its fixed scratch.

Kept in a file that pytest collects last, so a run that stops at the first
failure has run every other test before this one."""
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
    torch.cuda.set_device(0)


def test_noalloc_seek_equals_seek_on_calls_in_a_row():
    data = synth.generate("mixed", 2_500_000, 21)
    arc = ace.ace_encode(data, 14, 4)
    da = DeviceArchive(arc, max_seek_blocks=256)
    for coord, length in [(37 * 16384, 16384), (5000, 300_000), (len(data) - 7, 7)]:
        ref = da.seek(coord, length)
        assert da.sync() == ace.ACE_OK
        out = torch.full((length,), 0xAB, dtype=torch.uint8, device="cuda")
        st = ace.ace_seek_noalloc(da.idx, coord, length, out, length)
        assert st == ace.ACE_OK, ace.ace_status_str(st)
        assert torch.equal(out, ref)
        assert np.array_equal(out.cpu().numpy(), data[coord:coord + length])
    # another archive on the same shared scratch, whose layout differs
    data2 = synth.generate("fastq", 1_000_000, 22)
    arc2 = ace.ace_encode(data2, 12, 16)
    db = DeviceArchive(arc2, max_seek_blocks=64)
    for coord, length in [(123_457, 4096), (0, 20_000)]:
        ref = db.seek(coord, length)
        assert db.sync() == ace.ACE_OK
        out = torch.empty(length, dtype=torch.uint8, device="cuda")
        assert ace.ace_seek_noalloc(db.idx, coord, length, out, length) == ace.ACE_OK
        assert torch.equal(out, ref)
    da.close()
    db.close()


def test_noalloc_seek_rejects_requests_beyond_its_scratch():
    # 64 KiB blocks: the fixed 32 MiB scratch holds fewer than 512 of them
    data = synth.generate("genome", 40 << 20, 23)
    arc = ace.ace_encode(data, 16, 20)
    da = DeviceArchive(arc)
    out = torch.empty(len(data), dtype=torch.uint8, device="cuda")
    assert ace.ace_seek_noalloc(da.idx, 0, len(data), out, len(data)) == ace.ACE_E_NOMEM
    # a request that fits still works afterwards
    st = ace.ace_seek_noalloc(da.idx, 5 << 20, 65536, out, 65536)
    assert st == ace.ACE_OK
    assert np.array_equal(out[:65536].cpu().numpy(), data[5 << 20:(5 << 20) + 65536])
    da.close()


def test_noalloc_seek_reports_a_corrupt_archive_after_another_layout():
    """The fixed scratch keeps whatever the last call left in it.  After calls
    on an archive of another shape (another block size, other block counts
    and token records), an archive whose block lost its dependency list on the
    host must come back as ACE_E_CORRUPT -- its source blocks are outside the
    seek's closure -- and never read through a stale block-to-slot entry.  A
    clean seek still works afterwards."""
    data_a = synth.generate("mixed", 3_000_000, 24)
    arc_a = ace.ace_encode(data_a, 14, 4)
    da = DeviceArchive(arc_a)
    out = torch.empty(300_000, dtype=torch.uint8, device="cuda")
    for coord, length in [(0, 16384), (1_000_000, 300_000), (2_990_000, 10_000)]:
        assert ace.ace_seek_noalloc(da.idx, coord, length, out, length) == ace.ACE_OK
        assert np.array_equal(out[:length].cpu().numpy(), data_a[coord:coord + length])
    data_b = synth.generate("text", 200_000, 12)
    arc_b = oracle.encode(data_b, 12, 4, 16)
    b = 30
    assert oracle.deps(arc_b)[b] not in ([], [(0, 0)])
    db = DeviceArchive(with_dep_removed(arc_b, b))
    for _ in range(2):
        st = ace.ace_seek_noalloc(db.idx, b * 4096, 100, out, 100)
        assert st == ace.ACE_E_CORRUPT, ace.ace_status_str(st)
    st = ace.ace_seek_noalloc(db.idx, 0, 4096, out, 4096)
    assert st == ace.ACE_OK, ace.ace_status_str(st)
    assert np.array_equal(out[:4096].cpu().numpy(), data_b[:4096])
    # and the first archive again, on the same array
    assert ace.ace_seek_noalloc(da.idx, 5000, 70_000, out, 70_000) == ace.ACE_OK
    assert np.array_equal(out[:70_000].cpu().numpy(), data_a[5000:75_000])
    da.close()
    db.close()
