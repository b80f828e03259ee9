"""ace_seek_noalloc, the seek for callers that cannot allocate device memory
(an application that owns all device memory through its own pool, a
plug-in inside one, a request thread that must never reach the allocator):
its output through the C ABI equals ace_seek's, bit for bit, on calls in a
row, and it refuses requests larger than its fixed scratch.

Kept in a file that pytest collects last, so a run that stops at the first
failure has run every other test before this one."""
import numpy as np
import pytest

import synth
import __graft_entry__

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
