"""Archives and indices from storage, and archives that stay in host memory
(Section 7's VRAM wall, Section 8's next step: a prepared archive loaded
from disk).  Decoded bytes are checked bit-exact against the originals;
stored indices that do not belong to their archive, or whose levels or
order disagree with it, are rejected with ACE_E_CORRUPT."""
import os

import numpy as np
import pytest

import oracle
import synth
import __graft_entry__

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_24531_gb300 import ace  # noqa: E402
from paper_2606_24531_gb300.archive import (DeviceArchive, HostArchive, load_archive, save_archive,  # noqa: E402
                                            save_index)


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _check_archive(da, data, seeks=8):
    out = da.decode_all()
    assert da.sync() == ace.ACE_OK
    assert np.array_equal(out.cpu().numpy()[:data.size], data)
    rng = np.random.default_rng(3)
    for c in rng.integers(0, data.size - 50_000, seeks):
        c, n = int(c), int(rng.integers(1, 50_000))
        s = da.seek(c, n)
        assert da.sync() == ace.ACE_OK
        assert np.array_equal(s.cpu().numpy(), data[c:c + n]), (c, n)


def test_archive_and_index_from_files(tmp_path):
    for name, data, arc in [
            ("fastq", synth.generate("fastq", 3_000_000, 81), None),
            ("deep", synth.generate("text", 400_000, 82), "oracle")]:
        arc = oracle.encode(data, 10, 4, 16) if arc == "oracle" else ace.ace_encode(data, 14, 16)
        pa, pi = os.path.join(tmp_path, name + ".ace"), os.path.join(tmp_path, name + ".idx")
        save_archive(pa, arc)
        built = DeviceArchive(pa, max_seek_blocks=1024)
        save_index(pi, built)
        nb = built.info["n_blocks"]
        span = 256 + 2 * ((4 * nb + 255) & ~255)  # header, levels, order
        lv_built = built.d_index[:span].cpu().numpy().copy()
        loaded = DeviceArchive(pa, max_seek_blocks=1024, index=pi)
        assert loaded.info == built.info
        assert np.array_equal(loaded.d_index[:span].cpu().numpy(), lv_built)
        _check_archive(loaded, data)
        built.close()
        loaded.close()


def _blob_parts(blob):
    return blob[:256], blob[256:]


def _refresh_checksum(blob):
    """A tampered body with a consistent checksum, so that the device-side
    checks, not the checksum, must catch it."""
    b = blob.copy()
    b[80:88] = np.array([oracle.fnv1a64(b[256:])], np.uint64).view(np.uint8)
    return b


def test_stored_index_checks():
    data = synth.generate("mixed", 2_000_000, 83)
    arc = ace.ace_encode(data, 12, 4)
    other = ace.ace_encode(synth.generate("mixed", 2_000_000, 84), 12, 4)
    da = DeviceArchive(arc)
    blob = ace.ace_index_export(da.idx)
    nb = da.info["n_blocks"]

    def load(a, b):
        return DeviceArchive(a, index=b)

    assert load(arc, blob).info == da.info  # the untouched blob loads
    with pytest.raises(ace.AceError) as e:
        load(other, blob)  # another archive's index
    assert e.value.status == ace.ACE_E_CORRUPT
    bad = blob.copy()
    bad[300] ^= 1  # a flipped byte: the checksum
    with pytest.raises(ace.AceError) as e:
        load(arc, bad)
    assert e.value.status == ace.ACE_E_CORRUPT
    lv = da.d_index[256:256 + 4 * nb].cpu().numpy().view(np.uint32)
    b = int(np.argmax(lv))  # a block of the deepest level
    bad = blob.copy()
    bad[256 + 256 + 4 * b:256 + 256 + 4 * b + 4] = np.array([lv[b] + 1], np.uint32).view(np.uint8)
    with pytest.raises(ace.AceError) as e:
        load(arc, _refresh_checksum(bad))  # a level that breaks the level rule
    assert e.value.status == ace.ACE_E_CORRUPT
    order_off = 256 + ((256 + 4 * nb + 255) & ~255)
    order = blob[order_off:order_off + 4 * nb].view(np.uint32)
    i0 = 0
    i1 = int(np.argmax(lv[order] > lv[order[0]]))  # the first block of a deeper level
    assert i1 > 0
    bad = blob.copy()
    o = bad[order_off:order_off + 4 * nb].view(np.uint32)
    o[i0], o[i1] = order[i1], order[i0]  # a permutation out of level order
    with pytest.raises(ace.AceError) as e:
        load(arc, _refresh_checksum(bad))
    assert e.value.status == ace.ACE_E_CORRUPT
    bad = blob.copy()
    o = bad[order_off:order_off + 4 * nb].view(np.uint32)
    o[1] = o[0]  # a block twice, another never
    with pytest.raises(ace.AceError) as e:
        load(arc, _refresh_checksum(bad))
    assert e.value.status == ace.ACE_E_CORRUPT
    da.close()


def test_host_resident_archive(tmp_path):
    """The archive stays in host memory (pinned and mapped); index and
    scratch on the device.  Whole decode, seeks, and a range decoded to host
    memory in sub-ranges, with a built and with a stored index."""
    data = synth.generate("genome", 24 << 20, 85)
    arc = ace.ace_encode(data, 14, 20)
    pa = os.path.join(tmp_path, "g.ace")
    save_archive(pa, arc)
    ha = HostArchive(pa, max_seek_blocks=2048)
    _check_archive(ha, data)
    h = ha.decode_range_to_host(12345, data.size - 20000, chunk_blocks=256)
    assert np.array_equal(h.numpy(), data[12345:12345 + data.size - 20000])
    pi = os.path.join(tmp_path, "g.idx")
    save_index(pi, ha)
    hb = HostArchive(load_archive(pa), max_seek_blocks=2048, index=pi)
    assert hb.info == ha.info
    B = hb.block_size
    s = hb.seek(0, 1001 * B)  # blocks 0..1000, the paper's range decode
    assert hb.sync() == ace.ACE_OK
    assert np.array_equal(s.cpu().numpy(), data[:1001 * B])
    ha.close()
    hb.close()
