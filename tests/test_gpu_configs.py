"""Full-size parity for the FASTQ and genome workloads, in the launch
configuration the benchmark times: the decoded bytes equal the regenerated
original (a property that holds at any size), and sampled seeks equal the
original slices."""
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


def _seek_many(da, d_data, blocks):
    B = da.block_size
    out = torch.empty((len(blocks), B), dtype=torch.uint8, device="cuda")
    for i, b in enumerate(blocks):
        ace.ace_seek(da.idx, int(b) * B, B, out[i], B, da.d_scratch, da.scratch_bytes)
    assert da.sync() == ace.ACE_OK
    ref = d_data[: (da.total // B) * B].view(-1, B)[torch.as_tensor(blocks.astype(np.int64), device="cuda")]
    assert torch.equal(out, ref)


def test_fastq_256mib_decode_and_10000_seeks():
    data = synth.generate("fastq", 1 << 28, 1)
    arc = ace.ace_encode(data, 14, 16)
    da = DeviceArchive(arc, max_seek_blocks=512)
    assert da.info["n_blocks"] == 16384
    d_data = torch.from_numpy(data).cuda()
    out = da.decode_all()
    assert da.sync() == ace.ACE_OK
    assert torch.equal(out, d_data)
    blocks = synth.uniform(2, 10000, 0, da.info["n_blocks"] - 1)
    _seek_many(da, d_data, blocks)
    da.close()


def test_genome_1gib_decode():
    data = synth.generate("genome", 1 << 30, 3)
    arc = ace.ace_encode(data, 14, 20)
    da = DeviceArchive(arc, max_seek_blocks=512)
    assert da.info["n_blocks"] == 65536
    d_data = torch.from_numpy(data).cuda()
    out = da.decode_all()
    assert da.sync() == ace.ACE_OK
    assert torch.equal(out, d_data)
    blocks = synth.uniform(6, 500, 0, da.info["n_blocks"] - 1)
    _seek_many(da, d_data, blocks)
    da.close()
