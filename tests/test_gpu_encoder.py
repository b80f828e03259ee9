"""The GPU encoder: every archive it writes decodes to the original through
the oracle (the plain sequential decoder, sharing no code with the GPU
path) and through the GPU decoder, seeks included; its dependency levels
stay at most 3; and each rANS-coded stream is byte for byte what the
oracle's own rANS encoder writes for the same symbols, with the same
quantised frequencies."""
import numpy as np
import pytest

import oracle
import synth
import __graft_entry__

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2606_24531_gb300 import ace  # noqa: E402
from paper_2606_24531_gb300.archive import DeviceArchive  # noqa: E402

MM = {"mixed": 4, "text": 4, "fastq": 16, "genome": 20}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _encode(data, log2b, mm, **kw):
    d = torch.from_numpy(data).cuda()
    arc, st = ace.ace_encode_gpu(d, log2b, mm, stats=True, **kw)
    return arc.cpu().numpy(), st


def _dir(arc):
    hdr = arc[:64].view(np.uint64)
    nb, dir_off, payload_off = int(hdr[3]), int(hdr[4]), int(hdr[6])
    d = arc[dir_off:dir_off + 64 * nb].reshape(nb, 64)
    return nb, payload_off, d


@pytest.mark.parametrize("profile", ["mixed", "fastq", "genome", "text"])
@pytest.mark.parametrize("log2b", [8, 12, 14, 16])
def test_gpu_archives_decode_everywhere(profile, log2b):
    data = synth.generate(profile, 2_000_000 + 777, 90 + log2b)
    arc, st = _encode(data, log2b, MM[profile])
    assert np.array_equal(oracle.decode(arc), data)
    assert st["n_levels"] <= 4 and int(oracle.levels(arc).max()) + 1 == st["n_levels"]
    assert st["literal_bytes"] + st["match_bytes"] == data.size
    da = DeviceArchive(arc, max_seek_blocks=4096)
    out = da.decode_all()
    assert da.sync() == ace.ACE_OK
    assert np.array_equal(out.cpu().numpy()[:data.size], data)
    rng = np.random.default_rng(log2b)
    for c in rng.integers(0, data.size - 100_000, 6):
        c, n = int(c), int(rng.integers(1, 100_000))
        s = da.seek(c, n)
        assert da.sync() == ace.ACE_OK
        assert np.array_equal(s.cpu().numpy(), data[c:c + n])
    da.close()


def test_gpu_rans_streams_equal_the_oracles_encoder():
    data = synth.generate("mixed", 1_500_000, 93)
    arc, _ = _encode(data, 12, 4)
    nb, payload_off, d = _dir(arc)
    offs = d[:, :24].copy().view(np.uint64)
    sbytes = d[:, 24:36].copy().view(np.uint32)
    nsym = d[:, 36:48].copy().view(np.uint32)
    checked = 0
    for b in range(0, nb, max(1, nb // 40)):
        for k in range(3):
            n = int(nsym[b, k])
            if n == 0 or d[b, 56 + k] != 0:
                continue
            p = arc[payload_off + int(offs[b, k]): payload_off + int(offs[b, k]) + int(sbytes[b, k])]
            states = p[:128].view(np.uint32)
            present = np.unpackbits(p[128:160], bitorder="little").astype(bool)
            freq = np.zeros(256, np.uint16)
            fv = p[160:160 + 2 * int(present.sum())].view(np.uint16)
            freq[present] = fv
            head = 160 + ((2 * int(present.sum()) + 15) & ~15)
            sym = oracle.rans_decode(p[head:], states, freq, n)
            assert np.array_equal(oracle.rans_freqs(sym), freq), (b, k)  # the same quantisation
            st2, body = oracle.rans_encode(sym, freq)
            assert np.array_equal(st2, states), (b, k)
            assert np.array_equal(body, p[head:]), (b, k)
            checked += 1
    assert checked > 20


def test_gpu_encoder_adaptive_offsets_and_edges():
    data = synth.generate("genome", 3_000_000, 94)
    for kw in ({"adaptive": True}, {"off_width": 5}, {"adaptive": True, "chunk_blocks": 7}):
        arc, _ = _encode(data, 12, 20, **kw)
        assert np.array_equal(oracle.decode(arc), data), kw
        if kw.get("adaptive"):
            _, _, d = _dir(arc)
            assert (d[:, 56:59] == 1).any()
        if kw.get("off_width"):
            assert oracle.info(arc)["off_width"] == 5
    rng = np.random.default_rng(6)
    for n in (1, 3, 255, 256, 257, 4097):
        for alpha in (1, 2, 256):
            x = rng.integers(0, alpha, n).astype(np.uint8)
            arc, _ = _encode(x, 8, 4)
            assert np.array_equal(oracle.decode(arc), x), (n, alpha)
