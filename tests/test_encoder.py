"""The library's host encoder, checked with the oracle decoder: every
archive it writes decodes to the original, every match is valid, the
dependency table is exact, and dependency levels stay within the cap."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_24531_gb300 import ace
import __graft_entry__

from test_oracle_lz import _check_parse, _deps_from_tokens


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


@pytest.mark.parametrize("profile,mm", [("mixed", 4), ("fastq", 16), ("genome", 20), ("text", 4)])
@pytest.mark.parametrize("log2b", [8, 12, 14, 16])
def test_round_trip_through_oracle(profile, mm, log2b):
    data = synth.generate(profile, 300_000, 21)
    arc = ace.ace_encode(data, log2b, mm)
    assert np.array_equal(oracle.decode(arc), data)
    lv = oracle.levels(arc)
    assert lv.max() <= 3


def test_edge_sizes():
    rng = np.random.default_rng(0)
    B = 256
    for n in [0, 1, 2, 3, 4, 5, B - 1, B, B + 1, 3 * B + 7, 64 * B, 64 * B + 1]:
        for alpha in (1, 3, 256):
            data = rng.integers(0, alpha, n).astype(np.uint8)
            arc = ace.ace_encode(data, 8, 4)
            assert np.array_equal(oracle.decode(arc), data)


def test_matches_valid_and_dependencies_exact():
    data = synth.generate("mixed", 200_000, 3)
    arc = ace.ace_encode(data, 12, 4)
    _check_parse(data, arc, 4096, 4, exhaustive=False)
    want = _deps_from_tokens(arc)
    for b, ivs in enumerate(oracle.deps(arc)):
        s = set()
        for f, l in ivs:
            s.update(range(f, l + 1))
        assert s == want[b]


def test_deterministic_across_thread_counts():
    data = synth.generate("fastq", 1 << 21, 8)
    a1 = ace.ace_encode(data, 14, 16, threads=1)
    a8 = ace.ace_encode(data, 14, 16, threads=8)
    assert np.array_equal(a1, a8)


def test_five_byte_offsets_round_trip():
    """Offsets are stored in 5 bytes above 2^32 bytes of input; the encoder can
    force that width on small inputs so the path is covered without 4 GiB."""
    data = synth.generate("mixed", 400_000, 5)
    a4 = ace.ace_encode(data, 12, 4)
    a5 = ace.ace_encode(data, 12, 4, off_width=5)
    assert oracle.info(a4)["off_width"] == 4 and oracle.info(a5)["off_width"] == 5
    assert np.array_equal(oracle.decode(a5), data)
    assert np.array_equal(oracle.levels(a5), oracle.levels(a4))
    with pytest.raises(Exception):
        ace.ace_encode(data, 12, 4, off_width=3)


@pytest.mark.parametrize("profile,mm,log2b", [("fastq", 16, 14), ("genome", 20, 12), ("text", 4, 10)])
def test_stats_behind_the_roofline(profile, mm, log2b):
    """The parse statistics that the benchmark's algorithmic bytes come from,
    recounted from the oracle's decode of each block's tokens: matches,
    literal bytes, matched bytes, and the source bytes a match reads
    (min(length, distance): an overlapping match re-reads its own output),
    plus the level count."""
    data = synth.generate(profile, 600_000, 17)
    arc, st = ace.ace_encode(data, log2b, mm, stats=True)
    B = 1 << log2b
    nb = oracle.info(arc)["n_blocks"]
    toks = matches = lits = mbytes = src_bytes = 0
    for b in range(nb):
        lr, ml, src = oracle.block_tokens(arc, b)
        dst = b * B
        for t in range(len(lr)):
            dst += int(lr[t])
            if ml[t]:
                matches += 1
                mbytes += int(ml[t])
                src_bytes += min(int(ml[t]), dst - int(src[t]))
            dst += int(ml[t])
        toks += len(lr)
        lits += int(lr.sum())
    assert st["n_tokens"] == toks
    assert st["n_matches"] == matches
    assert st["literal_bytes"] == lits
    assert st["match_bytes"] == mbytes and lits + mbytes == data.size
    assert st["match_src_bytes"] == src_bytes
    assert st["n_levels"] == int(oracle.levels(arc).max()) + 1
