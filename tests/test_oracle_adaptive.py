"""Per-stream adaptive entropy (Section 4: whether rANS pays is data-dependent,
so it is decided per stream at encode time).  The oracle stores a stream
verbatim (directory mode 1) exactly when its rANS coding would take at least
as many bytes; everything else about the archive stays the same.  Pinned
against the rANS-only archive of the same input, the original bytes, and
the token counts the streams must hold."""
import numpy as np
import pytest

import oracle
import synth
from paper_2606_24531_gb300.archive import stream_report


def _dir(arc):
    hdr = arc[:64].view(np.uint64)
    nb, dir_off = int(hdr[3]), int(hdr[4])
    d = arc[dir_off:dir_off + 64 * nb].reshape(nb, 64)
    return {"stored": d[:, 24:36].copy().view(np.uint32), "nsym": d[:, 36:48].copy().view(np.uint32),
            "ntok": d[:, 48:52].copy().view(np.uint32)[:, 0], "nesc": d[:, 52:56].copy().view(np.uint32)[:, 0],
            "mode": d[:, 56:59].copy()}


@pytest.mark.parametrize("profile", ["genome", "fastq", "text", "mixed"])
@pytest.mark.parametrize("log2b", [8, 12, 14])
def test_stored_exactly_when_rans_does_not_shrink(profile, log2b):
    data = synth.generate(profile, 300_000, 11)
    a0 = oracle.encode(data, log2b, 4, 16)
    a1 = oracle.encode(data, log2b, 4, 16, adaptive=True)
    assert np.array_equal(oracle.decode(a1), data)
    d0, d1 = _dir(a0), _dir(a1)
    assert (d0["mode"] == 0).all()
    for key in ("nsym", "ntok", "nesc"):
        assert np.array_equal(d0[key], d1[key])  # the same parse and streams
    stored = (d0["stored"] >= d0["nsym"]) & (d0["nsym"] > 0)
    assert np.array_equal(d1["mode"] == 1, stored)
    assert np.array_equal(d1["stored"], np.where(stored, d0["nsym"], d0["stored"]))
    assert np.array_equal(oracle.levels(a1), oracle.levels(a0))
    assert a1.size <= a0.size


def test_small_blocks_store_the_structural_streams():
    """At 256-byte blocks the length and offset streams are a few dozen
    bytes, far below rANS's 160-byte stream head: stored, as the paper
    finds for structural streams."""
    data = synth.generate("genome", 200_000, 2)
    rep = stream_report(oracle.encode(data, 8, 4, 16, adaptive=True))
    assert rep["lengths"]["stored_verbatim_blocks"] > 0 and rep["offsets"]["stored_verbatim_blocks"] > 0
    assert rep["lengths"]["ratio"] >= 1.0 and rep["offsets"]["ratio"] >= 1.0


def test_seek_through_stored_streams():
    data = synth.generate("mixed", 400_000, 6)
    arc = oracle.encode(data, 10, 4, 16, adaptive=True)
    assert (_dir(arc)["mode"] == 1).any()
    for coord, n in ((0, 1), (5000, 3000), (399_000, 1000), (123_456, 77_777)):
        assert np.array_equal(oracle.seek(arc, coord, n), data[coord:coord + n])


def test_stored_stream_checks():
    data = synth.generate("mixed", 100_000, 7)
    arc = oracle.encode(data, 8, 4, 16, adaptive=True)
    d = _dir(arc)
    b, k = map(int, np.argwhere(d["mode"] == 1)[0])
    dir_off = int(arc[32:40].view(np.uint64)[0])
    e = dir_off + 64 * b
    bad = arc.copy()
    bad[e + 24 + 4 * k: e + 28 + 4 * k] = np.array([int(d["nsym"][b, k]) + 1], np.uint32).view(np.uint8)
    with pytest.raises(Exception):
        oracle.decode(bad)  # a stored stream holds exactly its symbols
    bad = arc.copy()
    bad[e + 56 + k] = 2
    with pytest.raises(Exception):
        oracle.decode(bad)  # no third mode


def test_report_counts_the_token_streams():
    """stream_report's symbol totals are what the tokens imply: every literal,
    two codes per token plus two bytes per escape, off_width bytes per match."""
    data = synth.generate("text", 150_000, 9)
    arc = oracle.encode(data, 12, 4, 16)
    rep = stream_report(arc)
    nb = oracle.info(arc)["n_blocks"]
    w = oracle.info(arc)["off_width"]
    lits = toks = matches = 0
    for b in range(nb):
        lr, ml, _ = oracle.block_tokens(arc, b)
        lits += int(lr.sum())
        toks += len(lr)
        matches += len(lr) - 1
    nesc = int(_dir(arc)["nesc"].sum())
    assert rep["literals"]["raw"] == lits
    assert rep["lengths"]["raw"] == 2 * toks + 2 * nesc
    assert rep["offsets"]["raw"] == w * matches
    assert rep["literals"]["stored_verbatim_blocks"] == 0


@pytest.mark.parametrize("profile", ["genome", "fastq", "text", "mixed"])
def test_library_encoder_adaptive_option(profile):
    """The library's host encoder with adaptive set: the oracle decodes its
    archive to the original, and a stream is stored exactly when the
    library's rANS-only archive of the same input spends at least its symbol
    count on it, with the same parse (every other directory count equal)."""
    from paper_2606_24531_gb300 import ace

    data = synth.generate(profile, 1_500_000, 12)
    mm = {"genome": 20, "fastq": 16, "text": 4, "mixed": 4}[profile]
    for log2b in (10, 14):
        a0 = ace.ace_encode(data, log2b, mm)
        a1 = ace.ace_encode(data, log2b, mm, adaptive=True)
        assert np.array_equal(oracle.decode(a1), data)
        d0, d1 = _dir(a0), _dir(a1)
        for key in ("nsym", "ntok", "nesc"):
            assert np.array_equal(d0[key], d1[key])
        stored = (d0["stored"] >= d0["nsym"]) & (d0["nsym"] > 0)
        assert np.array_equal(d1["mode"] == 1, stored)
        assert np.array_equal(d1["stored"], np.where(stored, d0["nsym"], d0["stored"]))
        assert a1.size <= a0.size
        for coord, n in ((0, 1), (len(data) // 3, 5000), (len(data) - 100, 100)):
            assert np.array_equal(oracle.seek(a1, coord, n), data[coord:coord + n])
