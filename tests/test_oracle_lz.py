"""Pins for the oracle's match layer, archive, dependency levels and seek
(absolute-offset LZ77 over fixed blocks, Section 2 and Section 3; unified
seek and its three-phase check, Section 5).

Decoding has exactly one correct result -- the original bytes -- so the
strongest pin is the input itself.  The parse is pinned by brute force on
short strings (every match is the longest earlier occurrence, its source
precedes its destination and reproduces it), by hand-worked cases, and the
dependency section by recomputing it from the decoded tokens.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_lines


def _tokens_all(arc):
    nb = oracle.info(arc)["n_blocks"]
    return [oracle.block_tokens(arc, b) for b in range(nb)]


def _check_parse(data, arc, B, min_match, exhaustive):
    """Every match: src < dst, orig[src+i] == orig[dst+i] (sequential overlap
    semantics hold on the original), dst range inside its block, at least
    min_match long; if exhaustive, no earlier position gives a longer match."""
    data = bytes(data)
    n = len(data)
    dst = 0
    for b, (lr, ml, src) in enumerate(_tokens_all(arc)):
        bend = min((b + 1) * B, n)
        for t in range(len(lr)):
            # literal positions: no match of >= min_match starts there (when exhaustive)
            for p in range(dst, dst + int(lr[t])):
                if exhaustive and bend - p >= min_match:
                    best = max((_match_len(data, q, p, bend) for q in range(p)), default=0)
                    assert best < min_match
            dst += int(lr[t])
            m = int(ml[t])
            if t == len(lr) - 1:
                assert m == 0
                continue
            s = int(src[t])
            assert m >= min_match and s < dst and dst + m <= bend
            assert all(data[s + i] == data[dst + i] for i in range(m))
            if exhaustive:
                lens = [_match_len(data, q, dst, bend) for q in range(dst)]
                assert m == max(lens)
                assert s == lens.index(m)  # ties go to the smallest source
            dst += m
        assert dst == bend


def _match_len(data, q, p, end):
    l = 0
    while p + l < end and data[q + l] == data[p + l]:
        l += 1
    return l


def test_hand_worked_parses():
    for line in golden_lines("lz_worked.txt"):
        fields = dict(kv.split("=", 1) for kv in line.split())
        data = fields["input"].encode()
        arc = oracle.encode(data, 8, 4, 0)
        lr, ml, src = oracle.block_tokens(arc, 0)
        got = ";".join("%d,%d,%d" % (a, b, c) for a, b, c in zip(lr, ml, src))
        assert got == fields["tokens"]
        assert bytes(oracle.decode(arc)) == data


def test_brute_force_binary_strings():
    """Every {a,b} string of length 0..10 round-trips and parses greedily."""
    for n in range(0, 11):
        for tup in itertools.product(b"ab", repeat=n):
            data = bytes(tup)
            arc = oracle.encode(data, 8, 4, 0)
            assert bytes(oracle.decode(arc)) == data
            _check_parse(data, arc, 256, 4, exhaustive=True)


def test_random_multi_block_parses():
    rng = np.random.default_rng(3)
    for trial in range(12):
        n = int(rng.integers(1, 1500))
        alpha = int(rng.integers(2, 6))
        data = bytes(rng.integers(97, 97 + alpha, n).astype(np.uint8))
        arc = oracle.encode(data, 8, 4, 0)
        assert bytes(oracle.decode(arc)) == data
        _check_parse(data, arc, 256, 4, exhaustive=(n <= 600))


def test_special_cases():
    # no byte string repeats: no matches at all
    data = bytes(range(256)) * 1
    arc = oracle.encode(data, 8, 4, 0)
    lr, ml, _ = oracle.block_tokens(arc, 0)
    assert list(lr) == [256] and list(ml) == [0]
    # a run of one byte: one literal, then one overlapping match at distance 1
    data = b"z" * 200
    arc = oracle.encode(data, 8, 4, 0)
    lr, ml, src = oracle.block_tokens(arc, 0)
    assert list(lr) == [1, 0] and list(ml) == [199, 0] and src[0] == 0
    # the empty input
    arc = oracle.encode(b"", 8, 4, 0)
    assert oracle.info(arc)["n_blocks"] == 0
    assert oracle.decode(arc).size == 0


def test_matches_clip_at_block_end():
    """A long repeat spanning blocks is cut at each block end; the next block
    starts a new match from the next source position."""
    unit = bytes(np.random.default_rng(5).integers(0, 256, 300).astype(np.uint8))
    data = unit + unit * 4
    arc = oracle.encode(data, 8, 4, 0)
    assert bytes(oracle.decode(arc)) == data
    _check_parse(data, arc, 256, 4, exhaustive=False)


def _deps_from_tokens(arc):
    hdr = oracle.info(arc)
    B = hdr["block_size"]
    out = []
    dst = 0
    for b, (lr, ml, src) in enumerate(_tokens_all(arc)):
        blocks = set()
        for t in range(len(lr)):
            dst += int(lr[t])
            m = int(ml[t])
            if m:
                s = int(src[t])
                rl = min(m, dst - s)
                blocks.update(k for k in range(s // B, (s + rl - 1) // B + 1) if k != b)
            dst += m
        out.append(blocks)
    return out


@pytest.mark.parametrize("profile", ["mixed", "fastq", "genome", "text"])
def test_profiles_round_trip_and_dependencies(profile):
    data = synth.generate(profile, 200_000, 9)
    arc = oracle.encode(data, 12, 4, 16)
    out = oracle.decode(arc)
    assert np.array_equal(out, data)
    assert oracle.fnv1a64(out) == oracle.fnv1a64(data)
    # the dependency section equals the block set recomputed from the tokens
    want = _deps_from_tokens(arc)
    got = oracle.deps(arc)
    for b, ivs in enumerate(got):
        s = set()
        for f, l in ivs:
            assert f <= l < b
            s.update(range(f, l + 1))
        assert s == want[b]
        # intervals are maximal: sorted, disjoint, not adjacent
        for (f0, l0), (f1, l1) in zip(ivs, ivs[1:]):
            assert l0 + 1 < f1
    # levels: 0 without dependencies, else one more than the deepest source
    lv = oracle.levels(arc)
    for b, blocks in enumerate(want):
        assert lv[b] == (1 + max(lv[k] for k in blocks) if blocks else 0)


def test_seek_slices_and_closure():
    data = synth.generate("mixed", 300_000, 4)
    arc = oracle.encode(data, 12, 4, 16)
    B = 4096
    deps = _deps_from_tokens(arc)
    rng = np.random.default_rng(1)
    cases = [(0, 1), (len(data) - 1, 1), (37 * B, B), (5 * B - 3, 7), (0, len(data))]
    cases += [(int(c), int(rng.integers(1, 20000))) for c in rng.integers(0, len(data) - 20000, 20)]
    for coord, length in cases:
        got = oracle.seek(arc, coord, length)
        assert np.array_equal(got, data[coord:coord + length])
        first, last = coord // B, (coord + length - 1) // B
        cl = set(oracle.closure(arc, first, last).tolist())
        assert set(range(first, last + 1)) <= cl
        for b in cl:  # closed under "reads from"
            assert deps[b] <= cl
    for coord, length in [(len(data), 1), (0, 0), (10, len(data))]:
        with pytest.raises(oracle.OracleError):
            oracle.seek(arc, coord, length)


def test_corrupted_archives_fail_cleanly():
    """A flipped byte either makes the oracle report the archive corrupt, or
    the decode has the original length and differs from the original only
    from the block holding the flipped byte onward: blocks before it never
    read it.  (rANS carries no checksum: a flipped payload bit is caught by
    the end-of-stream checks -- every state back at L, every byte consumed --
    nearly always, not always, since a perturbed state can converge back.)
    Nothing is read outside the archive."""
    data = synth.generate("text", 20_000, 2)
    B = 1024
    arc = oracle.encode(data, 10, 4, 16)
    hdr = arc[:64].view(np.uint64)
    nb, dir_off, payload_off = int(hdr[3]), int(hdr[4]), int(hdr[6])
    start = arc[dir_off:dir_off + 64 * nb].reshape(nb, 64)[:, :8].copy().view(np.uint64)[:, 0] + payload_off
    rng = np.random.default_rng(0)
    errors = silent = 0
    for _ in range(400):
        bad = arc.copy()
        k = int(rng.integers(0, bad.size))
        bad[k] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            out = oracle.decode(bad)
        except oracle.OracleError:
            errors += 1
            continue
        assert out.size == data.size
        if not np.array_equal(out, data):
            silent += 1
            assert k >= payload_off, "a flip outside the payload changed the output silently"
            blk = int(np.searchsorted(start, k, side="right")) - 1  # the block whose payload holds byte k
            assert np.array_equal(out[:blk * B], data[:blk * B]), k
    assert errors > 0.9 * 400 * (arc.size - payload_off) / arc.size * 0.9
