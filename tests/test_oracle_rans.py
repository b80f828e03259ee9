"""Pins for the oracle's interleaved rANS coder (per-block entropy layer,
Section 3; interleaved rANS, Section 1 and Section 9).

The coder is pinned by things other than itself: hand-worked examples,
closed-form byte counts for uniform tables, the information identity that
ties the emitted bits to the symbols' code lengths, round trips over every
short string of small alphabets, and the state invariants.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from conftest import golden_lines

L = 1 << 23


def _freq_from_spec(spec):
    f = np.zeros(256, np.uint16)
    if spec == "uniform256":
        f[:] = 16
    else:
        for item in spec.split(","):
            s, v = item.split(":")
            f[int(s, 16)] = int(v)
    return f


def test_hand_worked_examples():
    for line in golden_lines("rans_worked.txt"):
        fields = dict(kv.split("=") for kv in line.split()[1:])
        freq = _freq_from_spec(fields["freq"])
        sym = bytes.fromhex(fields["symbols"])
        st, stream = oracle.rans_encode(sym, freq)
        want = np.full(32, L, np.uint32)
        for j in range(32):
            if "states%d" % j in fields:
                want[j] = int(fields["states%d" % j], 16)
        assert st.tolist() == want.tolist()
        assert bytes(stream) == bytes.fromhex(fields["stream"])
        assert bytes(oracle.rans_decode(stream, st, freq, len(sym))) == sym


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_uniform_table_exact_byte_count(k):
    """With 2^k equal frequencies every symbol adds exactly k bits to its
    state's bit length and each emitted byte removes 8, so a lane that codes m
    symbols emits floor(m k / 8) bytes and ends with bit length
    24 + (m k mod 8)."""
    rng = np.random.default_rng(k)
    freq = np.zeros(256, np.uint16)
    freq[: 1 << k] = 4096 >> k
    for n in [0, 1, 31, 32, 33, 100, 1000, 4097]:
        sym = rng.integers(0, 1 << k, n).astype(np.uint8)
        st, stream = oracle.rans_encode(sym, freq)
        m = [len(range(j, n, 32)) for j in range(32)]
        assert stream.size == sum(mj * k // 8 for mj in m)
        for j in range(32):
            assert int(st[j]).bit_length() == 24 + (m[j] * k) % 8
        assert np.array_equal(oracle.rans_decode(stream, st, freq, n), sym)


def test_information_identity():
    """Coding symbol s multiplies the state by about 4096 / f_s and each
    emitted byte divides it by 256, so the emitted bits plus the states' growth
    above L equal the symbols' total code length sum(log2(4096 / f_s)), up to
    a rounding term bounded per step.  A dropped or wrong term in the coding
    step breaks this identity."""
    rng = np.random.default_rng(7)
    for alpha, n in [(3, 5000), (20, 20000), (200, 20000)]:
        p = rng.dirichlet(np.ones(alpha) * 0.5)
        sym = rng.choice(alpha, n, p=p).astype(np.uint8)
        freq = oracle.rans_freqs(sym)
        st, stream = oracle.rans_encode(sym, freq)
        code_bits = sum(math.log2(4096 / freq[s]) for s in sym)
        state_bits = sum(math.log2(int(x) / L) for x in st)
        got = 8 * stream.size + state_bits
        # x' = floor(x/f) 4096 + (x mod f) + c_s differs from x 4096 / f by at
        # most 4096 while x' >= 2^23, so each step is off by < 2^-11 / ln 2 bits
        assert abs(got - code_bits) <= n * 2.0 ** -10 + 1e-6
        assert np.array_equal(oracle.rans_decode(stream, st, freq, n), sym)


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_exhaustive_short_strings(alpha):
    """Every string of length 0..6 over an alphabet of 1, 2 or 3 symbols
    round-trips, the frequencies sum to 4096, and every stored state lies in
    [L, 2^31)."""
    for n in range(0, 7):
        for tup in itertools.product(range(alpha), repeat=n):
            sym = np.array([65 + t for t in tup], np.uint8)
            freq = oracle.rans_freqs(sym)
            if n:
                assert int(freq.sum()) == 4096
                assert all((freq[65 + t] > 0) for t in tup)
            st, stream = oracle.rans_encode(sym, freq)
            assert all(L <= int(x) < (1 << 31) for x in st)
            assert np.array_equal(oracle.rans_decode(stream, st, freq, n), sym)


def test_random_lengths_round_trip():
    rng = np.random.default_rng(11)
    for n in list(range(0, 70)) + list(rng.integers(0, 5000, 40)):
        alpha = int(rng.integers(1, 257))
        sym = rng.integers(0, alpha, int(n)).astype(np.uint8)
        freq = oracle.rans_freqs(sym)
        st, stream = oracle.rans_encode(sym, freq)
        assert all(L <= int(x) < (1 << 31) for x in st)
        assert np.array_equal(oracle.rans_decode(stream, st, freq, int(n)), sym)


def test_frequency_normalisation_cases():
    # one symbol takes the whole scale
    f = oracle.rans_freqs(np.full(10, 7, np.uint8))
    assert f[7] == 4096 and f.sum() == 4096
    # two equal symbols split it
    f = oracle.rans_freqs(np.array([1, 2] * 50, np.uint8))
    assert f[1] == 2048 and f[2] == 2048
    # a rare symbol keeps frequency 1, the shortfall goes to the common one
    sym = np.concatenate([np.zeros(10 ** 6, np.uint8), np.ones(1, np.uint8)])
    f = oracle.rans_freqs(sym)
    assert f[1] == 1 and f[0] == 4095
    # 255 rare symbols at 1 each push the sum over; the excess comes off the big one
    sym = np.concatenate([np.zeros(10 ** 6, np.uint8), np.arange(1, 256, dtype=np.uint8)])
    f = oracle.rans_freqs(sym)
    assert (f[1:] == 1).all() and f[0] == 4096 - 255
    assert f.sum() == 4096


def test_decoder_rejects_bad_states_and_leftover_bytes():
    sym = np.frombuffer(b"hello world, hello rans", np.uint8)
    freq = oracle.rans_freqs(sym)
    st, stream = oracle.rans_encode(sym, freq)
    bad = st.copy()
    bad[3] = L - 1
    with pytest.raises(oracle.OracleError):
        oracle.rans_decode(stream, bad, freq, sym.size)
    with pytest.raises(oracle.OracleError):
        oracle.rans_decode(np.concatenate([stream, [0]]).astype(np.uint8), st, freq, sym.size)


def test_fnv_published_vectors():
    for line in golden_lines("fnv1a_vectors.txt"):
        text, h32, h64 = line.split()
        data = text.strip('"').encode()
        assert oracle.fnv1a32(data) == int(h32, 16)
        assert oracle.fnv1a64(data) == int(h64, 16)
