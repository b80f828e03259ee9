"""The seeded input recipes: determinism and the stated shapes of each
profile (FASTQ records, genome alphabet, mixed copy fraction), and the
workload tables."""
import math

import numpy as np

import synth


def test_deterministic_and_seeded():
    for p in synth.PROFILES:
        a = synth.generate(p, 50_000, 5)
        b = synth.generate(p, 50_000, 5)
        c = synth.generate(p, 50_000, 6)
        assert np.array_equal(a, b)
        assert not np.array_equal(a, c)
        # a prefix of a longer run is the shorter run
        assert np.array_equal(synth.generate(p, 70_000, 5)[:50_000], a)


def test_fastq_shape():
    data = bytes(synth.generate("fastq", 200_000, 1))
    lines = data.split(b"\n")[:-1]
    nrec = len(lines) // 4
    assert nrec > 100
    for r in range(nrec):
        h, seq, plus, qual = lines[4 * r: 4 * r + 4]
        assert h.startswith(b"@SIM:1:FC:1:1101:")
        assert len(seq) == 150 and set(seq) <= set(b"ACGTN")
        assert plus == b"+"
        assert len(qual) == 150 and min(qual) >= 2 + 33 and max(qual) <= 41 + 33
        for s, q in zip(seq, qual):
            if s == ord("N"):
                assert q == 2 + 33
    # mean quality falls along the read
    q = np.array([list(lines[4 * r + 3]) for r in range(nrec)], float) - 33
    assert q[:, :10].mean() > q[:, -10:].mean() + 7


def test_genome_shape():
    data = synth.generate("genome", 3_000_000, 3)
    assert set(np.unique(data).tolist()) <= set(b"ACGT")
    base = bytes(data[:1_000_000])
    # after the tandem region a mutated copy of the base follows: its first kilobase
    # appears again almost unchanged
    assert bytes(data[1_000_000:]).find(base[:64]) > 0


def test_mixed_copy_fraction_and_text():
    data = synth.generate("mixed", 1 << 20, 0)
    text = synth.generate("text", 1 << 20, 0)
    assert set(np.unique(text).tolist()) <= set(b"abcdefghijklmnopqrstuvwxyz ")
    assert set(np.unique(data).tolist()) <= set(b"abcdefghijklmnopqrstuvwxyz ")
    # the text profile starts identical to mixed until the first copy at >= 512 bytes
    assert np.array_equal(data[:512], text[:512])


def test_objects_table():
    sizes, profiles, bsz, seeds = synth.objects(4, 4096)
    assert sizes.min() >= 4096 and sizes.max() <= 1 << 26
    assert set(np.unique(bsz).tolist()) == {4096, 16384, 65536}
    assert set(np.unique(profiles).tolist()) == {0, 1, 2, 3}
    assert seeds[0] == 1000 and seeds[-1] == 1000 + 4095
    # log-uniform: the mean of log(size) sits in the middle of [ln 4096, ln 2^26]
    mid = (math.log(4096) + math.log(1 << 26)) / 2
    assert abs(np.log(sizes.astype(float)).mean() - mid) < 0.2


def test_det_math_and_requests():
    for x in [1e-9, 0.5, 1.0, 2.0, 10.0, 12345.678]:
        assert abs(synth.det_log(x) - math.log(x)) < 1e-12 * max(1.0, abs(math.log(x)))
    for x in [-20.0, -1.0, 0.0, 0.3, 5.0, 30.0]:
        assert abs(synth.det_exp(x) - math.exp(x)) <= 1e-14 * math.exp(x)
    sizes = np.array([1 << 30] * 8, np.uint64)
    t, a, c, ln = synth.requests(5, 20000, 1e5, sizes)
    assert np.all(np.diff(t.astype(np.int64)) >= 0)
    gaps = np.diff(t.astype(float))
    assert abs(gaps.mean() - 1e4) < 500  # 1e5 req/s -> 10 us mean gap
    assert np.all(c + ln <= sizes[a])
    assert ln.min() >= 1 and ln.max() <= 1 << 20
