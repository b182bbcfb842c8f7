"""The span encoding of the warp row rasteriser, checked on the CPU.

A row's spans [a, b) of region v enter a difference array as +w at a and -w
at b with w = 2^17 + v - R (mod 2^32, R = the background id <= 65534); with P
the prefix sum at a pixel (mod 2^32), the kernel takes the low 16 bits of
R + P as the pixel's label and flags the pixel as inside two or more spans
when P >= 2^17.  This test checks that arithmetic against painting the spans
directly (the label is the region of the only covering span, the background
when none covers), for random rows, for every count of covering spans up to
the 128 spans one warp row holds, and at the largest background id.
"""
import numpy as np
import pytest

MASK = (1 << 32) - 1


def encode_decode(spans, n, R):
    diff = np.zeros(n + 1, np.uint64)
    for a, b, v in spans:
        if a < b:
            w = (0x20000 + v - R) & MASK
            diff[a] = (int(diff[a]) + w) & MASK
            diff[b] = (int(diff[b]) - w) & MASK
    P = np.zeros(n, np.uint64)
    acc = 0
    for i in range(n):
        acc = (acc + int(diff[i])) & MASK
        P[i] = acc
    label = ((P + R) & 0xFFFF).astype(np.int64)
    multi = P >= 0x20000
    return label, multi


def paint(spans, n, R):
    cover = np.zeros(n, np.int64)
    label = np.full(n, R, np.int64)
    for a, b, v in spans:
        cover[a:b] += 1
        label[a:b] = v
    return label, cover


@pytest.mark.parametrize("R", [1, 2, 200, 4096, 65534])
def test_single_coverage_labels_and_flags(R):
    rng = np.random.default_rng(R)
    n = 1024
    for _ in range(20):
        # disjoint spans (a valid subdivision of the row), region ids in [0, R)
        cuts = np.sort(rng.choice(np.arange(1, n), size=2 * int(rng.integers(1, 60)), replace=False))
        spans = [(int(cuts[2 * k]), int(cuts[2 * k + 1]), int(rng.integers(0, R))) for k in range(len(cuts) // 2)]
        got, multi = encode_decode(spans, n, R)
        want, cover = paint(spans, n, R)
        assert not multi.any()
        np.testing.assert_array_equal(got, want)
        assert cover.max() <= 1


@pytest.mark.parametrize("R", [2, 300, 65534])
def test_multiple_coverage_is_flagged_exactly(R):
    rng = np.random.default_rng(7 + R)
    n = 512
    for _ in range(20):
        k = int(rng.integers(2, 128))                     # up to the 128 spans of one warp row
        spans = []
        for _ in range(k):
            a, b = sorted(rng.integers(0, n + 1, size=2).tolist())
            spans.append((a, b, int(rng.integers(0, R))))
        got, multi = encode_decode(spans, n, R)
        want, cover = paint(spans, n, R)
        np.testing.assert_array_equal(multi, cover >= 2)
        one = cover <= 1
        np.testing.assert_array_equal(got[one], want[one])


def test_extreme_stack_does_not_wrap():
    # 128 spans over the same pixels, all of the largest region id, at the
    # largest background id: the prefix stays below 2^32 and is flagged
    R = 65534
    spans = [(0, 16, R - 1)] * 128
    got, multi = encode_decode(spans, 32, R)
    assert multi[:16].all() and not multi[16:].any()
    assert (got[16:] == R).all()
