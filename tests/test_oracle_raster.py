"""Pins of the oracle's rasteriser and pixel areas (Sec. 4.1 step 2)."""
import json
import os

import numpy as np
import pytest

from oracle import inim_oracle as O
from paper_2604_13880_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _arrays(m):
    return m.ring_off, m.ring_idx, m.ring_region, m.n_regions


def _poly_mesh(poly):
    p = np.array(poly, np.float64)
    return synth.Mesh(p, np.array([0, len(p)], np.int32), np.arange(len(p), dtype=np.int32),
                      np.zeros(1, np.int32), 1)


def test_golden_cases():
    gold = json.load(open(os.path.join(GOLD, "raster_cases.json")))
    for c in gold["cases"]:
        m = _poly_mesh(c["poly"])
        k = c["log2_res"]
        for fn in (O.labels_bruteforce, O.labels_scanline):
            lab, cnt, ov = fn(m.verts, *_arrays(m), k)
            got = sorted((int(i), int(j)) for j, i in zip(*np.nonzero(lab == 0)))
            if "pixel_list" in c:
                want = sorted(map(tuple, c["pixel_list"]))
            else:
                lo, hi = (2, 5) if c["count"] == 16 else (2, 4)
                want = [(i, j) for i in range(lo, hi + 1) for j in range(lo, hi + 1)]
            assert got == sorted(want), (c["name"], fn.__name__)
            assert cnt[0] == c["count"] and not ov


@pytest.mark.parametrize("seed,R,V,k", [(1, 6, 200, 4), (2, 12, 500, 5), (3, 30, 1500, 6)])
def test_scanline_equals_bruteforce(seed, R, V, k):
    m = synth.voronoi_map(R, V, seed=seed, jitter=0.3)
    a = O.labels_bruteforce(m.verts, *_arrays(m), k)
    b = O.labels_scanline(m.verts, *_arrays(m), k)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2] == False  # noqa: E712  (valid subdivision: no overlap)


def test_snapped_onto_centres_and_junctions():
    # vertices snapped exactly onto pixel-centre rows/columns, shared edges:
    # every pixel still gets exactly one owner (no overlap, no gap inside)
    k = 5
    N = 1 << k
    m = synth.voronoi_map(10, 300, seed=11)
    xy = (np.floor(m.verts * N) + 0.5) / N
    lab_b, cnt_b, ov_b = O.labels_bruteforce(xy, *_arrays(m), k)
    lab_s, cnt_s, ov_s = O.labels_scanline(xy, *_arrays(m), k)
    np.testing.assert_array_equal(lab_b, lab_s)
    assert not ov_b and not ov_s


def test_overlap_rule():
    # two overlapping squares: the smaller id wins and the flag is raised
    m = synth.square_map([(0.2, 0.2, 0.6, 0.6), (0.4, 0.4, 0.8, 0.8)])
    for fn in (O.labels_bruteforce, O.labels_scanline):
        lab, cnt, ov = fn(m.verts, *_arrays(m), 4)
        assert ov
        assert lab[8, 8] == 0           # pixel centre (0.53, 0.53) in both
        assert lab[11, 11] == 1          # only in the second
        assert cnt.sum() == (lab >= 0).sum()


def test_counts_partition():
    m = synth.voronoi_map(40, 3000, seed=5, jitter=0.3)
    lab, cnt, ov = O.labels_scanline(m.verts, *_arrays(m), 8)
    N = 256
    assert cnt.sum() + (lab < 0).sum() == N * N
    # pixel areas approximate shoelace areas
    area = np.abs(O.signed_areas(m.verts, *_arrays(m)))
    np.testing.assert_allclose(cnt / N**2, area, atol=0.004)


def test_holes_even_odd():
    # a ring inside another ring of the same region is a hole (even-odd)
    outer = [(0.1, 0.1), (0.1, 0.9), (0.9, 0.9), (0.9, 0.1)]
    inner = [(0.3, 0.3), (0.3, 0.7), (0.7, 0.7), (0.7, 0.3)]
    v = np.array(outer + inner, np.float64)
    m = synth.Mesh(v, np.array([0, 4, 8], np.int32), np.arange(8, dtype=np.int32),
                   np.array([0, 0], np.int32), 1)
    lab, cnt, ov = O.labels_scanline(v, *_arrays(m), 5)
    lab2, _, _ = O.labels_bruteforce(v, *_arrays(m), 5)
    np.testing.assert_array_equal(lab, lab2)
    assert lab[16, 16] < 0 and lab[4, 16] == 0
