"""Pins of the quality-measure oracle (Sec. 3.3): closed forms on constructed
maps and label rasters."""
import numpy as np
import pytest

from oracle import quality as Q
from paper_2604_13880_gb300 import synth


def _raster(rects, n=32):
    """Label raster with region v filling rects[v] = (i0, j0, i1, j1) (half-open)."""
    lab = np.full((n, n), -1, np.int64)
    for v, (i0, j0, i1, j1) in enumerate(rects):
        lab[j0:j1, i0:i1] = v
    return lab


def test_identical_maps_have_no_distortion():
    lab = _raster([(2, 2, 10, 12), (10, 2, 20, 12), (2, 12, 20, 25)])
    assert Q.topology_distortion(lab, lab) == 0.0
    per, mean = Q.shape_distortion(lab, lab, 3)
    assert mean == 0.0 and np.all(per == 0.0)
    mesh = synth.square_map([(0.1, 0.1, 0.4, 0.5), (0.4, 0.1, 0.9, 0.5), (0.1, 0.5, 0.9, 0.8)])
    b = Q.barycenters(mesh.verts, mesh.ring_off, mesh.ring_idx, mesh.ring_region, 3)
    assert Q.relative_position_error(b, b) == 0.0


def test_topology_distortion_closed_forms():
    m = _raster([(0, 0, 5, 5), (5, 0, 10, 5)])
    c = _raster([(0, 0, 5, 5), (6, 0, 11, 5)])                  # a one-pixel gap
    assert Q.raster_adjacency(m) == {(0, 1)} and Q.raster_adjacency(c) == set()
    assert Q.topology_distortion(m, c) == 1.0
    # A|B|C in the map, A|C|B in the cartogram: E_m = {AB, BC}, E_c = {AC, BC}
    m3 = _raster([(0, 0, 4, 4), (4, 0, 8, 4), (8, 0, 12, 4)])
    c3 = _raster([(0, 0, 4, 4), (8, 0, 12, 4), (4, 0, 8, 4)])
    assert Q.topology_distortion(m3, c3) == pytest.approx(1.0 - 1.0 / 3.0)
    # diagonal contact is no adjacency (4-neighbours)
    assert Q.raster_adjacency(_raster([(0, 0, 2, 2), (2, 2, 4, 4)])) == set()


def test_shape_distortion_closed_forms():
    m = _raster([(3, 4, 9, 8)])
    moved = _raster([(15, 20, 21, 24)])                           # translated: 0
    assert Q.shape_distortion(m, moved, 1)[1] == 0.0
    big = _raster([(2, 2, 10, 10)])                               # side 8
    small = _raster([(20, 20, 24, 24)])                           # side 4, a quarter of it
    assert Q.shape_distortion(small, big, 1)[1] == pytest.approx(3.0 / 4.0)
    w = _raster([(0, 0, 4, 2)])                                   # 4 x 2 against 2 x 4
    t = _raster([(10, 10, 12, 14)])
    assert Q.shape_distortion(w, t, 1)[1] == pytest.approx((8 + 8 - 2 * 4) / (8 + 8 - 4))
    # a region missing from the cartogram scores 1 and is left out of the mean
    per, mean = Q.shape_distortion(_raster([(0, 0, 2, 2), (4, 4, 6, 6)]), _raster([(0, 0, 2, 2)]), 2)
    assert per[1] == 1.0 and mean == 0.0


def test_barycenters_closed_forms():
    mesh = synth.square_map([(0.2, 0.3, 0.6, 0.5)])
    b = Q.barycenters(mesh.verts, mesh.ring_off, mesh.ring_idx, mesh.ring_region, 1)
    np.testing.assert_allclose(b[0], [0.4, 0.4], atol=1e-15)
    # an L made of two rectangles of one region: the area-weighted centroid
    L = synth.square_map([(0.0, 0.0, 0.4, 0.2), (0.0, 0.2, 0.2, 0.6)], n_regions=1)
    L.ring_region[:] = 0
    b = Q.barycenters(L.verts, L.ring_off, L.ring_idx, L.ring_region, 1)
    a1, c1 = 0.08, np.array([0.2, 0.1])
    a2, c2 = 0.08, np.array([0.1, 0.4])
    np.testing.assert_allclose(b[0], (a1 * c1 + a2 * c2) / (a1 + a2), atol=1e-14)


@pytest.mark.parametrize("theta", [0.1, 1.0, 2.5, -0.7])
def test_relative_position_error_of_a_rotation(theta):
    rng = np.random.default_rng(3)
    bm = rng.uniform(0, 1, (9, 2))
    c, s = np.cos(theta), np.sin(theta)
    rot = np.array([[c, -s], [s, c]])
    bc = (bm - 0.5) @ rot.T + 0.5
    assert Q.relative_position_error(bm, bc) == pytest.approx(abs(theta) / np.pi, rel=1e-12)
    # translation and uniform scaling keep every direction: R = 0
    assert Q.relative_position_error(bm, 2.0 * bm + 0.3) == pytest.approx(0.0, abs=1e-12)


def test_shape_distortion_brute_force_on_tiny_rasters():
    # the minimum over whole-pixel translations of |P sym-diff C| / |P union C|,
    # enumerated with explicit pixel sets on random 8 x 8 rasters
    rng = np.random.default_rng(9)
    for _ in range(6):
        lm = rng.integers(-1, 3, (8, 8))
        lc = rng.integers(-1, 3, (8, 8))
        per, mean = Q.shape_distortion(lm, lc, 3)
        vals = []
        for v in range(3):
            pm = set(zip(*np.nonzero(lm == v)))
            pc = set(zip(*np.nonzero(lc == v)))
            if not pm or not pc:
                assert per[v] == 1.0
                continue
            best = min(len(pm ^ s) / len(pm | s)
                       for dy in range(-8, 9) for dx in range(-8, 9)
                       for s in [{(y + dy, x + dx) for y, x in pc}])
            assert per[v] == pytest.approx(best, rel=1e-15)
            vals.append(best)
        assert mean == pytest.approx(np.mean(vals) if vals else 0.0, rel=1e-15)
