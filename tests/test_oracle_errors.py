"""Pins of the oracle's error denominators and of Eq. (Mb) by hand-worked cases.

desired_areas is the w(v) of the cartographic errors (Sec. 3.3) under the
reading w(v) = s(v) / M, with M = sum_{o(v)>0} s(v) + BDV * o_bg the total
mass of the density texture (equalised density: area proportional to mass).
The expected numbers below are worked out by hand in the comments, so a
dropped background term, a sum over every region instead of the regions
with pixels, or a wrong background pixel count fails.

background_values is Eq. (Mb) of Sec. 4.3 (its reading is stated in the
oracle): the values here are worked by hand at steps where the map is away
from its target area fraction.
"""
import numpy as np
import pytest

from oracle import inim_oracle as O
from paper_2604_13880_gb300 import synth


def test_desired_areas_hand_worked():
    # N = 4: 16 pixels.  Three regions, s = (2, 3, 5), o = (4, 6, 0): region 2
    # has no pixel.  Background pixels o_bg = 16 - 10 = 6.
    # d0 = (2 + 3) / (4 + 6) = 0.5 (regions with pixels only), BDV = 1 * d0.
    # M = 2 + 3 + 0.5 * 6 = 8, so w = (2/8, 3/8, 5/8) = (0.25, 0.375, 0.625).
    values = [2.0, 3.0, 5.0]
    counts = [4, 6, 0]
    labels = np.array([[0, 0, 1, 1],
                       [0, 0, 1, 1],
                       [-1, -1, 1, 1],
                       [-1, -1, -1, -1]])
    d, d0, bdv = O.density(labels, counts, values)
    assert d0 == 0.5 and bdv == 0.5
    w = O.desired_areas(values, counts, bdv, 4)
    np.testing.assert_array_equal(w, [0.25, 0.375, 0.625])
    # the total mass M is the sum of the density texture: w = s / sum(d)
    np.testing.assert_allclose(np.asarray(values) / d.sum(), w, rtol=0, atol=1e-15)


def test_desired_areas_with_scaled_background():
    # same raster, BDV = 2 d0 = 1: M = 5 + 1 * 6 = 11, w = (2, 3, 5) / 11
    w = O.desired_areas([2.0, 3.0, 5.0], [4, 6, 0], 1.0, 4)
    np.testing.assert_allclose(w, [2 / 11, 3 / 11, 5 / 11], rtol=1e-15)
    # no background pixel at all (16 region pixels): M = sum of the values
    w = O.desired_areas([1.0, 3.0], [8, 8], 123.0, 4)
    np.testing.assert_array_equal(w, [0.25, 0.75])


def test_cartographic_errors_hand_worked():
    # e(v) = |o - w| / max(o, w): (0.1 - 0.2)/0.2 = 0.5, (0.3 - 0.3) = 0,
    # (0.4 - 0.1)/0.4 = 0.75, and a region with o = w = 0 counts 0
    eps, xi = O.cartographic_errors([0.1, -0.3, 0.4, 0.0], [0.2, 0.3, 0.1, 0.0])
    assert xi == pytest.approx(0.75, abs=1e-15)
    assert eps == pytest.approx((0.5 + 0.0 + 0.75 + 0.0) / 4, abs=1e-15)


def test_background_values_hand_worked_away_from_target():
    # global integrals M_i = (10, 20, 30) over t = 0..2, selected interval the
    # whole series: w = (0, 0.5, 1); a_min = 0.25, a_max = 0.5 give
    # A = (0.25, 0.375, 0.5);  M_b = M_i (1 - A) / A = (30, 100/3, 30);
    # N = 4: BDV = M_b / ((1 - A) N^2) = (30/12, (100/3)/10, 30/8)
    #                                  = (2.5, 10/3, 3.75).
    vals = np.array([[4.0, 6.0], [5.0, 15.0], [10.0, 20.0]])
    bdv, m_b, a_i = O.background_values(vals, 2, 0.25, 0.5)
    np.testing.assert_allclose(a_i, [0.25, 0.375, 0.5], rtol=1e-15)
    np.testing.assert_allclose(m_b, [30.0, 100.0 / 3.0, 30.0], rtol=1e-15)
    np.testing.assert_allclose(bdv, [2.5, 10.0 / 3.0, 3.75], rtol=1e-15)
    # a sub-interval [1, 2]: w = (-1 -> clipped 0, 0, 1), A = (0.25, 0.25, 0.5)
    bdv, m_b, a_i = O.background_values(vals, 2, 0.25, 0.5, t0=1, t1=2)
    np.testing.assert_allclose(a_i, [0.25, 0.25, 0.5], rtol=1e-15)
    np.testing.assert_allclose(m_b, [30.0, 60.0, 30.0], rtol=1e-15)
    np.testing.assert_allclose(bdv, [2.5, 5.0, 3.75], rtol=1e-15)


def test_background_density_of_a_map_away_from_its_target():
    # A centred square of 16 x 16 pixels of a 32^2 texture covers 1/4 of it;
    # the target fraction of step 1 is 1/2 (a_max, the larger integral).
    # Its background value divides M_b by the pixels the target leaves,
    # (1 - 1/2) N^2 = 512, not by the 768 background pixels of the current
    # raster.  Values (64, 192): M_i = 256, M_b = 256, BDV = 256 / 512 = 0.5.
    N, K = 32, 5
    m = synth.square_map([(0.25, 0.25, 0.5, 0.75), (0.5, 0.25, 0.75, 0.75)])
    vals = np.array([[32.0, 96.0], [64.0, 192.0]])
    bdv, m_b, a_i = O.background_values(vals, K, 0.25, 0.5)
    assert a_i[1] == 0.5 and m_b[1] == 256.0 and bdv[1] == 0.5
    arrays = (m.ring_off, m.ring_idx, m.ring_region, m.n_regions)
    _, info = O.iterate(m.verts, arrays, vals[1], K, 0.5, bdv_abs=bdv[1])
    assert info["counts"].tolist() == [128, 128]
    d, _, _ = O.density(info["labels"], info["counts"], vals[1], bdv_abs=bdv[1])
    assert np.all(d[info["labels"] < 0] == 0.5)
    # total mass of the texture: 256 + 0.5 * 768 = 640, so w = (64, 192) / 640
    np.testing.assert_allclose(info["desired"], [0.1, 0.3], rtol=1e-15)
    assert N * N - 256 == 768
