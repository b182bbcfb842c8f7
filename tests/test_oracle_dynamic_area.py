"""Pins of the oracle's dynamic-area background (Sec. 4.3, Eq. (Mb)).

The background value of a time step makes the map cover the area fraction
A_i(t) of the domain once its density is equalised.  Pinned by what that
means, not by the formula: (1) a map that already covers exactly A_i(t) of
the pixels, with values proportional to its regions' pixel counts, gets a
uniform density texture, so the InIm field (Eq. 3) is zero and nothing
moves; (2) a map that covers less than A_i(t) grows toward it, one that
covers more shrinks toward it; (3) at the extreme steps of the selected
interval the fraction is a_min and a_max.
"""
import numpy as np
import pytest

from oracle import inim_oracle as O
from paper_2604_13880_gb300 import synth

K = 6
N = 1 << K


def _arrays(mesh):
    return mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions


def _square_map(side_px):
    """Two regions side by side filling a centred square of side_px pixels,
    edges on pixel boundaries (so the pixel counts are exact)."""
    lo = (N - side_px) // 2
    a, m, b = lo / N, (lo + side_px // 2) / N, (lo + side_px) / N
    return synth.square_map([(a, a, m, b), (m, a, b, b)])


def _map_fraction(xy, mesh):
    return float(np.abs(O.signed_areas(xy, *_arrays(mesh))).sum())


def test_map_at_its_target_fraction_does_not_move():
    # 32 x 32 pixels of 64 x 64: fraction 0.25 = a_min (step 0 holds the
    # smaller global integral); values = c * pixel counts
    mesh = _square_map(32)
    xy = mesh.verts.astype(np.float64)
    lab, cnt, _ = O.labels_scanline(xy, *_arrays(mesh), K)
    assert cnt.sum() == 32 * 32
    c = 3.7
    series = np.stack([c * cnt.astype(np.float64), 2.0 * c * cnt.astype(np.float64)])
    bdv, m_b, a_i = O.background_values(series, K, 0.25, 0.6)
    assert a_i[0] == pytest.approx(0.25, abs=1e-15) and a_i[1] == pytest.approx(0.6, abs=1e-15)
    d, d0, b = O.density(lab, cnt, series[0], bdv_abs=bdv[0])
    assert np.allclose(d, c, rtol=1e-14, atol=0.0)          # one density everywhere
    new, info = O.iterate(xy, _arrays(mesh), series[0], K, shape=0.0, bdv_abs=bdv[0])
    assert np.abs(new - xy).max() <= 1e-9


@pytest.mark.parametrize("step,grows", [(1, True), (0, False)])
def test_map_moves_toward_its_target_fraction(step, grows):
    # the map covers 0.25; step 1 asks for a_max = 0.6 (it must grow), step 0
    # for a_min = 0.1 (it must shrink)
    mesh = _square_map(32)
    xy = mesh.verts.astype(np.float64)
    _, cnt, _ = O.labels_scanline(xy, *_arrays(mesh), K)
    series = np.stack([np.array([1.0, 2.0]), np.array([4.0, 3.0])])
    bdv, m_b, a_i = O.background_values(series, K, 0.1, 0.6)
    target = a_i[step]
    start = _map_fraction(xy, mesh)
    frac = [start]
    for _ in range(12):
        xy, _ = O.iterate(xy, _arrays(mesh), series[step], K, shape=0.0, bdv_abs=bdv[step])
        frac.append(_map_fraction(xy, mesh))
    assert (frac[-1] > start) == grows
    assert abs(frac[-1] - target) < 0.5 * abs(start - target)


def test_extreme_steps_and_degenerate_series():
    rng = np.random.default_rng(5)
    vals = rng.lognormal(0.0, 1.0, (9, 7))
    m = vals.sum(1)
    bdv, m_b, a_i = O.background_values(vals, K, 0.2, 0.9)
    assert a_i[np.argmin(m)] == pytest.approx(0.2) and a_i[np.argmax(m)] == pytest.approx(0.9)
    # the map's share of the total mass is the area fraction
    np.testing.assert_allclose(m / (m + m_b), a_i, rtol=1e-12)
    # the background value is the equalised density (M_i + M_b) / N^2
    np.testing.assert_allclose(bdv, (m + m_b) / (N * N), rtol=1e-12)
    # steps outside the selected interval are clipped to its fractions
    bdv2, _, a2 = O.background_values(vals, K, 0.2, 0.9, t0=2, t1=4)
    assert a2.min() >= 0.2 - 1e-15 and a2.max() <= 0.9 + 1e-15
    # a constant global integral: every step at a_max
    _, _, a3 = O.background_values(np.ones((3, 4)), K, 0.3, 0.8)
    np.testing.assert_array_equal(a3, [0.8, 0.8, 0.8])
    with pytest.raises(ValueError):
        O.background_values(vals, K, 0.9, 0.2)
