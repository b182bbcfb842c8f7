"""Pins of the oracle's iteration as a whole (Sec. 4.1 steps 2-7)."""
import numpy as np
import pytest

from oracle import inim_oracle as O
from paper_2604_13880_gb300 import synth


def _arrays(m):
    return (m.ring_off, m.ring_idx, m.ring_region, m.n_regions)


def test_identity_under_uniform_density():
    # s(v) = c * o(v): every region and the background get density c = d0,
    # so Eq. (3) is the identity and no vertex moves
    m = synth.voronoi_map(20, 800, seed=21)
    k = 6
    _, cnt, _ = O.labels_scanline(m.verts, *_arrays(m), k)
    vals = 2.5 * cnt
    xy = m.verts.copy()
    for _ in range(3):
        xy, info = O.iterate(xy, _arrays(m), vals, k, shape=0.0)
    assert np.abs(xy - m.verts).max() < 1e-12


def test_density_mean_is_d0():
    m = synth.voronoi_map(15, 600, seed=8)
    lab, cnt, _ = O.labels_scanline(m.verts, *_arrays(m), 6)
    vals = synth.lognormal_values(15, seed=3)
    d, d0, bdv = O.density(lab, cnt, vals, 1.0)
    assert abs(d.mean() - d0) < 1e-12 * d0
    for v in range(15):
        assert abs(d[lab == v].sum() - vals[v]) < 1e-9 * vals[v]


def test_errors_decrease_and_no_foldover():
    m = synth.voronoi_map(12, 600, seed=4)
    vals = synth.lognormal_values(12, seed=44)
    k = 7
    xy = m.verts.copy()
    sign0 = np.sign(O.signed_areas(xy, *_arrays(m)))
    errs = []
    for _ in range(30):
        xy, info = O.iterate(xy, _arrays(m), vals, k, shape=0.0)
        a = O.signed_areas(xy, *_arrays(m))
        errs.append(O.cartographic_errors(a, info["desired"]))
        assert (np.sign(a) == sign0).all()
        assert not info["overlap"]
    eps = [e[0] for e in errs]
    assert eps[-1] < 0.5 * eps[0]
    assert len(synth.crossing_segment_pairs(xy, synth.mesh_segments(m))) == 0


def test_total_area_conserved():
    # with BDV = d0 the mean density stays d0, so the map's total area
    # stays close to its start value while regions trade area
    m = synth.voronoi_map(16, 800, seed=6)
    vals = synth.lognormal_values(16, seed=61)
    xy = m.verts.copy()
    a0 = O.signed_areas(xy, *_arrays(m)).sum()
    for _ in range(20):
        xy, _ = O.iterate(xy, _arrays(m), vals, 7, shape=0.5)
    a1 = O.signed_areas(xy, *_arrays(m)).sum()
    assert abs(a1 - a0) / abs(a0) < 0.03
    # shared edges cancel: the sum of region areas is the outline's area
    # (a property of the mesh; checks that the generator shares every edge)


def test_shape_blend_scales_step():
    m = synth.voronoi_map(8, 300, seed=2)
    vals = synth.lognormal_values(8, seed=22)
    x0 = m.verts.copy()
    full, _ = O.iterate(x0, _arrays(m), vals, 6, shape=0.0)
    half, _ = O.iterate(x0, _arrays(m), vals, 6, shape=0.5)
    np.testing.assert_allclose(half - x0, 0.5 * (full - x0), atol=1e-15)


def test_shoelace_and_errors():
    m = synth.square_map([(0.0, 0.0, 1.0, 1.0), (0.25, 0.25, 0.75, 0.5)])
    a = O.signed_areas(m.verts, *_arrays(m))
    np.testing.assert_allclose(np.abs(a), [1.0, 0.125])
    eps, xi = O.cartographic_errors([0.5, 0.25], [0.25, 0.25])
    assert eps == 0.25 and xi == 0.5


def test_stop_rule():
    r = O.StopRule(max_iters=512, xi_stop=0.01, stall_window=3)
    seq = [0.5, 0.4, 0.45, 0.41, 0.42]
    out = [r.update(0.1, x) for x in seq]
    assert out == [False, False, False, False, True]
    r = O.StopRule(max_iters=512, xi_stop=0.01, stall_window=32)
    assert r.update(0.005, 0.009) is True
    r = O.StopRule(max_iters=2, xi_stop=0.0, stall_window=0)
    assert [r.update(1, 1), r.update(1, 1)] == [False, True]


def test_run_direct_vs_cumulative():
    m = synth.voronoi_map(10, 400, seed=3)
    vals = synth.random_walk_values(10, 3, seed=7)
    xd, sd = O.run(m, vals, 6, max_iters=5, xi_stop=0, stall_window=0, mode="direct")
    xc, sc = O.run(m, vals, 6, max_iters=5, xi_stop=0, stall_window=0, mode="cumulative")
    np.testing.assert_array_equal(xd[0], xc[0])           # step 0 is the same solve
    assert np.abs(xd[1] - xc[1]).max() > 0                 # later steps differ
    # a direct step equals a fresh single-step run on that step's values
    x1, _ = O.run(m, vals[1:2], 6, max_iters=5, xi_stop=0, stall_window=0)
    np.testing.assert_array_equal(xd[1], x1[0])


def test_pooled_log_density_closed_forms():
    # uniform density (s proportional to o): log(d / d0) = 0 in every block
    m = synth.voronoi_map(12, 500, seed=4)
    lab, cnt, _ = O.labels_scanline(m.verts, *_arrays(m), 6)
    assert np.abs(O.pooled_log_density(lab, cnt, 3.0 * cnt, 8)).max() < 1e-12
    # two half-plane regions: left density 3 units, right 1 unit, no
    # background -> d0 = 2, blocks are log(3/2) on the left, log(1/2) on the right
    N, pool = 16, 4
    lab = np.zeros((N, N), np.int64)
    lab[:, N // 2:] = 1
    cnt = np.array([N * N // 2, N * N // 2])
    out = O.pooled_log_density(lab, cnt, np.array([3.0, 1.0]) * cnt, pool)
    assert out.shape == (N // pool, N // pool)
    assert np.allclose(out[:, :2], np.log(1.5)) and np.allclose(out[:, 2:], np.log(0.5))
    # a block straddling the boundary averages the logs of its pixels
    out2 = O.pooled_log_density(lab, cnt, np.array([3.0, 1.0]) * cnt, 16)
    assert np.isclose(out2[0, 0], 0.5 * (np.log(1.5) + np.log(0.5)))
    # a region without pixels contributes nothing; the background takes bdv_scale * d0
    lab3 = np.full((N, N), O.BACKGROUND)
    lab3[:8] = 0
    cnt3 = np.array([128, 0])
    out3 = O.pooled_log_density(lab3, cnt3, np.array([5.0, 1.0]), 8, bdv_scale=0.25)
    assert np.allclose(out3[0], 0.0) and np.allclose(out3[1], np.log(0.25))


def test_interpolated_frames_closed_forms():
    # Sec. 5.5 frames: the time steps themselves every f frames, the mean of
    # two steps half-way, a constant series stays constant
    a = np.array([[1.0, 4.0, 0.0], [3.0, 2.0, 8.0], [3.0, 2.0, 8.0]])
    fr = O.interpolate_series(a, 2)
    assert fr.shape == (5, 3)
    np.testing.assert_array_equal(fr[[0, 2, 4]], a)
    np.testing.assert_array_equal(fr[1], [2.0, 3.0, 4.0])
    np.testing.assert_array_equal(fr[3], a[1])
    q = O.interpolate_series(a[:2], 4)
    np.testing.assert_allclose(q[:, 2], [0.0, 2.0, 4.0, 6.0, 8.0], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(O.interpolate_series(a[:1], 10), a[:1])
