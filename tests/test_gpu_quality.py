"""GPU quality measures of Sec. 3.3 (inim_quality) against the oracle of
``oracle/quality.py`` on the same float32 vertices.

Tolerances: adjacency counts and tau exact (integer sets, one division);
per-region shape distortion to 1e-14 relative (the same integers and one
division on both sides; the mean is summed in another order); the relative
position error to 1e-10 relative (double atan2 of the two math libraries and
the summation order).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402
from paper_2604_13880_gb300 import synth  # noqa: E402
from oracle import inim_oracle as O  # noqa: E402
from oracle import quality as Q  # noqa: E402

pytestmark = pytest.mark.gpu


def arrays(mesh):
    return (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)


def oracle_quality(mesh, xy_map, xy_cart, k):
    lm, _, _ = O.labels_scanline(xy_map.astype(np.float64), *arrays(mesh), k)
    lc, _, _ = O.labels_scanline(xy_cart.astype(np.float64), *arrays(mesh), k)
    em, ec = Q.raster_adjacency(lm), Q.raster_adjacency(lc)
    per, mean = Q.shape_distortion(lm, lc, mesh.n_regions)
    bary = [Q.barycenters(x.astype(np.float64), mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
            for x in (xy_map, xy_cart)]
    present = [(lm == v).any() and (lc == v).any() for v in range(mesh.n_regions)]
    return dict(tau=Q.topology_distortion(lm, lc), shape=mean, rel_pos=Q.relative_position_error(*bary),
                adj_map=len(em), adj_cart=len(ec), adj_both=len(em & ec), n_present=int(sum(present))), per


def check(got, gper, want, wper):
    for key in ("adj_map", "adj_cart", "adj_both", "n_present"):
        assert got[key] == want[key], key
    assert got["tau"] == want["tau"]
    np.testing.assert_allclose(gper, wper, rtol=1e-14, atol=0.0)
    assert got["shape"] == pytest.approx(want["shape"], rel=1e-13, abs=1e-15)
    assert got["rel_pos"] == pytest.approx(want["rel_pos"], rel=1e-10, abs=1e-15)


def cartogram(mesh, k, iters, seed):
    m = P.inim_map_create(mesh)
    vals = synth.lognormal_values(mesh.n_regions, seed=seed).astype(np.float32)
    x = torch.as_tensor(mesh.verts_f32(), device="cuda")
    P.inim_iterate(m, x, torch.as_tensor(vals, device="cuda"), P.params(log2_res=k, shape=0.25), iters)
    return m, x


def test_identical_maps_are_undistorted():
    mesh = synth.voronoi_map(30, 1500, seed=71)
    m = P.inim_map_create(mesh)
    got, per = P.inim_quality(m, mesh.verts_f32(), 8)
    want, _ = oracle_quality(mesh, mesh.verts_f32(), mesh.verts_f32(), 8)
    assert got["tau"] == 0.0 and got["shape"] == 0.0 and got["rel_pos"] == 0.0
    assert np.all(per == 0.0)
    assert got["adj_map"] == got["adj_cart"] == got["adj_both"] == want["adj_map"] > 0
    assert got["n_present"] == 30


@pytest.mark.parametrize("k,iters", [(8, 8), (9, 20)])
def test_cartogram_quality_matches_oracle(k, iters):
    mesh = synth.voronoi_map(30, 1500, seed=72)
    m, x = cartogram(mesh, k, iters, seed=73)
    got, per = P.inim_quality(m, x, k)                   # device vertices
    cart = x.cpu().numpy()
    want, wper = oracle_quality(mesh, mesh.verts_f32(), cart, k)
    check(got, per, want, wper)
    assert got["shape"] > 0.0 and got["rel_pos"] > 0.0
    host, hper = P.inim_quality(m, cart, k)              # host vertices: the same
    assert host == got and np.array_equal(hper, per)


def test_quality_paper_scale_map():
    # 200 jittered regions, 50k vertices, 1024^2 (the time-varying workload's map)
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    m = P.inim_map_create(mesh)
    x = torch.as_tensor(mesh.verts_f32(), device="cuda")
    vals = w["values"][-1].astype(np.float32)
    P.inim_iterate(m, x, torch.as_tensor(vals, device="cuda"), P.params(log2_res=10, shape=0.5), 10)
    got, per = P.inim_quality(m, x, 10)
    want, wper = oracle_quality(mesh, mesh.verts_f32(), x.cpu().numpy(), 10)
    check(got, per, want, wper)


def test_rotation_gives_its_angle():
    """A global rotation by theta turns every barycentre vector by theta:
    R = theta / pi (up to the float32 rounding of the vertices); tau and the
    shape distortion follow the oracle on the rotated rasters."""
    mesh = synth.voronoi_map(25, 1200, seed=74)
    theta = 0.3
    base = 0.5 + 0.7 * (mesh.verts - 0.5)                 # inside the disc of radius 0.45
    c, s = np.cos(theta), np.sin(theta)
    rot = 0.5 + (base - 0.5) @ np.array([[c, -s], [s, c]]).T
    xm, xc = base.astype(np.float32), rot.astype(np.float32)
    m = P.inim_map_create(mesh)
    got, per = P.inim_quality(m, xc, 9, xy_map=xm)
    want, wper = oracle_quality(mesh, xm, xc, 9)
    check(got, per, want, wper)
    assert got["rel_pos"] == pytest.approx(theta / np.pi, abs=1e-5)


def test_region_missing_from_a_raster():
    # region 1 lies between pixel centres (no pixel in either raster): it
    # scores 1 and is left out of the mean; region 0 is moved by whole pixels
    mesh = synth.square_map([(0.25, 0.25, 0.5, 0.5), (0.7001, 0.7001, 0.7002, 0.7002)])
    m = P.inim_map_create(mesh)
    moved = mesh.verts.copy()
    moved[:4] += 8.0 / 256
    got, per = P.inim_quality(m, moved.astype(np.float32), 8)
    want, wper = oracle_quality(mesh, mesh.verts_f32(), moved.astype(np.float32), 8)
    check(got, per, want, wper)
    assert per[1] == 1.0 and per[0] == 0.0 and got["n_present"] == 1 and got["shape"] == 0.0
