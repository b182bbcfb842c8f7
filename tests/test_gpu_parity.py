"""GPU parity: every step of the CUDA path against the CPU oracle, through the
C ABI, on seeded synthetic inputs.

Tolerances (derived in the design notes):
  labels / counts       bit-exact (integer rule)
  FIX64 integral images bit-exact (integer sums of the quantised texture)
  FP32 integral images  |err| <= 2 * depth * 2^-24 * C, depth = N/8 + 64
                        (a linear bound in the number of additions on any path)
  KAHAN integral images |err| <= 1e-10 * C
  displacement          3e-5 (FP32 sums), 1e-6 (FIX64 / KAHAN)
  one iteration         max |dp| <= 1e-5 of the map extent
  N iterations          max |dp| <= 1e-4 of the map extent, areas <= 1e-4 of the
                        mean region area
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402
from paper_2604_13880_gb300 import synth  # noqa: E402
from oracle import inim_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
EXTENT = 0.9


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def arrays(mesh):
    return (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)


def gpu_raster(m, xy32, k):
    N = 1 << k
    lab = torch.empty((N, N), dtype=torch.int16, device="cuda")
    cnt = torch.empty(m.n_regions + 1, dtype=torch.int32, device="cuda")
    ov = P.inim_raster(m, dev(xy32), k, lab, cnt)
    return lab.cpu().numpy().view(np.uint16).astype(np.int64), cnt.cpu().numpy(), ov


def oracle_raster(mesh, xy32, k):
    lab, cnt, ov = O.labels_scanline(xy32.astype(np.float64), *arrays(mesh), k)
    lab = np.where(lab < 0, mesh.n_regions, lab)
    return lab, cnt, ov


# ---------------------------------------------------------------------------
# A1: rasterisation, bit-exact
# ---------------------------------------------------------------------------
def _raster_cases():
    yield "voronoi32", synth.voronoi_map(32, 2000, seed=1), 8
    yield "voronoi60_jitter", synth.voronoi_map(60, 3000, seed=7, jitter=0.3), 9
    yield "voronoi200_jitter", synth.voronoi_map(200, 50_000, seed=2, jitter=0.3), 10
    m = synth.voronoi_map(25, 1500, seed=11)
    m = m.with_verts((np.floor(m.verts * 256) + 0.5) / 256)      # vertices on pixel centres
    yield "on_centres", m, 8
    yield "overlap", synth.square_map([(0.2, 0.2, 0.6, 0.6), (0.4, 0.4, 0.8, 0.8)]), 8
    outer = [(0.1, 0.1), (0.1, 0.9), (0.9, 0.9), (0.9, 0.1)]
    inner = [(0.3, 0.3), (0.3, 0.7), (0.7, 0.7), (0.7, 0.3)]
    yield "hole", synth.Mesh(np.array(outer + inner, np.float64), np.array([0, 4, 8], np.int32),
                             np.arange(8, dtype=np.int32), np.array([0, 0], np.int32), 1), 8
    # fold-overs: vertex noise of about a tenth of a cell makes neighbouring
    # regions overlap in many rows (pixels inside two or three spans, in every
    # crossing-count class and, at 2048 and 4096, in several 32-pixel windows
    # of one lane)
    for nm, (R, V, seed, k, sd) in {"foldover60_256": (60, 3000, 21, 8, 0.006),
                                    "foldover200_1024": (200, 20_000, 22, 10, 0.002),
                                    "foldover200_1024_big": (200, 50_000, 22, 10, 0.004),
                                    "foldover400_2048": (400, 40_000, 23, 11, 0.0008),
                                    "foldover300_4096": (300, 20_000, 24, 12, 0.0005)}.items():
        m = synth.voronoi_map(R, V, seed=seed, jitter=0.3)
        noise = np.random.default_rng(seed + 100).normal(0.0, sd, m.verts.shape)
        yield nm, m.with_verts(np.clip(m.verts + noise, 0.0, 1.0)), k
    # stacked rectangles: up to ~250 crossings per row (the widest warp
    # class), then more than 256 (the block-per-row path), most pixels inside
    # several rectangles
    for nm, (nr, h0, h1, k) in {"stacked_rects_2048": (200, 0.2, 0.5, 11),
                                "stacked_rects_big_1024": (400, 0.3, 0.6, 10)}.items():
        rng = np.random.default_rng(25 + k)
        lo = rng.uniform(0.0, 0.45, (nr, 2))
        hi = lo + np.stack([rng.uniform(0.02, 0.5, nr), rng.uniform(h0, h1, nr)], 1)
        yield nm, synth.square_map([(a, b, c, d) for (a, b), (c, d) in zip(lo, hi)]), k


@pytest.mark.parametrize("name,mesh,k", list(_raster_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_raster_bit_exact(name, mesh, k):
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    lab, cnt, ov = gpu_raster(m, xy, k)
    olab, ocnt, oov = oracle_raster(mesh, xy, k)
    np.testing.assert_array_equal(lab, olab)
    np.testing.assert_array_equal(cnt[:-1], ocnt)
    assert cnt[-1] == (1 << (2 * k)) - ocnt.sum()
    assert bool(ov) == oov


def test_raster_bit_exact_far_vertices():
    """End points far outside the unit square (a map's own vertices lie in
    [-1, 2], but inim_raster takes any positions): the warps holding such
    edges form the crossing keys in 64-bit fixed point, the others in 32-bit,
    with the same keys."""
    base = synth.voronoi_map(40, 2000, seed=5)
    nb = base.verts.shape[0]
    tri = [(0.2, 0.2), (0.9, 0.5), (0.2, 0.8), (0.5, 0.9), (0.1, 0.61), (0.5, 0.3)]
    mesh = synth.Mesh(np.concatenate([base.verts, np.array(tri, np.float64)]),
                      np.concatenate([base.ring_off, base.ring_off[-1] + np.array([3, 6])]).astype(np.int32),
                      np.concatenate([base.ring_idx, nb + np.arange(6)]).astype(np.int32),
                      np.concatenate([base.ring_region, [0, 1]]).astype(np.int32), base.n_regions)
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    xy[nb + 1] = (700.25, 0.5)          # beyond the 32-bit form's range (512)
    xy[nb + 4] = (-600.5, 0.61)
    for k in (9, 12):
        lab, cnt, ov = gpu_raster(m, xy, k)
        olab, ocnt, oov = oracle_raster(mesh, xy, k)
        np.testing.assert_array_equal(lab, olab)
        np.testing.assert_array_equal(cnt[:-1], ocnt)
        assert bool(ov) == oov


def test_raster_bit_exact_4096():
    w = synth.precision_workload()
    mesh = w["mesh"]
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    lab, cnt, ov = gpu_raster(m, xy, 12)
    olab, ocnt, oov = oracle_raster(mesh, xy, 12)
    np.testing.assert_array_equal(lab, olab)
    np.testing.assert_array_equal(cnt[:-1], ocnt)
    assert not ov and not oov


# ---------------------------------------------------------------------------
# A3: integral images on given textures
# ---------------------------------------------------------------------------
def gpu_inims(d32, k, precision, frac_bits=30):
    N = 1 << k
    dt = torch.float32 if precision == P.INIM_FP32 else (torch.int64 if precision == P.INIM_FIX64 else torch.float64)
    # KAHAN elements are float pairs (hi, lo): allocate as float32 [.., 2]
    if precision == P.INIM_KAHAN:
        S = torch.empty((N, N, 2), dtype=torch.float32, device="cuda")
        T = torch.empty((N, N, 2), dtype=torch.float32, device="cuda")
        A = torch.empty((2 * N - 1, 2), dtype=torch.float32, device="cuda")
        B = torch.empty((2 * N - 1, 2), dtype=torch.float32, device="cuda")
    else:
        S = torch.empty((N, N), dtype=dt, device="cuda")
        T = torch.empty((N, N), dtype=dt, device="cuda")
        A = torch.empty(2 * N - 1, dtype=dt, device="cuda")
        B = torch.empty(2 * N - 1, dtype=dt, device="cuda")
    P.inim_inims(dev(d32), k, precision, frac_bits, S, T, A, B)
    torch.cuda.synchronize()
    out = [x.cpu().numpy() for x in (S, T, A, B)]
    if precision == P.INIM_KAHAN:
        out = [x[..., 0].astype(np.float64) + x[..., 1].astype(np.float64) for x in out]
    return out


def texture(k, seed, sigma=1.0):
    N = 1 << k
    rng = np.random.default_rng(seed)
    return rng.lognormal(0.0, sigma, (N, N)).astype(np.float32)


@pytest.mark.parametrize("k", [8, 9, 10, 11])
def test_inims_fp32(k):
    d = texture(k, 100 + k)
    S, T, A, B = gpu_inims(d, k, P.INIM_FP32)
    I = O.inims(d.astype(np.float64))
    N = 1 << k
    tol = 2 * (N / 8 + 64) * 2.0 ** -24 * I["C"]
    for g, o, nm in ((S, I["a"], "S"), (T, I["at"], "T"), (A, I["A"], "A"), (B, I["B"], "B")):
        err = np.abs(g.astype(np.float64) - o).max()
        assert err <= tol, (nm, err / I["C"])


@pytest.mark.parametrize("k", [8, 10, 12])
def test_inims_fix64_bit_exact(k):
    d = texture(k, 200 + k)
    fb = 30
    q = np.rint(d.astype(np.float64) * 2.0 ** fb).astype(np.int64)
    S, T, A, B = gpu_inims(d, k, P.INIM_FIX64, fb)
    I = O.inims(q)
    np.testing.assert_array_equal(S, I["a"])
    np.testing.assert_array_equal(T, I["at"])
    np.testing.assert_array_equal(A, I["A"])
    np.testing.assert_array_equal(B, I["B"])


@pytest.mark.parametrize("k", [8, 10])
def test_inims_kahan(k):
    d = texture(k, 300 + k, sigma=2.0)
    S, T, A, B = gpu_inims(d, k, P.INIM_KAHAN)
    I = O.inims(d.astype(np.float64))
    tol = 1e-10 * I["C"]
    for g, o, nm in ((S, I["a"], "S"), (T, I["at"], "T"), (A, I["A"], "A"), (B, I["B"], "B")):
        assert np.abs(g - o).max() <= tol, nm


# ---------------------------------------------------------------------------
# A4: Eq. (3) displacement at points; identity at constant density
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tol", [(P.INIM_FP32, 3e-5), (P.INIM_FIX64, 1e-6), (P.INIM_KAHAN, 1e-6)])
def test_displacement(precision, tol):
    k = 8
    d = texture(k, 7)
    pts = np.random.default_rng(8).uniform(0.01, 0.99, (5000, 2)).astype(np.float32)
    out = torch.empty((len(pts), 2), dtype=torch.float32, device="cuda")
    P.inim_displacement(dev(d), k, precision, dev(pts), out)
    torch.cuda.synchronize()
    fx, fy = O.displacement_field(d.astype(np.float64))
    want = np.stack([O.bilinear(fx, pts), O.bilinear(fy, pts)], 1)
    assert np.abs(out.cpu().numpy() - want).max() <= tol


@pytest.mark.parametrize("precision", [P.INIM_FP32, P.INIM_FIX64, P.INIM_KAHAN])
def test_identity_at_constant_density(precision):
    k = 9
    N = 1 << k
    pts = np.random.default_rng(9).uniform(0.0, 1.0, (4000, 2)).astype(np.float32)
    out = torch.empty((len(pts), 2), dtype=torch.float32, device="cuda")
    P.inim_displacement(dev(np.ones((N, N), np.float32)), k, precision, dev(pts), out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy()).max() == 0.0
    P.inim_displacement(dev(np.full((N, N), 3.7, np.float32)), k, precision, dev(pts), out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy()).max() <= 1e-6


def test_identity_mapping_iteration():
    mesh = synth.voronoi_map(20, 800, seed=21)
    k = 8
    xy = mesh.verts_f32()
    _, cnt, _ = O.labels_scanline(xy.astype(np.float64), *arrays(mesh), k)
    vals = (2.5 * cnt).astype(np.float32)
    m = P.inim_map_create(mesh)
    x = dev(xy)
    st, _ = P.inim_iterate(m, x, dev(vals), P.params(log2_res=k, shape=0.0), 5)
    assert np.abs(x.cpu().numpy() - xy).max() == 0.0


# ---------------------------------------------------------------------------
# A5 / A6: one iteration, trajectories, areas, errors
# ---------------------------------------------------------------------------
def test_areas():
    mesh = synth.voronoi_map(50, 4000, seed=5, jitter=0.3)
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    a = torch.empty(mesh.n_regions, dtype=torch.float64, device="cuda")
    P.inim_areas(m, dev(xy), a)
    want = O.signed_areas(xy.astype(np.float64), *arrays(mesh))
    # compensated FP32 sums of exact products: error <= (edges per lane + 2)
    # * 2^-47 * sum over the region's edges of |x_a y_b| + |x_b y_a|
    x = xy.astype(np.float64)
    bound = np.zeros(mesh.n_regions)
    for r in range(mesh.n_rings):
        idx = mesh.ring_idx[mesh.ring_off[r]:mesh.ring_off[r + 1]]
        nxt = np.roll(idx, -1)
        mag = np.abs(x[idx, 0] * x[nxt, 1]) + np.abs(x[nxt, 0] * x[idx, 1])
        bound[mesh.ring_region[r]] += (len(idx) / 32 + 2) * 2.0 ** -47 * mag.sum()
    assert (np.abs(a.cpu().numpy() - want) <= bound + 1e-16).all()


@pytest.mark.parametrize("shape", [0.25, 0.5, 0.75])
def test_one_iteration(shape):
    w = synth.single_step_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    x = dev(xy)
    P.inim_iterate(m, x, dev(vals), P.params(log2_res=k, shape=shape), 1)
    want, _ = O.iterate(xy.astype(np.float64), arrays(mesh), vals.astype(np.float64), k, shape)
    assert np.abs(x.cpu().numpy() - want).max() <= 1e-5 * EXTENT


# degenerate cases of the method: a region whose value is zero (density 0,
# it can only shrink), a single region in a large background, values over
# twelve decades, the smallest texture, a vertex count that is no multiple of
# the block size
def _one_iteration_case(mesh, vals, k, shape, iters=1):
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    x = dev(xy)
    P.inim_iterate(m, x, dev(vals.astype(np.float32)), P.params(log2_res=k, shape=shape), iters)
    want = xy.astype(np.float64)
    for _ in range(iters):
        want, _ = O.iterate(want, arrays(mesh), vals.astype(np.float32).astype(np.float64), k, shape)
    return x.cpu().numpy(), want


def test_zero_valued_region():
    mesh = synth.voronoi_map(30, 1500, seed=61)
    vals = synth.lognormal_values(30, seed=62)
    vals[[3, 17]] = 0.0
    got, want = _one_iteration_case(mesh, vals, 9, 0.0)
    assert np.abs(got - want).max() <= 1e-5 * EXTENT


def test_single_region_in_background():
    mesh = synth.square_map([(0.3, 0.35, 0.55, 0.7)])
    got, want = _one_iteration_case(mesh, np.array([5.0]), 8, 0.25, iters=3)
    assert np.abs(got - want).max() <= 1e-5 * EXTENT
    # one region of any value fills its share of the mass: with bdv = d0 it
    # already has the mean density, so nothing moves
    assert np.abs(got - mesh.verts).max() <= 1e-6


def test_values_over_twelve_decades_at_smallest_texture():
    mesh = synth.voronoi_map(25, 1233, seed=63)          # 1233: no multiple of 256 vertices
    vals = 10.0 ** np.random.default_rng(64).uniform(-6, 6, 25)
    got, want = _one_iteration_case(mesh, vals, 8, 0.5)
    assert mesh.n_verts % 256 != 0
    assert np.abs(got - want).max() <= 1e-5 * EXTENT


def test_one_iteration_config_timevarying():
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    xy = mesh.verts_f32()
    x = dev(xy)
    P.inim_iterate(m, x, dev(vals), P.params(log2_res=k, shape=0.5), 1)
    want, _ = O.iterate(xy.astype(np.float64), arrays(mesh), vals.astype(np.float64), k, 0.5)
    assert np.abs(x.cpu().numpy() - want).max() <= 1e-5 * EXTENT


def test_trajectory_single_step_config():
    """20 iterations, shape 0.5 (the single-step workload): vertices, areas,
    and bit-exact labels of the GPU's own vertices at every iteration."""
    w = synth.single_step_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    xy0 = mesh.verts_f32()
    x = dev(xy0)
    ora = xy0.astype(np.float64)
    t0 = O.transform_uniform(1 << k)
    p = P.params(log2_res=k, shape=0.5)
    for it in range(w["iters"]):
        g = x.cpu().numpy()
        lab, cnt, _ = gpu_raster(m, g, k)
        olab, ocnt, _ = oracle_raster(mesh, g, k)
        np.testing.assert_array_equal(lab, olab)
        P.inim_iterate(m, x, dev(vals), p, 1)
        ora, _ = O.iterate(ora, arrays(mesh), vals.astype(np.float64), k, 0.5, t0=t0)
    g = x.cpu().numpy()
    dp = np.abs(g - ora).max()
    assert dp <= 1e-4 * EXTENT, dp
    ga = O.signed_areas(g.astype(np.float64), *arrays(mesh))
    oa = O.signed_areas(ora, *arrays(mesh))
    # area errors relative to the mean region area: a region's area moves by at
    # most (its perimeter) x (vertex error), so a bound relative to its own area
    # would be tighter than the vertex bound for small regions
    rel = np.abs(ga - oa).max() / np.abs(oa).mean()
    assert rel <= 1e-4, (rel, dp)


@pytest.mark.parametrize("precision", [P.INIM_FIX64, P.INIM_KAHAN])
def test_precision_variants_trajectory(precision):
    w = synth.single_step_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    x = dev(mesh.verts_f32())
    P.inim_iterate(m, x, dev(vals), P.params(log2_res=k, shape=0.5, precision=precision), 20)
    ora, _ = O.run(mesh.with_verts(mesh.verts_f32().astype(np.float64)), vals[None].astype(np.float64), k,
                   shape=0.5, max_iters=20, xi_stop=0, stall_window=0)
    assert np.abs(x.cpu().numpy() - ora[0]).max() <= 1e-4 * EXTENT


def test_plain_form_matches_fused():
    w = synth.single_step_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    a = dev(mesh.verts_f32())
    b = dev(mesh.verts_f32())
    P.inim_iterate(m, a, dev(vals), P.params(log2_res=k, shape=0.5), 10)
    P.inim_iterate(m, b, dev(vals), P.params(log2_res=k, shape=0.5, form=P.INIM_FORM_PLAIN), 10)
    assert (a - b).abs().max().item() <= 1e-5


# ---------------------------------------------------------------------------
# A7 / A8: time loop (direct, cumulative), batches, the stop rule
# ---------------------------------------------------------------------------
def test_direct_steps_are_independent_solves():
    mesh = synth.voronoi_map(30, 1500, seed=31)
    vals = synth.random_walk_values(30, 3, seed=32).astype(np.float32)
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.5, max_iters=12, xi_stop=0.0, stall_window=0)
    out, stats, _ = P.inim_run(m, vals, p)
    for t in range(3):
        one, _, _ = P.inim_run(m, vals[t:t + 1], p)
        np.testing.assert_array_equal(out[t], one[0])
        assert stats[t]["iters"] == 12


def test_cumulative_matches_oracle():
    mesh = synth.voronoi_map(30, 1500, seed=33)
    vals = synth.random_walk_values(30, 3, seed=34).astype(np.float32)
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.25, max_iters=6, xi_stop=0.0, stall_window=0, mode=P.INIM_CUMULATIVE)
    out, stats, _ = P.inim_run(m, vals, p)
    ora, _ = O.run(mesh.with_verts(mesh.verts_f32().astype(np.float64)), vals.astype(np.float64), 8,
                   shape=0.25, max_iters=6, xi_stop=0, stall_window=0, mode="cumulative")
    assert np.abs(out - ora).max() <= 1e-4 * EXTENT
    d, _, _ = P.inim_run(m, vals[:1], P.params(log2_res=8, shape=0.25, max_iters=6, xi_stop=0.0, stall_window=0))
    np.testing.assert_array_equal(out[0], d[0])


def test_batch_mixed_resolutions_equals_single_runs():
    meshes = [synth.voronoi_map(20 + 10 * b, 1000 + 500 * b, seed=40 + b) for b in range(4)]
    ks = [8, 9, 10, 8]
    maps = [P.inim_map_create(mm) for mm in meshes]
    jobs = []
    for b, mm in enumerate(meshes):
        vals = synth.lognormal_values(mm.n_regions, seed=50 + b).astype(np.float32)
        jobs.append(dict(map=maps[b], values=vals,
                         params=P.params(log2_res=ks[b], shape=0.5, max_iters=10 + 3 * b, xi_stop=0.0,
                                         stall_window=0)))
    outs, stats, _ = P.inim_run_batch(jobs)
    for b, j in enumerate(jobs):
        one, st, _ = P.inim_run(j["map"], j["values"][None], j["params"])
        np.testing.assert_array_equal(outs[b], one[0])
        assert stats[b]["iters"] == 10 + 3 * b


def test_overlapped_graph_equals_sequential_graph():
    # a fixed-length batch runs its area kernels next to the next iteration's
    # raster (the default) or after the move: vertices and the reported errors
    # must be identical
    w = synth.time_varying_workload()
    mesh, vals = w["mesh"], w["values"].astype(np.float32)
    m = P.inim_map_create(mesh)
    res = []
    try:
        for ov in (True, False):
            P.inim_set_area_overlap(ov)
            jobs = [dict(map=m, values=vals[t], params=P.params(log2_res=10, shape=sh, max_iters=19, xi_stop=0.0,
                                                                stall_window=0))
                    for t, sh in ((0, 0.25), (5, 0.5), (11, 0.75))]
            res.append(P.inim_run_batch(jobs))
    finally:
        P.inim_set_area_overlap(True)
    for b in range(3):
        np.testing.assert_array_equal(res[0][0][b], res[1][0][b])
        for key in ("iters", "eps", "xi", "foldover", "overlap"):
            assert res[0][1][b][key] == res[1][1][b][key], (b, key)


def _stop_rule_runs(run):
    """run() with the area kernel overlapped and in sequence"""
    out = []
    try:
        for ov in (True, False):
            P.inim_set_area_overlap(ov)
            out.append(run())
    finally:
        P.inim_set_area_overlap(True)
    return out


def test_stop_rule_with_overlapped_area_kernel():
    # With a stop rule the raster and scan after the stopping iteration start
    # before the area kernel has stopped the job; the move after them must see
    # the stop: the same vertices, iteration counts and errors as in sequence,
    # and as a fixed run of the stopping iteration's length.  A batch whose
    # jobs stop at different iterations (eps target, xi stall rule, cap).
    mesh = synth.voronoi_map(40, 2500, seed=71, jitter=0.3)
    m = P.inim_map_create(mesh)
    vals = [synth.lognormal_values(40, seed=72 + t).astype(np.float32) for t in range(3)]
    prm = [dict(eps_stop=0.25, xi_stop=0.0, stall_window=0, max_iters=200),
           dict(eps_stop=0.0, xi_stop=0.0, stall_window=6, max_iters=200),
           dict(eps_stop=0.0, xi_stop=0.0, stall_window=0, max_iters=23)]

    def run():
        jobs = [dict(map=m, values=vals[t], params=P.params(log2_res=9, shape=0.5, **prm[t])) for t in range(3)]
        return P.inim_run_batch(jobs)

    (o_ov, s_ov, _), (o_sq, s_sq, _) = _stop_rule_runs(run)
    for t in range(3):
        np.testing.assert_array_equal(o_ov[t], o_sq[t], err_msg=str(t))
        for key in ("iters", "eps", "xi", "foldover"):
            assert s_ov[t][key] == s_sq[t][key], (t, key, s_ov[t][key], s_sq[t][key])
        assert 1 <= s_ov[t]["iters"] <= 200, s_ov[t]
        # a fixed run of exactly that many iterations ends at the same vertices
        n = s_ov[t]["iters"]
        fx, fs, _ = P.inim_run(m, vals[t][None], P.params(log2_res=9, shape=0.5, max_iters=n, xi_stop=0.0,
                                                           stall_window=0))
        np.testing.assert_array_equal(o_ov[t], fx[0], err_msg=str(t))
        assert fs[0]["iters"] == n and fs[0]["eps"] == s_ov[t]["eps"]
    assert s_ov[0]["iters"] < 200 and s_ov[0]["eps"] < 0.25 and s_ov[2]["iters"] == 23


def test_cumulative_stop_rule_with_overlapped_area_kernel():
    # a cumulative series with the stop rule, round by round: each step's
    # vertices and counts as in sequence
    mesh = synth.voronoi_map(30, 1500, seed=81)
    vals = synth.random_walk_values(30, 4, seed=82).astype(np.float32)
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.25, max_iters=120, xi_stop=0.02, stall_window=8, mode=P.INIM_CUMULATIVE)
    (o_ov, s_ov, _), (o_sq, s_sq, _) = _stop_rule_runs(lambda: P.inim_run(m, vals, p))
    np.testing.assert_array_equal(o_ov, o_sq)
    for t in range(4):
        for key in ("iters", "eps", "xi", "foldover"):
            assert s_ov[t][key] == s_sq[t][key], (t, key)


def test_stop_rule_reports_consistent_errors():
    w = synth.single_step_workload()
    mesh = w["mesh"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    out, stats, status = P.inim_run(m, vals[None], P.params(log2_res=8, shape=0.0))
    s = stats[0]
    assert 1 <= s["iters"] <= 512
    assert s["iters"] == 512 or s["xi"] < 0.01 or s["iters"] >= 33
    # the reported errors are the errors of the returned vertices
    g = out[0].astype(np.float64)
    _, cnt, _ = O.labels_scanline(g, *arrays(mesh), 8)
    areas = O.signed_areas(g, *arrays(mesh))
    d0 = vals[cnt > 0].astype(np.float64).sum() / cnt.sum()
    desired = O.desired_areas(vals.astype(np.float64), cnt, d0, 256)
    eps, xi = O.cartographic_errors(areas, desired)
    assert abs(eps - s["eps"]) <= 2e-3 and abs(xi - s["xi"]) <= 5e-3
    assert s["foldover"] == 0 and s["overlap"] == 0


# ---------------------------------------------------------------------------
# A8: scan tiles and the autotuner
# ---------------------------------------------------------------------------
TILES_1024 = ([(h, c, t) for h in (4, 8, 16, 32, 64) for (c, t) in ((8, 128), (4, 256), (16, 64), (32, 32))]
              + [(8, 0, 256), (16, 0, 256)])          # cols_per_thread 0: the parallel-rows band scan


@pytest.mark.parametrize("tile", TILES_1024)
def test_every_scan_tile_is_exact_in_fixed_point(tile):
    k = 10
    d = texture(k, 77)
    q = np.rint(d.astype(np.float64) * 2.0 ** 30).astype(np.int64)
    I = O.inims(q)
    try:
        P.inim_set_scan_tile(k, P.INIM_FIX64, 0, *tile)
        S, T, A, B = gpu_inims(d, k, P.INIM_FIX64, 30)
    finally:
        P.inim_set_scan_tile(k, P.INIM_FIX64, 0, 0, 0, 0)
    np.testing.assert_array_equal(S, I["a"])
    np.testing.assert_array_equal(T, I["at"])
    np.testing.assert_array_equal(A, I["A"])
    np.testing.assert_array_equal(B, I["B"])


@pytest.mark.parametrize("H", [8, 16])
@pytest.mark.parametrize("precision", [P.INIM_FIX64, P.INIM_KAHAN, P.INIM_FP32])
def test_parallel_rows_tiles_at_512(H, precision):
    # the parallel-rows band scan at N = 512 (two columns a thread in its
    # second stage, 8-byte windows for four-byte sums): exact in fixed point,
    # within the bounds of the other precisions
    k = 9
    d = texture(k, 78)
    try:
        P.inim_set_scan_tile(k, precision, 0, H, 0, 256)
        got = gpu_inims(d, k, precision, 30)
    finally:
        P.inim_set_scan_tile(k, precision, 0, 0, 0, 0)
    if precision == P.INIM_FIX64:
        I = O.inims(np.rint(d.astype(np.float64) * 2.0 ** 30).astype(np.int64))
        for g, o in zip(got, (I["a"], I["at"], I["A"], I["B"])):
            np.testing.assert_array_equal(g, o)
        return
    I = O.inims(d.astype(np.float64))
    N = 1 << k
    tol = (2 * (N / 8 + 64) * 2.0 ** -24 if precision == P.INIM_FP32 else 1e-10) * I["C"]
    for g, o in zip(got, (I["a"], I["at"], I["A"], I["B"])):
        assert np.abs(g.astype(np.float64) - o).max() <= tol


def test_every_scan_tile_gives_identical_iterations_in_fixed_point():
    # the label path (rows staged by bulk copies) in every tile: the 64-bit
    # tables are exact, so the moved vertices must not depend on the tile
    w = synth.time_varying_workload()
    mesh, vals = w["mesh"], w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    ref = None
    for tile in TILES_1024:
        for large in (0, 1):
            P.inim_set_scan_tile(10, P.INIM_FIX64, large, *tile)
        try:
            x = dev(mesh.verts_f32())
            P.inim_iterate(m, x, dev(vals), P.params(log2_res=10, shape=0.5, precision=P.INIM_FIX64), 2)
            got = x.cpu().numpy()
        finally:
            for large in (0, 1):
                P.inim_set_scan_tile(10, P.INIM_FIX64, large, 0, 0, 0)
        if ref is None:
            ref = got
        np.testing.assert_array_equal(got, ref, err_msg=str(tile))


def test_autotuner_picks_a_valid_tile_and_stays_on_the_oracle():
    w = synth.single_step_workload()
    mesh = w["mesh"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.5, max_iters=5, xi_stop=0.0, stall_window=0)
    arr = (P.inim_job * 4)()
    for q in range(4):
        arr[q].map = m.handle
        arr[q].values = vals.ctypes.data
        arr[q].params = p
    try:
        P.inim_autotune_scan(arr, reps=3)
        t = P.inim_get_scan_tile(8, P.INIM_FP32, 0)
        assert t["band_rows"] in (4, 8, 16, 32, 64) and t["cols_per_thread"] * t["threads"] == 256
        out, _, _ = P.inim_run(m, vals[None], p)
    finally:
        P.inim_set_scan_tile(8, P.INIM_FP32, 0, 0, 0, 0)
    ora, _ = O.run(mesh.with_verts(mesh.verts_f32().astype(np.float64)), vals[None].astype(np.float64), 8,
                   shape=0.5, max_iters=5, xi_stop=0, stall_window=0)
    assert np.abs(out[0] - ora[0]).max() <= 1e-4 * EXTENT


# ---------------------------------------------------------------------------
# A7 / A8: time series in one call; the persistent launch vs the graph path
# ---------------------------------------------------------------------------
def _series_case():
    mesh = synth.voronoi_map(40, 2500, seed=71, jitter=0.3)
    vals = synth.random_walk_values(40, 3, seed=72).astype(np.float32)
    return mesh, vals


def test_series_persistent_and_graph_paths_agree_with_oracle():
    mesh, vals = _series_case()
    m = P.inim_map_create(mesh)
    pd = P.params(log2_res=9, shape=0.5, max_iters=8, xi_stop=0.0, stall_window=0, mode=P.INIM_DIRECT)
    pc = P.params(log2_res=9, shape=0.25, max_iters=6, xi_stop=0.0, stall_window=0, mode=P.INIM_CUMULATIVE)
    series = [dict(map=m, values=vals[:2], params=pd), dict(map=m, values=vals, params=pc)]
    graph, gstats, _ = P.inim_run_series(series)          # per-step kernels under CUDA graphs
    try:
        P.inim_set_persistent(True)
        pers, pstats, _ = P.inim_run_series(series)       # one persistent launch per batch
    finally:
        P.inim_set_persistent(False)
    base = mesh.with_verts(mesh.verts_f32().astype(np.float64))
    od, _ = O.run(base, vals[:2].astype(np.float64), 9, shape=0.5, max_iters=8, xi_stop=0, stall_window=0)
    oc, _ = O.run(base, vals.astype(np.float64), 9, shape=0.25, max_iters=6, xi_stop=0, stall_window=0,
                  mode="cumulative")
    for got in (graph, pers):
        assert np.abs(got[0] - od).max() <= 1e-4 * EXTENT
        assert np.abs(got[1] - oc).max() <= 1e-4 * EXTENT
    # the two paths scan with different tiles (parallel-rows vs row-serial),
    # so their FP32 InIms round differently: each within the FP32 bound
    # 2 (N/8 + 64) 2^-24 C of the exact sums (test_inims_fp32), 1.5e-5 C at
    # N = 512; the cumulative trajectories may differ by the two bounds
    N = 1 << 9
    assert np.abs(graph[1] - pers[1]).max() <= 2 * 2 * (N / 8 + 64) * 2.0 ** -24 * EXTENT
    assert [s["iters"] for s in pstats[1]] == [6, 6, 6] and [s["iters"] for s in gstats[1]] == [6, 6, 6]


def test_cumulative_series_with_stop_rule_on_device():
    """Every time step stops by its own rule inside one persistent launch; the
    per-step statistics come back per step."""
    mesh, vals = _series_case()
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.0, max_iters=200, xi_stop=0.0, stall_window=0, eps_stop=0.08,
                 mode=P.INIM_CUMULATIVE)
    try:
        P.inim_set_persistent(True)
        out, stats, _ = P.inim_run(m, vals, p)
    finally:
        P.inim_set_persistent(False)
    gout, gstats, _ = P.inim_run(m, vals, p)           # the same series round by round
    # same stop decisions; vertices within the N-iteration bound (the two paths
    # tile the FP32 scan differently, hence round differently)
    assert [s["iters"] for s in gstats] == [s["iters"] for s in stats]
    assert np.abs(gout - out).max() <= 1e-4 * EXTENT
    for t, s in enumerate(stats):
        assert s["iters"] == 200 or s["eps"] < 0.08, (t, s)
    # the last step's reported eps is the error of its returned vertices
    g = out[-1].astype(np.float64)
    _, cnt, _ = O.labels_scanline(g, *arrays(mesh), 8)
    v = vals[-1].astype(np.float64)
    d0 = v[cnt > 0].sum() / cnt.sum()
    eps, _ = O.cartographic_errors(O.signed_areas(g, *arrays(mesh)), O.desired_areas(v, cnt, d0, 256))
    assert abs(eps - stats[-1]["eps"]) <= 2e-3


# ---------------------------------------------------------------------------
# A11: dynamic-area background value (Sec. 4.3, Eq. (Mb))
# ---------------------------------------------------------------------------
def test_dynamic_area_direct_series_matches_oracle():
    """Each step's background value from Eq. (Mb) (host), passed per solve as
    bdv_value: the batch of direct steps follows the oracle's run with the
    same area fractions (N-iteration bound), and one iteration through the
    single-step call stays within the one-iteration bound."""
    mesh = synth.voronoi_map(30, 1500, seed=35)
    vals = synth.random_walk_values(30, 3, seed=36).astype(np.float32)
    a_min, a_max, iters = 0.45, 0.65, 4
    bdv, frac = P.inim_background_values(vals, 8, a_min, a_max)
    m = P.inim_map_create(mesh)
    base = mesh.verts_f32().astype(np.float64)

    def prm(t, it):
        return P.params(log2_res=8, shape=0.25, max_iters=it, xi_stop=0.0, stall_window=0,
                        bdv_value=float(bdv[t]))

    outs, stats, _ = P.inim_run_batch([dict(map=m, values=vals[t], params=prm(t, iters)) for t in range(3)])
    ora, ostats = O.run(mesh.with_verts(base), vals.astype(np.float64), 8, shape=0.25, max_iters=iters,
                        xi_stop=0, stall_window=0, area_fractions=(a_min, a_max))
    for t in range(3):
        assert stats[t]["iters"] == iters
        assert np.abs(outs[t] - ora[t]).max() <= 1e-4 * EXTENT, t
        assert abs(stats[t]["eps"] - ostats[t]["eps"]) <= 2e-3 and abs(stats[t]["xi"] - ostats[t]["xi"]) <= 2e-3
    # the background value changes the solution: the default background differs
    plain, _, _ = P.inim_run_batch([dict(map=m, values=vals[2], params=P.params(
        log2_res=8, shape=0.25, max_iters=iters, xi_stop=0.0, stall_window=0))])
    assert np.abs(plain[0] - outs[2]).max() > 1e-3
    x = dev(mesh.verts_f32())
    P.inim_iterate(m, x, dev(vals[1]), prm(1, 1), 1)
    want, _ = O.iterate(base, arrays(mesh), vals[1].astype(np.float64), 8, 0.25,
                        bdv_abs=float(np.float32(bdv[1])))
    assert np.abs(x.cpu().numpy() - want).max() <= 1e-5 * EXTENT


def test_dynamic_area_map_at_its_target_fraction_does_not_move():
    """A map covering exactly the target fraction with values proportional to
    its pixel counts has one density everywhere once the background value is
    the equalised density: the InIm field is zero and no vertex moves."""
    lo, side = 64, 128                                  # 128^2 of 256^2 pixels: fraction 1/4
    a, mid, b = lo / 256, (lo + side // 2) / 256, (lo + side) / 256
    mesh = synth.square_map([(a, a, mid, b), (mid, a, b, b)])
    _, cnt, _ = O.labels_scanline(mesh.verts.astype(np.float64), *arrays(mesh), 8)
    assert cnt.sum() == side * side
    c = 3.5
    vals = (c * cnt).astype(np.float32)
    m = P.inim_map_create(mesh)
    x = dev(mesh.verts_f32())
    P.inim_iterate(m, x, dev(vals), P.params(log2_res=8, shape=0.0, bdv_value=c), 3)
    assert np.abs(x.cpu().numpy() - mesh.verts).max() <= 1e-6


# ---------------------------------------------------------------------------
# A9: precision study at 4096^2 (values over six decades), a few iterations
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_precision_variants_at_4096_against_fp64_oracle():
    w = synth.precision_workload()
    mesh = w["mesh"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    K = 3
    xy0 = mesh.verts_f32()
    ora = xy0.astype(np.float64)
    t0 = O.transform_uniform(4096)
    for _ in range(K):
        ora, _ = O.iterate(ora, arrays(mesh), vals.astype(np.float64), 12, 0.5, t0=t0)
    err = {}
    for name, prec in (("fp32", P.INIM_FP32), ("fix64", P.INIM_FIX64), ("kahan", P.INIM_KAHAN)):
        x = dev(xy0)
        P.inim_iterate(m, x, dev(vals), P.params(log2_res=12, shape=0.5, precision=prec), K)
        err[name] = np.abs(x.cpu().numpy() - ora).max()
    assert max(err.values()) <= 1e-5 * EXTENT, err           # the one-iteration bound, K = 3
    assert err["fix64"] <= err["fp32"] + 1e-7 and err["kahan"] <= err["fp32"] + 1e-7, err
