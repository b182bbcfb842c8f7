"""GPU parity at the benchmark's full size and launch configuration.

The time-varying sweep -- 200 jittered regions, ~50k vertices, 1024^2, 24
time steps, shapes {0.25, 0.5, 0.75}, direct (72 solves in one batch) and
cumulative (3 series advanced together) -- runs through one inim_run_series
call with the scan tiles of the benchmark's profiled launch (72-solve batch:
16-row bands, 4 columns x 256 threads; 3-solve batch: 8-row bands in the
parallel-rows form).  The oracle cannot follow its 7200 iterations, so
sampled solves are checked: the first iterations of three solves against the
oracle (N-iteration bound), and after the benchmark's 50 iterations what
holds at any size (labels of the returned vertices bit-exact; the reported
error equal to the error of the returned vertices).  The file runs last: its
solves are the largest of the GPU suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402
from paper_2604_13880_gb300 import synth  # noqa: E402
from oracle import inim_oracle as O  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
EXTENT = 0.9
SHAPES = (0.25, 0.5, 0.75)
K = 10


@pytest.fixture(scope="module")
def sweep_setup():
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    vals = np.ascontiguousarray(w["values"].astype(np.float32))         # [24, 200]
    m = P.inim_map_create(mesh)
    P.inim_set_scan_tile(K, P.INIM_FP32, 1, 16, 4, 256)
    P.inim_set_scan_tile(K, P.INIM_FP32, 0, 8, 0, 256)
    yield mesh, vals, m
    P.inim_set_scan_tile(K, P.INIM_FP32, 1, 0, 0, 0)                    # back to the defaults
    P.inim_set_scan_tile(K, P.INIM_FP32, 0, 0, 0, 0)


def arrays(mesh):
    return (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)


def run_sweep(m, vals, iters):
    """3 direct and 3 cumulative series (one per shape) in one call, as the
    benchmark's step; returns outputs and statistics in that order."""
    series = [dict(map=m, values=vals, params=P.params(log2_res=K, shape=sh, max_iters=iters, xi_stop=0.0,
                                                       stall_window=0, mode=mode))
              for mode in (P.INIM_DIRECT, P.INIM_CUMULATIVE) for sh in SHAPES]
    outs, stats, _ = P.inim_run_series(series)
    return outs, stats


def test_first_iterations_of_sampled_solves_match_the_oracle(sweep_setup):
    mesh, vals, m = sweep_setup
    iters = 3
    outs, stats = run_sweep(m, vals, iters)
    base = mesh.with_verts(mesh.verts_f32().astype(np.float64))
    # direct: shape 0.25 at step 0, shape 0.75 at step 23
    for s, t in ((0, 0), (2, 23)):
        ora, _ = O.run(base, vals[t:t + 1].astype(np.float64), K, shape=SHAPES[s], max_iters=iters, xi_stop=0,
                       stall_window=0)
        assert stats[s][t]["iters"] == iters
        assert np.abs(outs[s][t] - ora[0]).max() <= 1e-4 * EXTENT, (s, t)
    # cumulative: shape 0.5, step 1 (continues from step 0's result)
    ora, _ = O.run(base, vals[:2].astype(np.float64), K, shape=SHAPES[1], max_iters=iters, xi_stop=0,
                   stall_window=0, mode="cumulative")
    assert np.abs(outs[4][1] - ora[1]).max() <= 1e-4 * EXTENT


def test_benchmark_iteration_count_properties(sweep_setup):
    mesh, vals, m = sweep_setup
    iters = 50
    outs, stats = run_sweep(m, vals, iters)
    N = 1 << K
    for s, t in ((0, 0), (2, 23), (4, 23)):
        g = outs[s][t]
        assert np.isfinite(g).all() and np.abs(g - mesh.verts).max() > 1e-3
        assert stats[s][t]["iters"] == iters
        # labels and counts of the returned vertices: bit-exact
        lab = torch.empty((N, N), dtype=torch.int16, device="cuda")
        cnt = torch.empty(mesh.n_regions + 1, dtype=torch.int32, device="cuda")
        P.inim_raster(m, torch.as_tensor(g, device="cuda"), K, lab, cnt)
        olab, ocnt, _ = O.labels_scanline(g.astype(np.float64), *arrays(mesh), K)
        olab = np.where(olab < 0, mesh.n_regions, olab)
        np.testing.assert_array_equal(lab.cpu().numpy().view(np.uint16).astype(np.int64), olab)
        np.testing.assert_array_equal(cnt.cpu().numpy()[:-1], ocnt)
        # the reported error is the error of the returned vertices (desired
        # areas from the raster of those vertices, within the change of the
        # total mass over one iteration)
        v = vals[t].astype(np.float64)
        d0 = v[ocnt > 0].sum() / ocnt.sum()
        eps, _ = O.cartographic_errors(O.signed_areas(g.astype(np.float64), *arrays(mesh)),
                                       O.desired_areas(v, ocnt, d0, N))
        assert abs(eps - stats[s][t]["eps"]) <= 2e-3, (s, t, eps, stats[s][t]["eps"])
