"""GPU parity of the single-pass integral-image scan (Sec. 3.1, Sec. 4.1 step 4)
against the three-kernel scan, on batches large enough to take it.

The single-pass kernel sums the carries between bands by look-back in 64-bit
fixed point.  So: in FIX64 (exact integer sums either way) both forms give
bit-identical iterations in every row-serial tile; in FP32 and the
compensated form the single-pass result does not depend on which earlier
band a look-back stops at (two runs are bit-identical) and stays within the
N-iteration bound of the three-kernel result (the carries are the exactly
rounded sums instead of FP32 partial sums); the vertices follow the oracle
within the one-iteration bound after one iteration.
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
K = 10                       # 1024^2: eight solves make the 2^23 pixels of a large batch


@pytest.fixture(scope="module")
def work():
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    m = P.inim_map_create(mesh)
    vals = w["values"][:8].astype(np.float32)                 # 8 time steps: an 8-solve direct batch
    yield mesh, m, vals
    m.close()


def _run(m, vals, precision, iters, single_pass, tile=None):
    P.inim_set_single_pass_scan(single_pass)
    if tile:
        P.inim_set_scan_tile(K, precision, 1, *tile)
    try:
        out, st, _ = P.inim_run(m, vals, P.params(log2_res=K, shape=0.5, max_iters=iters, xi_stop=0.0,
                                                  stall_window=0, precision=precision))
    finally:
        if tile:
            P.inim_set_scan_tile(K, precision, 1, 0, 0, 0)
        P.inim_set_single_pass_scan(False)
    assert all(s["iters"] == iters for s in st)
    return out


ROW_SERIAL_TILES = [(16, 4, 256), (32, 4, 256), (8, 8, 128), (64, 16, 64), (4, 32, 32)]


@pytest.mark.parametrize("tile", ROW_SERIAL_TILES)
def test_fixed_point_single_pass_equals_three_kernels(work, tile):
    mesh, m, vals = work
    a = _run(m, vals, P.INIM_FIX64, 3, True, tile)
    b = _run(m, vals, P.INIM_FIX64, 3, False, tile)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", [P.INIM_FP32, P.INIM_KAHAN])
def test_single_pass_is_deterministic_and_close_to_three_kernels(work, precision):
    mesh, m, vals = work
    a = _run(m, vals, precision, 5, True)
    a2 = _run(m, vals, precision, 5, True)
    np.testing.assert_array_equal(a, a2)
    b = _run(m, vals, precision, 5, False)
    assert np.abs(a - b).max() <= 1e-4 * EXTENT


def test_single_pass_first_iteration_matches_oracle(work):
    mesh, m, vals = work
    out = _run(m, vals, P.INIM_FP32, 1, True)
    xy = mesh.verts_f32().astype(np.float64)
    t0 = O.transform_uniform(1 << K)
    arrays = (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
    for t in (0, 7):
        want, _ = O.iterate(xy, arrays, vals[t].astype(np.float64), K, 0.5, t0=t0)
        assert np.abs(out[t] - want).max() <= 1e-5 * EXTENT, t


def test_mixed_resolutions_in_one_large_batch(work):
    # a 2048^2 and a 1024^2 group in one batch: the 2048^2 group alone has
    # 2^22 pixels (three kernels), the 1024^2 group of eight solves 2^23
    # (single pass); each solve equals its own run
    mesh, m, vals = work
    p10 = P.params(log2_res=10, shape=0.5, max_iters=2, xi_stop=0.0, stall_window=0, precision=P.INIM_FIX64)
    p11 = P.params(log2_res=11, shape=0.5, max_iters=2, xi_stop=0.0, stall_window=0, precision=P.INIM_FIX64)
    series = [dict(map=m, values=vals, params=p10), dict(map=m, values=vals[:1], params=p11)]
    P.inim_set_single_pass_scan(True)
    try:
        outs, _, _ = P.inim_run_series(series)
    finally:
        P.inim_set_single_pass_scan(False)
    ref, _, _ = P.inim_run_series(series)
    np.testing.assert_array_equal(outs[0], ref[0])
    np.testing.assert_array_equal(outs[1], ref[1])
