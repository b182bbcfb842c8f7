"""The batched workload at its full size: 64 independent maps of 20-500 regions
with textures drawn from {256, 512, 1024, 2048}^2, solved in one batch.

Every solve of the batch equals the same solve run alone: bit-exactly in
64-bit fixed point (the integral images are exact integer sums whatever the
band tiles, and a size group of the batch shares its scan launches and tiles
while a single solve scans alone with its own), and within the N-iteration
bound in FP32.  Sampled solves (the largest 2048^2 map and a 256^2 map) follow the
FP64 oracle within the N-iteration bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402
from paper_2604_13880_gb300 import _lib, synth  # noqa: E402
from oracle import inim_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
EXTENT = 0.9


@pytest.fixture(scope="module")
def batch():
    w = synth.batched_workload()
    maps = [P.inim_map_create(x["mesh"]) for x in w]
    yield w, maps
    for m in maps:
        m.close()


def _run_batch(w, maps, iters, precision):
    jobs = (P.inim_job * len(w))()
    vals = [np.ascontiguousarray(x["values"][0], dtype=np.float32) for x in w]
    outs = [np.empty((x["mesh"].n_verts, 2), np.float32) for x in w]
    for q, (x, m) in enumerate(zip(w, maps)):
        jobs[q].map = m.handle
        jobs[q].values = vals[q].ctypes.data
        jobs[q].init_xy = None
        jobs[q].out_xy = outs[q].ctypes.data
        jobs[q].params = P.params(log2_res=x["log2_res"], shape=0.5, max_iters=iters, xi_stop=0.0, stall_window=0,
                                  precision=precision)
        jobs[q].stats = None
    _lib.check(_lib.load().inim_run_batch(jobs, len(jobs), None), "batched workload")
    return outs


def _single(x, m, iters, precision):
    out, st, _ = P.inim_run(m, x["values"].astype(np.float32),
                            P.params(log2_res=x["log2_res"], shape=0.5, max_iters=iters, xi_stop=0.0, stall_window=0,
                                     precision=precision))
    assert st[0]["iters"] == iters
    return out[0]


def test_workload_shape(batch):
    w, _ = batch
    ks = {x["log2_res"] for x in w}
    assert len(w) == 64 and ks == {8, 9, 10, 11}
    assert all(20 <= x["mesh"].n_regions <= 500 for x in w)


def test_batch_equals_single_runs_fixed_point(batch):
    w, maps = batch
    outs = _run_batch(w, maps, 2, P.INIM_FIX64)
    for q, (x, m) in enumerate(zip(w, maps)):
        np.testing.assert_array_equal(outs[q], _single(x, m, 2, P.INIM_FIX64), err_msg=f"solve {q}")


def test_batch_close_to_single_runs_fp32(batch):
    w, maps = batch
    outs = _run_batch(w, maps, 5, P.INIM_FP32)
    worst = 0.0
    for q, (x, m) in enumerate(zip(w, maps)):
        worst = max(worst, float(np.abs(outs[q] - _single(x, m, 5, P.INIM_FP32)).max()))
    assert worst <= 1e-4 * EXTENT, worst


def test_sampled_solves_follow_the_oracle(batch):
    w, maps = batch
    outs = _run_batch(w, maps, 2, P.INIM_FP32)
    big = max(range(len(w)), key=lambda q: (w[q]["log2_res"], w[q]["mesh"].n_verts))
    small = min(range(len(w)), key=lambda q: (w[q]["log2_res"], -w[q]["mesh"].n_regions))
    for q in (big, small):
        x = w[q]
        mesh = x["mesh"]
        xy = mesh.verts_f32().astype(np.float64)
        arrays = (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
        t0 = O.transform_uniform(1 << x["log2_res"])
        vals = x["values"][0].astype(np.float32).astype(np.float64)
        for _ in range(2):
            xy, _ = O.iterate(xy, arrays, vals, x["log2_res"], 0.5, t0=t0)
        assert np.abs(outs[q] - xy).max() <= 1e-4 * EXTENT, (q, x["log2_res"])
