"""The kernel timeline (a profiling aid of the library): with it on, a fixed
run of n iterations records n launches of every kernel of the iteration, in
order (each kernel starts after the previous one of its iteration ended,
the area kernel excepted, which runs beside the next raster), and the moved
vertices are the same as with the timeline off.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402
from paper_2604_13880_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_timeline_records_every_launch_in_order():
    mesh = synth.voronoi_map(30, 2000, seed=5)
    vals = synth.lognormal_values(30, seed=6)[None].astype(np.float32)
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=9, shape=0.5, max_iters=12, xi_stop=0.0, stall_window=0)
    ref, _, _ = P.inim_run(m, vals, p)
    P.inim_timeline(True)
    try:
        out, _, _ = P.inim_run(m, vals, p)
        st, en = P.inim_timeline_read()
    finally:
        P.inim_timeline(False)
    np.testing.assert_array_equal(out, ref)
    names = P.TIMELINE_KERNELS
    ran = [q for q in range(len(names)) if st[q, 0] > 0]
    assert {names[q] for q in ran} >= {"crossings", "rows", "scan_phase1", "scan_phase3", "gather_move",
                                       "areas_errors"}
    for q in ran:
        assert np.all(st[q, :12] > 0) and np.all(en[q, :12] >= st[q, :12]), names[q]
        assert np.all(st[q, 12:] == 0), names[q]               # exactly 12 launches
    path = [q for q in ran if names[q] != "areas_errors"]
    for i in range(12):
        for a, b in zip(path[:-1], path[1:]):
            assert st[b, i] >= en[a, i], (names[a], names[b], i)
        if i:
            assert st[path[0], i] >= en[path[-1], i - 1]
    with pytest.raises(P.InimError):
        P.inim_timeline_read()                                 # off again
    m.close()
