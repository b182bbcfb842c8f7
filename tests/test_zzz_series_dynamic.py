"""GPU parity of a dynamic-area series in one call (inim_run_dynamic; Sec. 4.3,
Eq. (Mb)): every step's background value from the series, direct and
cumulative, against the oracle's run with the same area fractions.  Runs
after the rest of the GPU suite.

Tolerance: the N-iteration bound, 1e-4 of the map extent.
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


def _case():
    mesh = synth.voronoi_map(30, 1500, seed=35)
    vals = synth.random_walk_values(30, 3, seed=36).astype(np.float32)
    return mesh, vals


@pytest.mark.parametrize("mode,name", [(P.INIM_DIRECT, "direct"), (P.INIM_CUMULATIVE, "cumulative")])
def test_dynamic_series_matches_oracle(mode, name):
    mesh, vals = _case()
    a_min, a_max, iters = 0.45, 0.65, 4
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.25, max_iters=iters, xi_stop=0.0, stall_window=0, mode=mode)
    out, stats, _ = P.inim_run_dynamic(m, vals, p, a_min, a_max)
    base = mesh.with_verts(mesh.verts_f32().astype(np.float64))
    ora, ostats = O.run(base, vals.astype(np.float64), 8, shape=0.25, max_iters=iters, xi_stop=0, stall_window=0,
                        mode=name, area_fractions=(a_min, a_max))
    for t in range(3):
        assert stats[t]["iters"] == iters
        assert np.abs(out[t] - ora[t]).max() <= 1e-4 * EXTENT, (name, t)
    if mode == P.INIM_DIRECT:
        # the same solves as a batch of jobs with the background values given
        bdv, _ = P.inim_background_values(vals, 8, a_min, a_max)
        jobs = [dict(map=m, values=vals[t], params=P.params(log2_res=8, shape=0.25, max_iters=iters, xi_stop=0.0,
                                                            stall_window=0, bdv_value=float(bdv[t])))
                for t in range(3)]
        outs, _, _ = P.inim_run_batch(jobs)
        for t in range(3):
            np.testing.assert_array_equal(out[t], outs[t])
