"""Animation frames (Sec. 5.5): the values are interpolated linearly between
consecutive time steps (10 frames per step) and a cartogram is computed for
every frame.  The GPU series runs the library's interpolated values through
inim_run_series, directly (every frame from the original map) and
cumulatively (every frame from the previous frame's cartogram); sampled
frames are compared with the oracle's run on the oracle's own interpolation
of the same series, within the N-iteration bound.
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
F = 10


@pytest.fixture(scope="module")
def series():
    mesh = synth.voronoi_map(24, 1500, seed=91, jitter=0.2)
    steps = synth.random_walk_values(24, 3, seed=92, sigma=0.4).astype(np.float32)
    frames = P.inim_interpolate_values(steps, F)
    want = O.interpolate_series(steps.astype(np.float64), F)
    assert frames.shape == ((3 - 1) * F + 1, 24)
    np.testing.assert_allclose(frames, want, rtol=1e-6)       # float values of the oracle's frames
    return mesh, frames


@pytest.mark.parametrize("mode,iters", [(P.INIM_DIRECT, 6), (P.INIM_CUMULATIVE, 2)])
def test_interpolated_series_matches_oracle(series, mode, iters):
    mesh, frames = series
    m = P.inim_map_create(mesh)
    p = P.params(log2_res=8, shape=0.5, max_iters=iters, xi_stop=0.0, stall_window=0, mode=mode)
    outs, stats, _ = P.inim_run_series([dict(map=m, values=frames, params=p)])
    out = outs[0]
    assert out.shape == (len(frames), mesh.n_verts, 2)
    assert all(s["iters"] == iters for s in stats[0])
    base = mesh.with_verts(mesh.verts_f32().astype(np.float64))
    name = "direct" if mode == P.INIM_DIRECT else "cumulative"
    sample = [0, 7, 13, 20] if mode == P.INIM_DIRECT else list(range(len(frames)))
    if mode == P.INIM_DIRECT:
        for f in sample:
            want, _ = O.run(base, frames[f:f + 1].astype(np.float64), 8, shape=0.5, max_iters=iters, xi_stop=0,
                            stall_window=0)
            assert np.abs(out[f] - want[0]).max() <= 1e-4 * EXTENT, (name, f)
    else:
        want, _ = O.run(base, frames.astype(np.float64), 8, shape=0.5, max_iters=iters, xi_stop=0, stall_window=0,
                        mode="cumulative")
        for f in (0, 5, 10, 20):
            assert np.abs(out[f] - want[f]).max() <= 1e-4 * EXTENT, (name, f)
    # consecutive frames of an animation move little compared with the whole deformation
    step = np.abs(np.diff(out, axis=0)).max()
    total = np.abs(out[-1] - mesh.verts_f32()).max()
    assert step < total
    m.close()
