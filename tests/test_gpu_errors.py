"""Failure detection on the GPU without a GPU fault.

(1) Invalid region values (NaN, negative) are refused: host values by the
entry point before any work, device values by the kernel that builds the
density table (Sec. 4.1 step 3), which records INIM_E_VALUE in the job state.
(2) A device-side wait that runs out: with the wait cap set to one poll,
the grid barrier of the persistent launch gives up at once, every block
returns, the call reports INIM_E_TIMEOUT, and the next call (default cap)
runs normally in the same context.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402
from paper_2604_13880_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    mesh = synth.voronoi_map(12, 600, seed=81)
    m = P.inim_map_create(mesh)
    vals = synth.random_walk_values(12, 3, seed=82).astype(np.float32)
    yield mesh, m, vals
    m.close()


@pytest.mark.parametrize("bad", [float("nan"), -1.0, float("inf")])
def test_host_values_refused(case, bad):
    _, m, vals = case
    v = vals.copy()
    v[1, 3] = bad
    with pytest.raises(P.InimError) as e:
        P.inim_run(m, v, P.params(log2_res=8, max_iters=3, xi_stop=0.0, stall_window=0))
    assert e.value.status == P.INIM_E_VALUE


@pytest.mark.parametrize("bad", [float("nan"), -2.0])
def test_device_values_refused_by_the_table_kernel(case, bad):
    _, m, vals = case
    v = vals[:1].copy()
    v[0, 5] = bad
    vd = torch.as_tensor(v, device="cuda")
    with pytest.raises(P.InimError) as e:
        P.inim_run(m, vd, P.params(log2_res=8, max_iters=3, xi_stop=0.0, stall_window=0))
    assert e.value.status == P.INIM_E_VALUE
    # the same call with valid values works afterwards
    out, st, status = P.inim_run(m, torch.as_tensor(vals[:1], device="cuda"),
                                 P.params(log2_res=8, max_iters=3, xi_stop=0.0, stall_window=0))
    assert status >= 0 and st[0]["iters"] == 3


def test_barrier_wait_runs_out_and_context_survives(case):
    mesh, m, vals = case
    p = P.params(log2_res=8, shape=0.5, max_iters=4, xi_stop=0.0, stall_window=0, mode=P.INIM_CUMULATIVE)
    ref, _, _ = P.inim_run(m, vals, p)                   # graph path, for the check after recovery
    try:
        P.inim_set_persistent(True)
        P.inim_set_wait_cap(1)
        with pytest.raises(P.InimError) as e:
            P.inim_run(m, vals, p)
        assert e.value.status == P.INIM_E_TIMEOUT
        P.inim_set_wait_cap(0)                           # the default cap again
        out, st, status = P.inim_run(m, vals, p)
    finally:
        P.inim_set_wait_cap(0)
        P.inim_set_persistent(False)
    assert status >= 0 and [s["iters"] for s in st] == [4, 4, 4]
    # the persistent path scans with other tiles than the graph path: within
    # the FP32 bound of the parity tests after a few iterations
    assert np.abs(out - ref).max() <= 1e-4
