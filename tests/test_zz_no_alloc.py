"""The allocation-free integral-image entry point against the regular one.

inim_inims_noalloc is for callers that cannot allocate device memory (another
framework owns the device pool, or a loop that cannot afford cudaMalloc's
device synchronisation): it keeps its working memory in a fixed array inside
the library.  Its results must equal inim_inims (FP32) within the FP32
integral-image tolerance of the parity tests, call after call.  This file is
collected last on purpose, and the test also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2604_13880_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu


def _buffers(N):
    return [torch.empty((N, N), dtype=torch.float32, device="cuda"),
            torch.empty((N, N), dtype=torch.float32, device="cuda"),
            torch.empty(2 * N - 1, dtype=torch.float32, device="cuda"),
            torch.empty(2 * N - 1, dtype=torch.float32, device="cuda")]


def _check_call(k, seed, label):
    N = 1 << k
    tol_depth = 2 * (N / 8 + 64) * 2.0 ** -24       # same bound as the FP32 parity test
    d = torch.as_tensor(np.random.default_rng(seed).lognormal(0.0, 1.0, (N, N)).astype(np.float32),
                        device="cuda")
    ref = _buffers(N)
    P.inim_inims(d, k, P.INIM_FP32, 0, *ref)
    got = _buffers(N)
    for x in got:
        x.fill_(float("nan"))                      # every output element must be written
    P.inim_inims_noalloc(d, k, *got)
    torch.cuda.synchronize()
    C = float(d.double().sum())
    for g, r, name in zip(got, ref, "STAB"):
        assert torch.isfinite(g).all(), (label, name)
        err = (g.double() - r.double()).abs().max().item()
        assert err <= tol_depth * C, (label, name, err / C)


@pytest.mark.parametrize("k", [8, 9, 10])
def test_noalloc_matches_regular_two_calls(k):
    for call, seed in enumerate((k, k + 100)):      # two calls in a row, different textures
        _check_call(k, seed, (k, call))


def test_noalloc_alternating_sizes():
    # the job descriptor in the shared array changes size between calls: each
    # call must use its own, never the previous call's
    for call, k in enumerate((10, 8, 10, 9, 8)):
        _check_call(k, 500 + call, (call, k))


def test_noalloc_rejects_large_texture():
    with pytest.raises(P.InimError) as e:
        bufs = _buffers(16)   # sizes are checked before any use of the buffers
        P.inim_inims_noalloc(torch.zeros(1, device="cuda"), 11, *bufs)
    assert e.value.status == -5
    assert "1024" in str(e.value)          # the message of inim_last_error()
