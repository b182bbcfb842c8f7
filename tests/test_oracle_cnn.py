"""Pins of the CPU oracle of the warm-start network."""
import numpy as np
import pytest

from oracle import cnn_oracle as C


def test_conv_matches_its_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 4, 5, 3))
    w = rng.normal(size=(4, 9, 3))
    b = rng.normal(size=4)
    y = C.conv3x3(x, w, b)
    N, H, W, Ci = x.shape
    ref = np.zeros((N, H, W, 4))
    for n in range(N):
        for i in range(H):
            for j in range(W):
                for o in range(4):
                    s = b[o]
                    for dy in range(3):
                        for dx in range(3):
                            ii, jj = i + dy - 1, j + dx - 1
                            if 0 <= ii < H and 0 <= jj < W:
                                s += (x[n, ii, jj] * w[o, 3 * dy + dx]).sum()
                    ref[n, i, j, o] = s
    np.testing.assert_allclose(y, ref, atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 5, 4, 2))
    w = rng.normal(size=(3, 9, 2))
    b = rng.normal(size=3)
    gy = rng.normal(size=(1, 5, 4, 3))
    gx, gw, gb = C.conv3x3_backward(x, w, gy)
    f = lambda x_, w_, b_: (C.conv3x3(x_, w_, b_) * gy).sum()          # noqa: E731
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 4, 3, 1), (0, 2, 1, 0)]:
        d = np.zeros_like(x); d[idx] = h
        assert abs((f(x + d, w, b) - f(x - d, w, b)) / (2 * h) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0), (2, 8, 1), (1, 4, 0)]:
        d = np.zeros_like(w); d[idx] = h
        assert abs((f(x, w + d, b) - f(x, w - d, b)) / (2 * h) - gw[idx]) < 1e-6
    d = np.zeros_like(b); d[1] = h
    assert abs((f(x, w, b + d) - f(x, w, b - d)) / (2 * h) - gb[1]) < 1e-6


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 8, 6, 3))
    y = rng.normal(size=(1, 4, 3, 3))
    assert abs((C.pool2(x) * y).sum() - (x * C.pool2_backward(y)).sum()) < 1e-12
    z = rng.normal(size=(1, 8, 6, 3))
    assert abs((C.up2(y) * z).sum() - (y * C.up2_backward(z)).sum()) < 1e-12


def test_network_gradient_finite_differences():
    params = C.he_init(3)
    assert params.size == C.n_params() == 1163234
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 16, 16))
    t = rng.normal(size=(1, 16, 16, 2)) * 0.1
    loss, g = C.loss_and_grads(params, x, t)
    # one parameter of every layer (weights and biases), central differences
    h = 1e-5
    off = 0
    checked = 0
    for ci, co, _ in C.LAYERS:
        for k in (off + (co * 9 * ci) // 3, off + co * 9 * ci):        # a weight, the first bias
            p1, p2 = params.copy(), params.copy()
            p1[k] += h
            p2[k] -= h
            fd = (C.loss_and_grads(p1, x, t)[0] - C.loss_and_grads(p2, x, t)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(fd), (k, fd, g[k])
            checked += 1
        off += co * 9 * ci + co
    assert checked == 28 and loss > 0


def test_bf16_round_definition():
    # BF16 keeps 7 fraction bits: the spacing at 1 is 2^-7
    u = 2.0 ** -7
    cases = {1.0: 1.0, 1 + u / 2: 1.0,                     # tie -> even fraction (0)
             1 + 1.5 * u: 1 + 2 * u,                       # tie -> even fraction (2)
             1 + u / 2 + 2.0 ** -20: 1 + u,                # just above the tie
             -(1 + 1.5 * u): -(1 + 2 * u), 3.0: 3.0, 0.0: 0.0}
    for x, want in cases.items():
        assert C.bf16_round(np.array([x]))[0] == want, x
    # nearest of the two BF16 neighbours, by brute force in float64
    rng = np.random.default_rng(9)
    x = (rng.normal(size=4000) * 10.0 ** rng.integers(-6, 6, 4000)).astype(np.float32).astype(np.float64)
    got = C.bf16_round(x)
    bits = x.astype(np.float32).view(np.uint32)
    lo = (bits & 0xFFFF0000).view(np.float32).astype(np.float64)             # toward zero
    hi = ((bits & 0xFFFF0000) + 0x10000).astype(np.uint32).view(np.float32).astype(np.float64)
    d_lo, d_hi = np.abs(x - lo), np.abs(hi - x)
    assert np.all((got == lo) | (got == hi))
    assert np.all(np.where(d_lo < d_hi, got == lo, True)) and np.all(np.where(d_hi < d_lo, got == hi, True))


def test_bf16_mode_rounds_only_what_is_stored():
    params = C.he_init(6)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(1, 16, 16))
    out64, s64 = C.forward(params, x)
    out16, s16 = C.forward(params, x, bf16=True)
    for name in ("x0", "a0", "e1", "p1", "d3", "d1b"):
        assert np.array_equal(C.bf16_round(s16[name]), s16[name]), name      # stored values are BF16
    assert not np.array_equal(C.bf16_round(out16), out16)                      # the head is not rounded
    rel = np.linalg.norm(out16 - out64) / np.linalg.norm(out64)
    assert 1e-4 < rel < 3e-2                                                   # roundings only: ~sqrt(40) 2^-9
    t = rng.normal(size=(1, 16, 16, 2)) * 0.1
    l64, g64 = C.loss_and_grads(params, x, t)
    saved = {}
    l16, g16 = C.loss_and_grads(params, x, t, bf16=True, saved=saved)
    assert np.array_equal(C.bf16_round(saved["ge1"]), saved["ge1"])
    assert abs(l16 - l64) < 3e-2 * l64
    assert np.dot(g16, g64) / (np.linalg.norm(g16) * np.linalg.norm(g64)) > 0.99


def _center_only_first_layer(params):
    # the first convolution reduced to its centre tap with positive weights:
    # on a non-negative input it is a per-pixel affine map followed by an
    # identity ReLU, so it commutes with 2x2 average pooling
    p = params.copy()
    ci, co, _ = C.LAYERS[0]
    w = p[:co * 9 * ci].reshape(co, 9, ci)
    w[:] = 0.0
    w[:, 4, :] = np.abs(np.random.default_rng(9).normal(size=(co, ci))) + 0.1
    p[co * 9 * ci:co * 9 * ci + co] = np.abs(p[co * 9 * ci:co * 9 * ci + co])
    return p


@pytest.mark.parametrize("stem", [1, 2])
def test_stem_equals_pooled_input_for_pointwise_first_layer(stem):
    params = _center_only_first_layer(C.he_init(8))
    rng = np.random.default_rng(10 + stem)
    x = rng.uniform(0.0, 2.0, size=(2, 16 << stem, 16 << stem))
    f = 1 << stem
    xp = x.reshape(2, 16, f, 16, f).mean(axis=(2, 4))
    got, _ = C.forward(params, x, stem=stem)
    want, _ = C.forward(params, xp)
    assert got.shape == (2, 16, 16, 2)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    # the same holds for the loss, and for every gradient past the first layer
    t = rng.normal(size=(2, 16, 16, 2)) * 0.1
    l1, g1 = C.loss_and_grads(params, x, t, stem=stem)
    l2, g2 = C.loss_and_grads(params, xp, t)
    ci, co, _ = C.LAYERS[0]
    n0 = co * 9 * ci + co
    assert abs(l1 - l2) <= 1e-12 * l2
    np.testing.assert_allclose(g1[n0:], g2[n0:], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("stem", [1, 2])
def test_stem_gradient_finite_differences(stem):
    params = C.he_init(12)
    rng = np.random.default_rng(13)
    x = rng.normal(size=(1, 16 << stem, 16 << stem))
    t = rng.normal(size=(1, 16, 16, 2)) * 0.1
    _, g = C.loss_and_grads(params, x, t, stem=stem)
    h = 1e-5
    ci, co, _ = C.LAYERS[0]
    ci1, co1, _ = C.LAYERS[1]
    n0 = co * 9 * ci
    # first-layer weights and bias (seen through the pools), and a second-layer weight
    for k in (0, n0 // 2, n0 - 1, n0, n0 + co - 1, n0 + co + (co1 * 9 * ci1) // 2):
        p1, p2 = params.copy(), params.copy()
        p1[k] += h
        p2[k] -= h
        fd = (C.loss_and_grads(p1, x, t, stem=stem)[0] - C.loss_and_grads(p2, x, t, stem=stem)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(fd), (k, fd, g[k])
