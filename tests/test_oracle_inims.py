"""Pins of the oracle's integral images and map t (Sec. 3.1, 3.2, Eq. 1-3)."""
import json
import os

import numpy as np
import pytest

from oracle import inim_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KEYS = ("a", "b", "g", "d", "at", "bt", "gt", "dt")


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 11, 16])
def test_fast_inims_equal_bruteforce(N):
    # integer-valued texture: every sum is exact in float64
    d = np.random.default_rng(N).integers(0, 50, size=(N, N)).astype(np.float64)
    bf = O.inims_bruteforce(d)
    fast = O.inims(d)
    for k in KEYS:
        np.testing.assert_array_equal(fast[k], bf[k], err_msg=k)


@pytest.mark.parametrize("N", [2, 7, 13])
def test_left_wedge_two_ways(N):
    d = np.random.default_rng(100 + N).integers(0, 9, size=(N, N)).astype(np.float64)
    np.testing.assert_array_equal(O.left_wedge_rows(d), O.left_wedge_sweep(d))


@pytest.mark.parametrize("N", [4, 9, 32])
def test_sum_identity_eq1(N):
    d = np.random.default_rng(N).random((N, N))
    I = O.inims(d)
    C = d.sum()
    np.testing.assert_allclose(I["a"] + I["b"] + I["g"] + I["d"], C, rtol=1e-12)
    np.testing.assert_allclose(I["at"] + I["bt"] + I["gt"] + I["dt"], C, rtol=1e-12)
    for k in KEYS:  # non-negative texture -> non-negative sums
        assert (I[k] >= -1e-9 * C).all(), k


def test_uniform_closed_forms():
    N = 16
    I = O.inims(np.ones((N, N)))
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    np.testing.assert_array_equal(I["a"], (i + 1) * (j + 1))
    np.testing.assert_array_equal(I["g"], (N - 1 - i) * (N - 1 - j))
    # left wedge pixel count: row j' holds max(0, i + 1 - |j' - j|) pixels
    L = np.zeros((N, N))
    for jp in range(N):
        L += np.maximum(0, i + 1 - np.abs(jp - j))
    np.testing.assert_array_equal(I["bt"], L)


def test_inims_monotone():
    d = np.random.default_rng(5).random((24, 24))
    I = O.inims(d)
    assert (np.diff(I["a"], axis=0) >= 0).all() and (np.diff(I["a"], axis=1) >= 0).all()
    assert (np.diff(I["bt"], axis=1) >= 0).all()   # left wedge grows to the right


def test_point_mass_golden():
    gold = json.load(open(os.path.join(GOLD, "point_mass_t.json")))
    for c in gold["cases"]:
        N = c["N"]
        d = np.zeros((N, N))
        d[c["mass"][1], c["mass"][0]] = 1.0
        x, y = O.pixel_centres(N)
        tx, ty = O.transform(O.inims(d), x, y)
        i, j = c["at"]
        assert (tx[j, i], ty[j, i]) == tuple(c["t"]), c


def test_uniform_t_golden():
    gold = json.load(open(os.path.join(GOLD, "uniform_t_2x2.json")))
    I = O.inims(np.ones((2, 2)))
    tx, ty = O.transform_uniform(2)
    for key, t in gold["t"].items():
        i, j = map(int, key.split(","))
        assert (tx[j, i], ty[j, i]) == tuple(t)
        for k, v in gold["counts"][key].items():
            assert I[k][j, i] == v, (key, k)


def test_t_in_unit_square_and_identity():
    rng = np.random.default_rng(9)
    N = 32
    d = rng.lognormal(0, 2, (N, N))
    x, y = O.pixel_centres(N)
    tx, ty = O.transform(O.inims(d), x, y)
    assert tx.min() >= 0 and tx.max() <= 1 and ty.min() >= 0 and ty.max() <= 1
    # Eq. (3) is the identity for a constant texture of any value
    fx, fy = O.displacement_field(np.full((N, N), 3.7))
    assert np.abs(fx).max() < 1e-14 and np.abs(fy).max() < 1e-14


def test_field_pushes_away_from_mass():
    # mass in the top-left quadrant pushes the domain centre to the bottom-right
    N = 32
    d = np.ones((N, N))
    d[: N // 2, : N // 2] = 5.0
    fx, fy = O.displacement_field(d)
    c = N // 2
    assert fx[c, c] > 1e-3 and fy[c, c] > 1e-3
    # and mass at the bottom pushes the centre up
    d = np.ones((N, N))
    d[N // 2:, :] = 5.0
    fx, fy = O.displacement_field(d)
    assert fy[c, c] < -1e-3 and abs(fx[c, c]) < 1e-2


def test_field_symmetry_approx():
    # mirroring the texture mirrors the field up to O(1/N) tie effects
    N = 64
    rng = np.random.default_rng(3)
    base = rng.random((8, 8)) + 0.2
    d = np.kron(base, np.ones((N // 8, N // 8)))
    fx, fy = O.displacement_field(d)
    gx, gy = O.displacement_field(d[:, ::-1])
    assert np.abs(fx + gx[:, ::-1]).max() < 4.0 / N
    assert np.abs(fy - gy[:, ::-1]).max() < 4.0 / N
    hx, hy = O.displacement_field(d.T)
    assert np.abs(fx - hy.T).max() < 4.0 / N
    assert np.abs(fy - hx.T).max() < 4.0 / N


def test_bilinear_reproduces_linear_field():
    N = 16
    x, y = O.pixel_centres(N)
    f = 0.3 * x - 1.7 * y + 0.25
    pts = np.random.default_rng(1).uniform(0.5 / N, 1 - 0.5 / N, (200, 2))
    np.testing.assert_allclose(O.bilinear(f, pts), 0.3 * pts[:, 0] - 1.7 * pts[:, 1] + 0.25,
                               atol=1e-13)
    # at a pixel centre it returns that pixel's value
    np.testing.assert_allclose(O.bilinear(f, np.array([[x[3, 5], y[3, 5]]])), f[3, 5], atol=1e-15)
