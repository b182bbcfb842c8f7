"""The range behind the crossing kernel's 32-bit fixed point.

The raster rule (Sec. 4.1 step 2, the exact integer reading) snaps a vertex
to X = rint(x 2^(k+8)) and, for a row centre Yc = 256 j + 128 inside an edge's
row range, counts the columns from
    c = ceil((dX (Yc - Y0) + (X0 - 128) dY) / (256 dY)).
The kernel forms X, Y, the differences dX, dY, Yc - Y0, X0 - 128 and the row
range in 32-bit integers when every end point of a warp's edges lies within 512
of the origin, and only the two products in 64 bits.  These checks run the
bound on the CPU: at the largest texture (k = 12) and coordinates up to the
limit, every one of those quantities fits a signed 32-bit integer, and the
column from 32-bit-wrapped differences equals the one from exact integers.
"""
import numpy as np

LIMIT = 512.0
K = 12


def _snap(x, k):
    # the product is exact in float32 (a power-of-two scale); ties to even
    return np.rint(np.float32(x) * np.float32(2.0 ** (k + 8))).astype(np.int64)


def _ceil_div(a, b):
    return -((-a) // b)


def _wrap32(v):
    return ((v + 2 ** 31) % 2 ** 32) - 2 ** 31


def test_snapped_coordinates_and_differences_fit_32_bits():
    rng = np.random.default_rng(3)
    lim = np.nextafter(np.float32(LIMIT), np.float32(0))            # largest float32 below the limit
    x = np.concatenate([rng.uniform(-LIMIT, LIMIT, 200_000).astype(np.float32),
                        np.array([lim, -lim, 0.0, 1.0], np.float32)])
    X = _snap(x, K)
    assert np.abs(X).max() < 2 ** 29
    Y0, Y1 = np.minimum(X[::2], X[1::2]), np.maximum(X[::2], X[1::2])
    for v in (Y1 - Y0, Y0 - 128, Y1 - 128, X[::2] - 128):
        assert np.abs(v).max() < 2 ** 31
    # the row centres inside the texture against any start point
    Yc = 256 * np.int64((1 << K) - 1) + 128
    assert np.abs(Yc - Y0).max() < 2 ** 31


def test_column_from_wrapped_differences_is_exact():
    rng = np.random.default_rng(4)
    n = 1 << K
    pts = rng.uniform(-LIMIT, LIMIT, (20_000, 4)).astype(np.float32)
    pts[:10_000] = rng.uniform(-0.2, 1.2, (10_000, 4)).astype(np.float32)   # the usual map range
    X0, Y0, X1, Y1 = (_snap(pts[:, q], K) for q in range(4))
    swap = Y1 < Y0
    X0, X1 = np.where(swap, X1, X0), np.where(swap, X0, X1)
    Y0, Y1 = np.where(swap, Y1, Y0), np.where(swap, Y0, Y1)
    keep = Y1 > Y0
    X0, Y0, X1, Y1 = X0[keep], Y0[keep], X1[keep], Y1[keep]
    jlo = np.maximum(_ceil_div(Y0 - 128, 256), 0)
    jhi = np.minimum(_ceil_div(Y1 - 128, 256) - 1, n - 1)
    # 32-bit row range: (a + 255) >> 8 on wrapped values
    jlo32 = np.maximum((_wrap32(Y0 - 128) + 255) >> 8, 0)
    jhi32 = np.minimum(((_wrap32(Y1 - 128) + 255) >> 8) - 1, n - 1)
    np.testing.assert_array_equal(jlo, jlo32)
    np.testing.assert_array_equal(jhi, jhi32)
    rows = jhi >= jlo
    j = np.where(rows, jlo, 0)
    Yc = 256 * j + 128
    dX, dY = X1 - X0, Y1 - Y0
    exact = np.clip(_ceil_div(dX * (Yc - Y0) + (X0 - 128) * dY, 256 * dY), 0, n)
    num32 = _wrap32(dX) * _wrap32(Yc - Y0) + _wrap32(X0 - 128) * _wrap32(dY)
    got = np.clip(_ceil_div(num32, 256 * _wrap32(dY)), 0, n)
    np.testing.assert_array_equal(exact[rows], got[rows])
    assert rows.sum() > 1000
