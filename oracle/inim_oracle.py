"""CPU oracle of the integral-image (InIm) cartogram iteration.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's ``smoke()`` check and
the benchmark's CPU-baseline leg may import this module.  It shares no code
with the CUDA path and imports nothing from it.

Plain, slow, obviously-correct numpy in float64.  Every function follows one
step of the paper's static algorithm (Sec. 4.1, steps 0-7) or one definition
of Sec. 3 and says which.  Where the paper is silent, the readings used here
are the ones listed in the design notes of the repository (pixel-centre
samples, half-open fixed-point rasterisation rule, tilted-wedge tie rule, the
shape blend, the desired area w(v)).

Pins: every function is checked in ``tests/test_oracle_*.py`` against brute
force on tiny inputs, closed forms, invariants of Eq. (1)-(3) and hand-derived
golden values (``tests/golden``); the dynamic-area background of Eq. (Mb) by
the fixed point of a map at its target area fraction, the direction in which
a map away from it moves and hand-worked values away from the target; the
desired areas and the cartographic errors by hand-worked cases; the
animation frames of Sec. 5.5 by closed forms.  Readings the paper does not
fix (pinned only by the shared reading; their arithmetic is pinned as
above): the shape-blend reading, the definition of the desired area w(v)
and the pixel-sample convention.
"""
from __future__ import annotations

import numpy as np

SUBPIXEL_BITS = 8          # fixed-point sub-pixel bits of the rasteriser
BACKGROUND = -1            # label of background pixels in this oracle


# ----------------------------------------------------------------------------
# mesh helpers
# ----------------------------------------------------------------------------

def region_edges(ring_off, ring_idx, ring_region, n_regions):
    """Per region: (a, b) vertex-index arrays of its boundary edges.

    Each ring is closed implicitly.  Sec. 4.1 step 0: regions are described by
    polygons.
    """
    out = [([], []) for _ in range(n_regions)]
    for r in range(len(ring_region)):
        idx = np.asarray(ring_idx[ring_off[r]:ring_off[r + 1]], dtype=np.int64)
        a, b = out[int(ring_region[r])]
        a.append(idx)
        b.append(np.roll(idx, -1))
    return [(np.concatenate(a) if a else np.zeros(0, np.int64),
             np.concatenate(b) if b else np.zeros(0, np.int64)) for a, b in out]


# ----------------------------------------------------------------------------
# Step 2: rasterisation (labels) and pixel areas o(v)
# ----------------------------------------------------------------------------

def snap(xy, log2_res):
    """Fixed-point snap: X = rint(x * 2^(k+8)), ties to even.

    Pixel (i, j) has its centre at (256 i + 128, 256 j + 128) in these units.
    """
    return np.rint(np.asarray(xy, dtype=np.float64) * float(1 << (log2_res + SUBPIXEL_BITS))).astype(np.int64)


def _edge_setup(P, a, b):
    """Order each edge by Y (Y0 < Y1); drop horizontal edges."""
    X0, Y0 = P[a, 0], P[a, 1]
    X1, Y1 = P[b, 0], P[b, 1]
    swap = Y1 < Y0
    X0, X1 = np.where(swap, X1, X0), np.where(swap, X0, X1)
    Y0, Y1 = np.where(swap, Y1, Y0), np.where(swap, Y0, Y1)
    keep = Y1 > Y0
    return X0[keep], Y0[keep], X1[keep], Y1[keep]


def labels_bruteforce(xy, ring_off, ring_idx, ring_region, n_regions, log2_res):
    """The rasterisation rule written out per pixel and per edge (tiny N only).

    Pixel centre (Xc, Yc) counts edge (X0,Y0)-(X1,Y1), Y0 < Y1, iff
    Y0 <= Yc < Y1 and (Xc - X0)(Y1 - Y0) >= (X1 - X0)(Yc - Y0).
    It lies in region v iff v's count is odd; in no region -> background;
    in several -> the smallest id, and the overlap flag is raised.
    Returns (labels [N, N] int, counts [R] int, overlap bool).
    """
    N = 1 << log2_res
    P = snap(xy, log2_res)
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    Xc = (256 * i + 128).ravel()
    Yc = (256 * j + 128).ravel()
    labels = np.full(N * N, BACKGROUND, dtype=np.int64)
    cover = np.zeros(N * N, dtype=np.int64)
    for v, (a, b) in enumerate(region_edges(ring_off, ring_idx, ring_region, n_regions)):
        X0, Y0, X1, Y1 = _edge_setup(P, a, b)
        cnt = np.zeros(N * N, dtype=np.int64)
        for e in range(len(X0)):
            in_row = (Y0[e] <= Yc) & (Yc < Y1[e])
            right = (Xc - X0[e]) * (Y1[e] - Y0[e]) >= (X1[e] - X0[e]) * (Yc - Y0[e])
            cnt += in_row & right
        inside = (cnt % 2) == 1
        labels[inside & (labels == BACKGROUND)] = v
        cover += inside
    counts = np.bincount(labels[labels >= 0], minlength=n_regions)[:n_regions]
    return labels.reshape(N, N), counts, bool((cover > 1).any())


def _floor_div(a, b):
    return np.floor_divide(a, b)


def labels_scanline(xy, ring_off, ring_idx, ring_region, n_regions, log2_res):
    """Same rule as ``labels_bruteforce``, evaluated row by row.

    For an edge crossing row j the pixels that count it are exactly i >= c with
    c = ceil(((X1-X0)(Yc-Y0) + (X0-128)(Y1-Y0)) / (256 (Y1-Y0))), clamped to
    [0, N]; a pixel's count is the number of crossings with c <= i.
    """
    N = 1 << log2_res
    P = snap(xy, log2_res)
    labels = np.full((N, N), BACKGROUND, dtype=np.int64)
    cover = np.zeros((N, N), dtype=np.int64)
    for v, (a, b) in enumerate(region_edges(ring_off, ring_idx, ring_region, n_regions)):
        X0, Y0, X1, Y1 = _edge_setup(P, a, b)
        if len(X0) == 0:
            continue
        # rows j with Y0 <= 256 j + 128 < Y1
        jlo = np.maximum(-_floor_div(-(Y0 - 128), 256), 0)
        jhi = np.minimum(-_floor_div(-(Y1 - 128), 256) - 1, N - 1)
        n_rows = np.maximum(jhi - jlo + 1, 0)
        if n_rows.sum() == 0:
            continue
        e = np.repeat(np.arange(len(X0)), n_rows)
        jj = jlo[e] + (np.arange(n_rows.sum()) - np.repeat(np.cumsum(n_rows) - n_rows, n_rows))
        Yc = 256 * jj + 128
        dY = Y1[e] - Y0[e]
        num = (X1[e] - X0[e]) * (Yc - Y0[e]) + (X0[e] - 128) * dY
        c = -_floor_div(-num, 256 * dY)
        c = np.clip(c, 0, N)
        r0, r1 = int(jj.min()), int(jj.max())
        hist = np.zeros((r1 - r0 + 1, N + 1), dtype=np.int64)
        np.add.at(hist, (jj - r0, c), 1)
        inside = (np.cumsum(hist[:, :N], axis=1) % 2) == 1
        band = labels[r0:r1 + 1]
        band[inside & (band == BACKGROUND)] = v
        cover[r0:r1 + 1] += inside
    counts = np.bincount(labels[labels >= 0], minlength=n_regions)[:n_regions]
    return labels, counts, bool((cover > 1).any())


# ----------------------------------------------------------------------------
# Step 3: piecewise-constant density texture and background density
# ----------------------------------------------------------------------------

def density(labels, counts, values, bdv_scale=1.0, bdv_abs=None):
    """d = s(v)/o(v) inside region v; background = bdv_scale * d0, or the
    given background value bdv_abs (value units per pixel, Eq. (Mb): see
    background_values).

    d0 is the area-weighted mean density of the regions,
    d0 = sum_{v: o(v)>0} s(v) / sum_v o(v), so that with bdv_scale = 1 the
    mean over the whole domain equals d0 (Sec. 4.1 step 3).  Regions without
    pixels carry no density.  Returns (d [N, N], d0, bdv).
    """
    values = np.asarray(values, dtype=np.float64)
    counts = np.asarray(counts, dtype=np.int64)
    has = counts > 0
    tot_o = counts.sum()
    if tot_o == 0:
        return np.ones(labels.shape), 1.0, 1.0
    d0 = values[has].sum() / tot_o
    bdv = bdv_scale * d0 if bdv_abs is None else float(bdv_abs)
    per_region = np.where(has, values / np.maximum(counts, 1), 0.0)
    d = np.where(labels >= 0, per_region[np.maximum(labels, 0)], bdv)
    return d, d0, bdv


def pooled_log_density(labels, counts, values, pool, bdv_scale=1.0):
    """Input of the learned warm start (no counterpart in the paper).

    The density texture of Sec. 4.1 step 3 as d / d0, floored at 1e-6, in
    logarithms, averaged over pool x pool pixel blocks.  Returns
    [N / pool, N / pool], indexed [block row, block column].
    """
    d, d0, _ = density(labels, counts, values, bdv_scale)
    lg = np.log(np.maximum(d / d0, 1e-6))
    N = lg.shape[0]
    m = N // pool
    return lg.reshape(m, pool, m, pool).mean(axis=(1, 3))


# ----------------------------------------------------------------------------
# Step 4: integral images (Sec. 3.1)
# ----------------------------------------------------------------------------

def inims_bruteforce(d):
    """The eight InIms by their definitions, one pixel at a time (tiny N).

    d is indexed [j, i] (row j = y downward, column i = x).
    Axis-aligned (Sec. 3.1): alpha: i'<=i, j'<=j; beta: i'<=i, j'>j;
    gamma: i'>i, j'>j; delta: i'>i, j'<=j.
    Tilted, with u = (i'-i)+(j'-j), w = (i'-i)-(j'-j): alpha_t = top wedge
    {u<=0, w>0}; beta_t = left wedge {u<=0, w<=0}; gamma_t = bottom wedge
    {u>0, w<=0}; delta_t = right wedge {u>0, w>0}.
    """
    N = d.shape[0]
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    out = {k: np.zeros((N, N)) for k in ("a", "b", "g", "d", "at", "bt", "gt", "dt")}
    for j in range(N):
        for i in range(N):
            left, top = ii <= i, jj <= j
            out["a"][j, i] = d[left & top].sum()
            out["b"][j, i] = d[left & ~top].sum()
            out["g"][j, i] = d[~left & ~top].sum()
            out["d"][j, i] = d[~left & top].sum()
            u = (ii - i) + (jj - j)
            w = (ii - i) - (jj - j)
            out["at"][j, i] = d[(u <= 0) & (w > 0)].sum()
            out["bt"][j, i] = d[(u <= 0) & (w <= 0)].sum()
            out["gt"][j, i] = d[(u > 0) & (w <= 0)].sum()
            out["dt"][j, i] = d[(u > 0) & (w > 0)].sum()
    return out


def left_wedge_rows(d):
    """beta_t as a union of row segments: row j' adds the pixels i' <= i - |j'-j|.

    O(N^3); the definition of the left wedge regrouped by rows.
    """
    N = d.shape[0]
    R = np.cumsum(d, axis=1)
    L = np.zeros((N, N))
    for j in range(N):
        for jp in range(N):
            s = abs(jp - j)
            if s < N:
                L[j, s:] += R[jp, :N - s]
    return L


def left_wedge_sweep(d):
    """beta_t by the column sweep L(i,j) = L(i-1,j) + D1 + D2 - d.

    D1(i,j) = d(i,j) + D1(i-1,j-1) and D2(i,j) = d(i,j) + D2(i-1,j+1) are the
    sums along the two diagonal rays that leave (i,j) to the left; the left
    wedge grows by exactly those rays from column i-1 to column i.
    """
    N = d.shape[0]
    L = np.zeros_like(d)
    D1 = np.zeros_like(d)
    D2 = np.zeros_like(d)
    for i in range(N):
        if i == 0:
            D1[:, 0] = d[:, 0]
            D2[:, 0] = d[:, 0]
            L[:, 0] = d[:, 0]
            continue
        D1[:, i] = d[:, i]
        D1[1:, i] += D1[:-1, i - 1]
        D2[:, i] = d[:, i]
        D2[:-1, i] += D2[1:, i - 1]
        L[:, i] = L[:, i - 1] + D1[:, i] + D2[:, i] - d[:, i]
    return L


def inims(d):
    """All eight InIms of Sec. 3.1 from prefix sums (library cumsum).

    alpha = 2-D inclusive prefix S; beta, delta from S's last row / column;
    gamma from Eq. (1).  beta_t = left wedge L (column sweep); with
    A(s) = sum_{i'+j'<=s} d and B(w) = sum_{i'-j'<=w} d:
    alpha_t = A(i+j) - L, gamma_t = B(i-j) - L, delta_t from Eq. (1).
    Returns a dict with the eight [N, N] tables and the total C.  Sums are
    accumulated in d's dtype, so an integer texture gives exact sums.
    """
    N = d.shape[0]
    S = np.cumsum(np.cumsum(d, axis=1), axis=0)
    C = S[-1, -1]
    alpha = S
    beta = S[-1:, :] - S                   # i'<=i, all rows, minus j'<=j
    delta = S[:, -1:] - S                  # j'<=j, all columns, minus i'<=i
    gamma = C - alpha - beta - delta
    L = left_wedge_sweep(d)
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    if np.issubdtype(d.dtype, np.integer):        # exact integer sums
        anti = np.zeros(2 * N - 1, dtype=d.dtype)
        diag = np.zeros(2 * N - 1, dtype=d.dtype)
        np.add.at(anti, (ii + jj).ravel(), d.ravel())
        np.add.at(diag, (ii - jj + N - 1).ravel(), d.ravel())
    else:
        anti = np.bincount((ii + jj).ravel(), weights=d.ravel(), minlength=2 * N - 1)
        diag = np.bincount((ii - jj + N - 1).ravel(), weights=d.ravel(), minlength=2 * N - 1)
    A = np.cumsum(anti)
    B = np.cumsum(diag)
    at = A[ii + jj] - L
    gt = B[ii - jj + N - 1] - L
    dt = C - L - at - gt
    return dict(a=alpha, b=beta, g=gamma, d=delta, at=at, bt=L, gt=gt, dt=dt, C=C, A=A, B=B)


# ----------------------------------------------------------------------------
# Step 5: the map t(x, y; d) (Eq. 2) and the DET displacement (Eq. 3)
# ----------------------------------------------------------------------------

def pixel_centres(N):
    """Sample positions: pixel centres ((i+1/2)/N, (j+1/2)/N), [N, N] each."""
    c = (np.arange(N) + 0.5) / N
    y, x = np.meshgrid(c, c, indexing="ij")
    return x, y


def anchors(x, y):
    """Anchor points q1..q4 of Sec. 3.2 (y downward); arrays of (qx, qy)."""
    lo = y < x
    q1 = (np.where(lo, 1.0, 1.0 - y + x), np.where(lo, 1.0 + y - x, 1.0))
    q3 = (np.where(lo, x - y, 0.0), np.where(lo, 0.0, y - x))
    s = x + y
    lt = s < 1.0
    q2 = (np.where(lt, s, 1.0), np.where(lt, 0.0, s - 1.0))
    q4 = (np.where(lt, 0.0, s - 1.0), np.where(lt, s, 1.0))
    return q1, q2, q3, q4


def transform(I, x, y):
    """Eq. (2): t = (1/2C)(alpha q1 + beta q2 + gamma q3 + delta q4
    + alpha_t (x,1) + beta_t (1,y) + gamma_t (x,0) + delta_t (0,y))."""
    q1, q2, q3, q4 = anchors(x, y)
    C = I["C"]
    tx = (I["a"] * q1[0] + I["b"] * q2[0] + I["g"] * q3[0] + I["d"] * q4[0]
          + I["at"] * x + I["bt"] * 1.0 + I["gt"] * x + I["dt"] * 0.0) / (2.0 * C)
    ty = (I["a"] * q1[1] + I["b"] * q2[1] + I["g"] * q3[1] + I["d"] * q4[1]
          + I["at"] * 1.0 + I["bt"] * y + I["gt"] * 0.0 + I["dt"] * y) / (2.0 * C)
    return tx, ty


def transform_uniform(N):
    """t(x, y; d0) of step 1: Eq. (2) on a constant texture (precomputed once)."""
    x, y = pixel_centres(N)
    return transform(inims(np.ones((N, N))), x, y)


def displacement_field(d, t0=None):
    """Eq. (3) per pixel: t(x,y;d) - t(x,y;d0), returned as ([N,N], [N,N])."""
    N = d.shape[0]
    x, y = pixel_centres(N)
    tx, ty = transform(inims(d), x, y)
    if t0 is None:
        t0 = transform_uniform(N)
    return tx - t0[0], ty - t0[1]


# ----------------------------------------------------------------------------
# Step 6: bilinear interpolation at the vertices and the move
# ----------------------------------------------------------------------------

def bilinear(field, xy):
    """Bilinear interpolation of a pixel-centre field at points xy [V, 2].

    f = x N - 1/2, i0 = clamp(floor f, 0, N-2), a = clamp(f - i0, 0, 1);
    the same along y.  field is indexed [j, i].
    """
    N = field.shape[0]
    xy = np.asarray(xy, dtype=np.float64)
    fx = xy[:, 0] * N - 0.5
    fy = xy[:, 1] * N - 0.5
    i0 = np.clip(np.floor(fx), 0, N - 2).astype(np.int64)
    j0 = np.clip(np.floor(fy), 0, N - 2).astype(np.int64)
    a = np.clip(fx - i0, 0.0, 1.0)
    b = np.clip(fy - j0, 0.0, 1.0)
    f00 = field[j0, i0]
    f01 = field[j0, i0 + 1]
    f10 = field[j0 + 1, i0]
    f11 = field[j0 + 1, i0 + 1]
    return (1 - b) * ((1 - a) * f00 + a * f01) + b * ((1 - a) * f10 + a * f11)


def blend_weight(shape):
    """Step-size reading of the shape parameter: lambda = 1 - shape."""
    return 1.0 - float(shape)


# ----------------------------------------------------------------------------
# Step 7 support: areas (shoelace) and cartographic errors (Sec. 3.3)
# ----------------------------------------------------------------------------

def signed_areas(xy, ring_off, ring_idx, ring_region, n_regions):
    """Per region: sum over its rings of the signed shoelace area."""
    xy = np.asarray(xy, dtype=np.float64)
    out = np.zeros(n_regions)
    for r in range(len(ring_region)):
        idx = np.asarray(ring_idx[ring_off[r]:ring_off[r + 1]], dtype=np.int64)
        x, y = xy[idx, 0], xy[idx, 1]
        out[int(ring_region[r])] += 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    return out


def background_values(values, log2_res, a_min, a_max, t0=0, t1=None):
    """Background value per time step for a map whose area follows its global
    integral (Sec. 4.3, Eq. (Mb)).

    M_i(t) = sum_v s_v(t) is the global integral; over the selected steps
    [t0, t1] its extremes M_min, M_max give the weight
    w(t) = (M_i(t) - M_min) / (M_max - M_min) and the map's area fraction
    A_i(t) = (1 - w) a_min + w a_max (0 < a_min < a_max < 1), from which the
    background mass is M_b(t) = M_i(t) (1 - A_i(t)) / A_i(t), i.e.
    A_i(t) = M_i(t) / (M_i(t) + M_b(t)).  The background value divides M_b(t)
    by the background pixels the target leaves, (1 - A_i(t)) N^2, which is
    the equalised density (M_i + M_b) / N^2: at equal density everywhere the
    map then covers exactly the fraction A_i(t) of the domain.  Readings: w is
    clipped to [0, 1] for steps outside [t0, t1]; with M_max = M_min, w = 1.
    Returns (bdv [T], m_b [T], a_i [T]).
    """
    vals = np.atleast_2d(np.asarray(values, dtype=np.float64))
    T = vals.shape[0]
    t1 = T - 1 if t1 is None else t1
    if not (0.0 < a_min < a_max < 1.0):
        raise ValueError("need 0 < a_min < a_max < 1")
    if not (0 <= t0 <= t1 < T):
        raise ValueError("need 0 <= t0 <= t1 < T")
    m_i = vals.sum(axis=1)
    m_min, m_max = m_i[t0:t1 + 1].min(), m_i[t0:t1 + 1].max()
    w = np.ones(T) if m_max == m_min else np.clip((m_i - m_min) / (m_max - m_min), 0.0, 1.0)
    a_i = (1.0 - w) * a_min + w * a_max
    m_b = m_i * (1.0 - a_i) / a_i
    N = 1 << log2_res
    bdv = m_b / ((1.0 - a_i) * N * N)
    return bdv, m_b, a_i


def interpolate_series(values, frames_per_step):
    """Value series of an animation with frames_per_step frames per time step
    (Sec. 5.5: in-between frames interpolate the statistical data linearly
    between consecutive steps; a cartogram is computed for every frame).
    Frame t f + q (0 <= q < f) holds (1 - q/f) s_t + (q/f) s_{t+1}; the last
    frame is the last step.  Returns [(T - 1) f + 1, R] float64."""
    vals = np.atleast_2d(np.asarray(values, dtype=np.float64))
    T = vals.shape[0]
    f = int(frames_per_step)
    if f < 1:
        raise ValueError("frames_per_step must be >= 1")
    out = []
    for t in range(T - 1):
        for q in range(f):
            w = q / f
            out.append((1.0 - w) * vals[t] + w * vals[t + 1])
    out.append(vals[T - 1])
    return np.stack(out)


def desired_areas(values, counts, bdv, N):
    """w(v) = s(v) / M with M = sum_{o(v)>0} s(v) + BDV * o_bg the total mass
    in the texture: when the density is equalised, area is proportional to
    mass (Sec. 4.3), in unit-square area units."""
    values = np.asarray(values, dtype=np.float64)
    counts = np.asarray(counts, dtype=np.int64)
    o_bg = N * N - counts.sum()
    M = values[counts > 0].sum() + bdv * o_bg
    return values / M


def cartographic_errors(areas, desired):
    """Average and maximum cartographic error epsilon, xi (Sec. 3.3)."""
    o = np.abs(np.asarray(areas, dtype=np.float64))
    w = np.asarray(desired, dtype=np.float64)
    den = np.maximum(o, w)
    e = np.where(den > 0, np.abs(o - w) / np.where(den > 0, den, 1.0), 0.0)
    return float(e.mean()), float(e.max())


# ----------------------------------------------------------------------------
# one iteration (steps 2-6) and the stop rule (step 7, Sec. 4.1 defaults)
# ----------------------------------------------------------------------------

def iterate(xy, mesh_arrays, values, log2_res, shape, bdv_scale=1.0, t0=None,
            raster_xy=None, raster="scanline", bdv_abs=None):
    """One InIm iteration: raster, density, InIms, Eq. (3) field, bilinear,
    blend, move.  Returns (new_xy, info).

    ``raster_xy`` lets a test rasterise a different (e.g. float32) copy of
    the vertices than the one that is moved.
    """
    ring_off, ring_idx, ring_region, R = mesh_arrays
    N = 1 << log2_res
    rxy = xy if raster_xy is None else raster_xy
    fn = labels_scanline if raster == "scanline" else labels_bruteforce
    labels, counts, overlap = fn(rxy, ring_off, ring_idx, ring_region, R, log2_res)
    d, d0, bdv = density(labels, counts, values, bdv_scale, bdv_abs)
    if t0 is None:
        t0 = transform_uniform(N)
    fx, fy = displacement_field(d, t0)
    xy = np.asarray(xy, dtype=np.float64)
    dx = bilinear(fx, xy)
    dy = bilinear(fy, xy)
    lam = blend_weight(shape)
    new = xy + lam * np.stack([dx, dy], 1)
    info = dict(labels=labels, counts=counts, overlap=overlap, d0=d0, bdv=bdv,
                delta=np.stack([dx, dy], 1), field=(fx, fy),
                desired=desired_areas(values, counts, bdv, N))
    return new, info


class StopRule:
    """Stop when xi < xi_stop, when xi has not dropped below its best value
    within the last ``stall_window`` iterations, or after ``max_iters``
    iterations (Sec. 4.1 defaults: 0.01, 32, 512).  eps_stop > 0 adds a stop on
    the average error (used for time-to-epsilon runs)."""

    def __init__(self, max_iters=512, xi_stop=0.01, stall_window=32, eps_stop=0.0):
        self.max_iters, self.xi_stop = max_iters, xi_stop
        self.stall_window, self.eps_stop = stall_window, eps_stop
        self.best, self.since, self.iters = np.inf, 0, 0

    def update(self, eps, xi):
        self.iters += 1
        if xi < self.best:
            self.best, self.since = xi, 0
        else:
            self.since += 1
        if self.iters >= self.max_iters:
            return True
        if self.xi_stop > 0 and xi < self.xi_stop:
            return True
        if self.eps_stop > 0 and eps < self.eps_stop:
            return True
        if self.stall_window > 0 and self.since >= self.stall_window:
            return True
        return False


def run(mesh, values, log2_res, shape=0.5, bdv_scale=1.0, max_iters=512, xi_stop=0.01,
        stall_window=32, mode="direct", eps_stop=0.0, init_xy=None, area_fractions=None):
    """Time-varying driver (Sec. 4.2): for each time step, iterate from the
    original map (direct) or from the previous step's result (cumulative)
    until the stop rule fires.  area_fractions = (a_min, a_max[, t0, t1])
    sets each step's background value by Eq. (Mb) (background_values)
    instead of bdv_scale * d0.  Returns (xy [T, V, 2], stats list)."""
    arrays = (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
    values = np.atleast_2d(np.asarray(values, dtype=np.float64))
    N = 1 << log2_res
    t0 = transform_uniform(N)
    orig = np.asarray(mesh.verts if init_xy is None else init_xy, dtype=np.float64)
    xy = orig.copy()
    bdv_t = background_values(values, log2_res, *area_fractions)[0] if area_fractions is not None else None
    out, stats = [], []
    for t in range(values.shape[0]):
        if mode == "direct" or t == 0:
            xy = orig.copy()
        rule = StopRule(max_iters, xi_stop, stall_window, eps_stop)
        while True:
            xy, info = iterate(xy, arrays, values[t], log2_res, shape, bdv_scale, t0,
                               bdv_abs=None if bdv_t is None else bdv_t[t])
            areas = signed_areas(xy, *arrays)
            eps, xi = cartographic_errors(areas, info["desired"])
            if rule.update(eps, xi):
                break
        out.append(xy.copy())
        stats.append(dict(iters=rule.iters, eps=eps, xi=xi, overlap=info["overlap"]))
    return np.stack(out), stats
