"""CPU oracle of the cartogram quality measures of Sec. 3.3 (geographic
distortion): topology distortion tau, shape distortion (normalised Hamming
distance) and relative position error R.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's ``smoke()`` check and
the benchmark's CPU-baseline leg may import this module.  It shares no code
with the CUDA path and imports nothing from it.

Plain numpy / scipy in float64 and exact integers.  Readings where Sec. 3.3
leaves the representation open (listed in the design notes): adjacency and
the polygons' superposition are taken on the label rasters of the original
map and the cartogram at the same resolution (4-neighbour pixel adjacency,
background excluded; a region's polygon = its pixels); barycentres are the
area centroids of the region polygons (shoelace moments over all rings).

Pins (``tests/test_oracle_quality.py``): closed forms on constructed maps --
identical maps give 0 for all three measures; separating two adjacent
regions gives tau = 1; a translated region has shape distortion 0 and a
doubled one 3/4; a global rotation by theta gives R = |theta| / pi; on
random 8 x 8 rasters the shape distortion equals the minimum over every
translation enumerated with explicit pixel sets.
"""
from __future__ import annotations

import numpy as np
from scipy import signal


def raster_adjacency(labels):
    """Pairs (u, v), u < v, of regions with 4-neighbouring pixels in a label
    raster (labels < 0 = background, not a region)."""
    lab = np.asarray(labels)
    pairs = set()
    for a, b in ((lab[:, :-1], lab[:, 1:]), (lab[:-1, :], lab[1:, :])):
        m = (a >= 0) & (b >= 0) & (a != b)
        u, v = np.minimum(a[m], b[m]), np.maximum(a[m], b[m])
        pairs.update(zip(u.tolist(), v.tolist()))
    return pairs


def topology_distortion(labels_map, labels_cart):
    """tau = 1 - |E_c & E_m| / |E_c | E_m| over the region adjacencies of the
    cartogram (E_c) and of the original map (E_m) (Sec. 3.3); 0 when neither
    has an adjacency."""
    em, ec = raster_adjacency(labels_map), raster_adjacency(labels_cart)
    union = em | ec
    return 0.0 if not union else 1.0 - len(em & ec) / len(union)


def _crop(mask):
    """A non-empty boolean mask cut to its bounding box, as integers."""
    rows, cols = np.flatnonzero(mask.any(1)), np.flatnonzero(mask.any(0))
    return mask[rows[0]:rows[-1] + 1, cols[0]:cols[-1] + 1].astype(np.int64)


def shape_distortion(labels_map, labels_cart, n_regions):
    """Per region, ||P_m sym-diff P_c|| / ||P_m union P_c|| minimised over
    relative translations by whole pixels (Sec. 3.3), with P = the region's
    pixels.  For overlap o between the superimposed polygons of areas |m|,
    |c| the value is (|m| + |c| - 2 o) / (|m| + |c| - o), which falls as o
    grows: the minimum is at the translation with the largest overlap, the
    maximum of the masks' cross-correlation (exact integer counts).
    Returns (per-region values [n_regions], mean over regions present in
    both rasters); a region missing from one raster scores 1."""
    lm, lc = np.asarray(labels_map), np.asarray(labels_cart)
    out = np.ones(n_regions)
    present = np.zeros(n_regions, bool)
    for v in range(n_regions):
        mm, mc = (lm == v), (lc == v)
        am, ac = int(mm.sum()), int(mc.sum())
        if am == 0 or ac == 0:
            continue
        present[v] = True
        # the empty border of a mask adds no overlap at any translation: the
        # correlation of the masks cut to their bounding boxes has the same
        # maximum
        o = int(signal.correlate2d(_crop(mc), _crop(mm), mode="full", boundary="fill").max())
        out[v] = (am + ac - 2 * o) / (am + ac - o)
    mean = float(out[present].mean()) if present.any() else 0.0
    return out, mean


def barycenters(xy, ring_off, ring_idx, ring_region, n_regions):
    """Area centroid of every region's polygon (all rings; holes oriented
    against their outer ring): C = sum over edges of (p_a + p_b) cross(p_a,
    p_b) / (6 A), A = the signed shoelace area."""
    xy = np.asarray(xy, dtype=np.float64)
    a2 = np.zeros(n_regions)
    cx = np.zeros(n_regions)
    cy = np.zeros(n_regions)
    for r in range(len(ring_off) - 1):
        idx = np.asarray(ring_idx[ring_off[r]:ring_off[r + 1]])
        p, q = xy[idx], xy[np.roll(idx, -1)]
        cr = p[:, 0] * q[:, 1] - q[:, 0] * p[:, 1]
        v = ring_region[r]
        a2[v] += cr.sum()
        cx[v] += ((p[:, 0] + q[:, 0]) * cr).sum()
        cy[v] += ((p[:, 1] + q[:, 1]) * cr).sum()
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.stack([cx / (3.0 * a2), cy / (3.0 * a2)], 1)


def _angle(u, v):
    """Signed angle from vector u to vector v in [-pi, pi)."""
    a = np.arctan2(u[..., 0] * v[..., 1] - u[..., 1] * v[..., 0], (u * v).sum(-1))
    return np.where(a >= np.pi, a - 2.0 * np.pi, a)


def relative_position_error(bary_map, bary_cart):
    """R = 1 / (pi |V| (|V| - 1)) sum over ordered pairs u != v of
    |angle(b_c(u, v), b_m(u, v))|, b(u, v) = the vector between the
    barycentres of u and v (Sec. 3.3)."""
    bm, bc = np.asarray(bary_map, np.float64), np.asarray(bary_cart, np.float64)
    n = len(bm)
    if n < 2:
        return 0.0
    dm = bm[None, :, :] - bm[:, None, :]
    dc = bc[None, :, :] - bc[:, None, :]
    off = ~np.eye(n, dtype=bool)
    return float(np.abs(_angle(dc[off], dm[off])).sum() / (np.pi * n * (n - 1)))
