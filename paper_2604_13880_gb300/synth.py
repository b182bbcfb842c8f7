"""Seeded synthetic inputs: region maps and per-region value series.

This module builds the inputs that both the CUDA path and the CPU oracle
consume.  It holds none of the cartogram method's arithmetic: it only creates
planar subdivisions of the unit square (Voronoi cells of seeded sites, cell
boundaries as shared polylines) and seeded value series.

Map recipe (stand-in for the paper's real maps, which are not available):
  * R region sites uniform in a disc around the domain centre plus a ring of
    background sites outside it; the Voronoi cells of the region sites are the
    regions, the cells of the background sites become background, so the map
    has an irregular outline surrounded by background (paper Sec. 4.1: the
    regions of interest rarely cover the whole domain).
  * Every Voronoi edge becomes ONE polyline shared by the two cells it
    separates, subdivided so that the whole map has about ``n_verts`` unique
    vertices; shared vertices keep the map contiguous.
  * Optional jitter moves interior polyline vertices perpendicular to the edge
    by U(-j, j) x (sub-segment length), tapered near junctions; a segment
    intersection check rejects (halves) jitter that would self-intersect.
  * The map is scaled isotropically so that its largest extent fits
    [0.05, 0.95] and centred along the other axis (paper Sec. 4.1, defaults).

Coordinates: x to the right, y downward (paper Sec. 3.2), unit square.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    """A region map: unique vertices plus CSR rings.

    verts       float64 [V, 2] vertex positions (x, y), y downward.
    ring_off    int32 [n_rings + 1] CSR offsets into ring_idx.
    ring_idx    int32 [ring_off[-1]] vertex indices; each ring is closed
                implicitly (last vertex connects back to the first).
    ring_region int32 [n_rings] region id of each ring (0 .. n_regions-1).
    n_regions   number of regions R (the background is implicit).
    """

    verts: np.ndarray
    ring_off: np.ndarray
    ring_idx: np.ndarray
    ring_region: np.ndarray
    n_regions: int
    meta: dict = field(default_factory=dict)

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_rings(self) -> int:
        return int(self.ring_region.shape[0])

    def verts_f32(self) -> np.ndarray:
        return np.ascontiguousarray(self.verts, dtype=np.float32)

    def with_verts(self, verts: np.ndarray) -> "Mesh":
        return Mesh(np.asarray(verts, dtype=np.float64), self.ring_off, self.ring_idx,
                    self.ring_region, self.n_regions, dict(self.meta))


# ----------------------------------------------------------------------------
# Voronoi construction (mirror trick: reflecting the sites across the four
# sides of the unit square makes every original cell finite and bounded by it)
# ----------------------------------------------------------------------------

def _voronoi_cells(sites: np.ndarray):
    from scipy.spatial import Voronoi

    n = len(sites)
    x, y = sites[:, 0], sites[:, 1]
    mirrored = np.vstack([
        sites,
        np.stack([-x, y], 1), np.stack([2.0 - x, y], 1),
        np.stack([x, -y], 1), np.stack([x, 2.0 - y], 1),
    ])
    vor = Voronoi(mirrored)
    cells = [list(vor.regions[vor.point_region[i]]) for i in range(n)]
    verts = np.array(vor.vertices, dtype=np.float64)
    # snap coordinates that lie on the square's sides
    for c in (0.0, 1.0):
        verts[np.abs(verts - c) < 1e-9] = c
    verts = np.clip(verts, 0.0, 1.0)
    return verts, cells


def _merge_close(verts: np.ndarray, cells, tol=1e-9):
    """Merge vertices closer than ``tol`` (degenerate co-circular sites)."""
    used = sorted({v for c in cells for v in c})
    pts = verts[used]
    key = np.round(pts / tol).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    remap = {old: int(inv[k]) for k, old in enumerate(used)}
    new_verts = pts[first]
    new_cells = []
    for c in cells:
        r = [remap[v] for v in c]
        out = []
        for v in r:
            if not out or out[-1] != v:
                out.append(v)
        while len(out) > 1 and out[0] == out[-1]:
            out.pop()
        new_cells.append(out)
    return new_verts, new_cells


def _signed_area(p: np.ndarray) -> float:
    x, y = p[:, 0], p[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def _sites(rng, n_regions: int, n_bg: int):
    """Region sites in a disc, background sites in the rest of the square."""
    reg = []
    while len(reg) < n_regions:
        p = rng.uniform(0.0, 1.0, size=(4 * n_regions, 2))
        r = np.hypot(p[:, 0] - 0.5, p[:, 1] - 0.5)
        reg.extend(p[r < 0.40])
    reg = np.array(reg[:n_regions])
    bg = []
    while len(bg) < n_bg:
        p = rng.uniform(0.0, 1.0, size=(8 * n_bg, 2))
        r = np.hypot(p[:, 0] - 0.5, p[:, 1] - 0.5)
        bg.extend(p[r > 0.46])
    bg = np.array(bg[:n_bg])
    return np.vstack([reg, bg])


# ----------------------------------------------------------------------------
# segment intersection check (uniform grid hash)
# ----------------------------------------------------------------------------

def _orient(ax, ay, bx, by, cx, cy):
    return np.sign((bx - ax) * (cy - ay) - (by - ay) * (cx - ax))


def crossing_segment_pairs(pts: np.ndarray, seg: np.ndarray) -> np.ndarray:
    """Pairs of segments (index pairs into ``seg``) that intersect.

    ``seg`` is int [S, 2] of vertex ids; segments sharing a vertex id are not
    tested against each other.  Used to reject jitter that breaks simplicity
    and, in the tests, to check that no fold-over appeared.
    """
    S = len(seg)
    if S < 2:
        return np.zeros((0, 2), np.int64)
    p, q = pts[seg[:, 0]], pts[seg[:, 1]]
    lo, hi = np.minimum(p, q), np.maximum(p, q)
    h = max(float(np.max(hi - lo)), 1e-6) * 1.01
    c0 = np.floor(lo / h).astype(np.int64)
    c1 = np.floor(hi / h).astype(np.int64)
    ids, cells = [], []
    for dx in (0, 1):
        for dy in (0, 1):
            cx, cy = c0[:, 0] + dx, c0[:, 1] + dy
            ok = (cx <= c1[:, 0]) & (cy <= c1[:, 1])
            ids.append(np.nonzero(ok)[0])
            cells.append(cx[ok] * 1_000_003 + cy[ok])
    ids = np.concatenate(ids)
    cells = np.concatenate(cells)
    order = np.lexsort((ids, cells))
    ids, cells = ids[order], cells[order]
    pairs = []
    k = 1
    while True:
        same = cells[k:] == cells[:-k] if k < len(cells) else np.zeros(0, bool)
        if not same.any():
            break
        pairs.append(np.stack([ids[:-k][same], ids[k:][same]], 1))
        k += 1
    if not pairs:
        return np.zeros((0, 2), np.int64)
    pr = np.unique(np.sort(np.concatenate(pairs), axis=1), axis=0)
    a, b = pr[:, 0], pr[:, 1]
    share = ((seg[a, 0] == seg[b, 0]) | (seg[a, 0] == seg[b, 1]) |
             (seg[a, 1] == seg[b, 0]) | (seg[a, 1] == seg[b, 1]))
    pr = pr[~share]
    if len(pr) == 0:
        return pr
    a, b = pr[:, 0], pr[:, 1]
    P1, Q1, P2, Q2 = p[a], q[a], p[b], q[b]
    o1 = _orient(P1[:, 0], P1[:, 1], Q1[:, 0], Q1[:, 1], P2[:, 0], P2[:, 1])
    o2 = _orient(P1[:, 0], P1[:, 1], Q1[:, 0], Q1[:, 1], Q2[:, 0], Q2[:, 1])
    o3 = _orient(P2[:, 0], P2[:, 1], Q2[:, 0], Q2[:, 1], P1[:, 0], P1[:, 1])
    o4 = _orient(P2[:, 0], P2[:, 1], Q2[:, 0], Q2[:, 1], Q1[:, 0], Q1[:, 1])
    hit = (o1 * o2 <= 0) & (o3 * o4 <= 0)
    colin = (o1 == 0) & (o2 == 0)
    if colin.any():
        bl1, bh1 = np.minimum(P1, Q1), np.maximum(P1, Q1)
        bl2, bh2 = np.minimum(P2, Q2), np.maximum(P2, Q2)
        ov = np.all((bl1 <= bh2) & (bl2 <= bh1), axis=1)
        hit = np.where(colin, ov, hit)
    return pr[hit]


def mesh_segments(mesh: Mesh) -> np.ndarray:
    """Unique undirected boundary segments of a mesh as vertex-id pairs."""
    segs = []
    for r in range(mesh.n_rings):
        idx = mesh.ring_idx[mesh.ring_off[r]:mesh.ring_off[r + 1]]
        segs.append(np.stack([idx, np.roll(idx, -1)], 1))
    s = np.sort(np.concatenate(segs), axis=1)
    return np.unique(s, axis=0)


# ----------------------------------------------------------------------------
# map generator
# ----------------------------------------------------------------------------

def voronoi_map(n_regions: int, n_verts: int, seed: int, jitter: float = 0.0,
                n_bg: int | None = None, fit=(0.05, 0.95)) -> Mesh:
    """Seeded Voronoi region map with about ``n_verts`` unique vertices."""
    rng = np.random.default_rng(seed)
    if n_bg is None:
        n_bg = max(8, n_regions // 3)
    sites = _sites(rng, n_regions, n_bg)
    gverts, cells = _voronoi_cells(sites)
    gverts, cells = _merge_close(gverts, cells)
    cells = cells[:n_regions]
    # orient every ring counter-clockwise in (x right, y down) coordinates,
    # i.e. negative shoelace sum; only consistency matters
    for k, c in enumerate(cells):
        if _signed_area(gverts[c]) > 0:
            cells[k] = c[::-1]
    # keep only vertices used by region cells, renumber
    used = np.array(sorted({v for c in cells for v in c}), dtype=np.int64)
    ren = -np.ones(len(gverts), dtype=np.int64)
    ren[used] = np.arange(len(used))
    gverts = gverts[used]
    cells = [[int(ren[v]) for v in c] for c in cells]

    # undirected graph edges
    ekeys = {}
    for c in cells:
        for a, b in zip(c, c[1:] + c[:1]):
            key = (min(a, b), max(a, b))
            ekeys.setdefault(key, len(ekeys))
    edges = np.array(sorted(ekeys, key=ekeys.get), dtype=np.int64)
    E = len(edges)
    ea, eb = gverts[edges[:, 0]], gverts[edges[:, 1]]
    elen = np.hypot(*(eb - ea).T)
    budget = max(n_verts - len(gverts), 0)
    seg_target = elen.sum() / max(budget + E, 1)
    k_int = np.maximum(np.rint(elen / seg_target).astype(np.int64) - 1, 0)

    # smallest angle at each graph vertex between incident edges
    dirs = {}
    for e, (a, b) in enumerate(edges):
        d = gverts[b] - gverts[a]
        dirs.setdefault(a, []).append(np.arctan2(d[1], d[0]))
        dirs.setdefault(b, []).append(np.arctan2(-d[1], -d[0]))
    min_ang = np.full(len(gverts), np.pi)
    for v, angs in dirs.items():
        if len(angs) > 1:
            a = np.sort(np.mod(angs, 2 * np.pi))
            gaps = np.diff(np.concatenate([a, a[:1] + 2 * np.pi]))
            min_ang[v] = gaps.min()
    ang_scale = np.minimum(1.0, np.sin(np.minimum(min_ang[edges[:, 0]], min_ang[edges[:, 1]])
                                       .clip(0, np.pi / 2)) / 0.7)

    # interior points, jitter, rejection by halving the jitter of bad edges
    offs = np.concatenate([[0], np.cumsum(k_int)])
    n_int = int(offs[-1])
    t_par = np.concatenate([np.arange(1, k + 1) / (k + 1) for k in k_int]) if n_int else np.zeros(0)
    e_of = np.repeat(np.arange(E), k_int)
    m_of = np.concatenate([np.arange(1, k + 1) for k in k_int]).astype(np.int64) if n_int else np.zeros(0, np.int64)
    base = ea[e_of] + t_par[:, None] * (eb - ea)[e_of]
    nrm = np.stack([-(eb - ea)[:, 1], (eb - ea)[:, 0]], 1) / np.maximum(elen, 1e-300)[:, None]
    segl = elen / (k_int + 1)
    taper = np.minimum(1.0, np.minimum((m_of - 1) / 2.0, (k_int[e_of] - m_of) / 2.0)).clip(0.0, 1.0)
    u = rng.uniform(-1.0, 1.0, size=n_int)
    scale = np.full(E, float(jitter))

    def build(scale_e):
        amp = u * scale_e[e_of] * segl[e_of] * taper * ang_scale[e_of]
        pts = np.vstack([gverts, base + amp[:, None] * nrm[e_of]])
        return pts

    def rings_from(pts):
        ring_idx, ring_off = [], [0]
        for c in cells:
            ring = []
            for a, b in zip(c, c[1:] + c[:1]):
                e = ekeys[(min(a, b), max(a, b))]
                inner = np.arange(offs[e], offs[e + 1]) + len(gverts)
                if a > b:
                    inner = inner[::-1]
                ring.append(a)
                ring.extend(inner.tolist())
            ring_idx.extend(ring)
            ring_off.append(len(ring_idx))
        return np.array(ring_idx, np.int32), np.array(ring_off, np.int32)

    ring_idx, ring_off = rings_from(None)
    pts = build(scale)
    if jitter > 0 and n_int:
        seg_edge = None
        for _ in range(6):
            m = Mesh(pts, ring_off, ring_idx, np.arange(n_regions, dtype=np.int32), n_regions)
            segs = mesh_segments(m)
            bad = crossing_segment_pairs(pts, segs)
            if len(bad) == 0:
                break
            if seg_edge is None:
                # map a vertex id to its graph edge (interior vertices only)
                seg_edge = np.full(len(pts), -1, np.int64)
                seg_edge[len(gverts):] = e_of
            bv = segs[bad.ravel()].ravel()
            be = np.unique(seg_edge[bv])
            be = be[be >= 0]
            scale[be] *= 0.5
            pts = build(scale)
        else:
            scale[:] = 0.0
            pts = build(scale)

    # isotropic fit of the map into [fit0, fit1], centred
    lo, hi = pts.min(0), pts.max(0)
    ext = float((hi - lo).max())
    s = (fit[1] - fit[0]) / ext
    ctr = 0.5 * (lo + hi)
    pts = (pts - ctr) * s + 0.5
    mesh = Mesh(pts, ring_off, ring_idx, np.arange(n_regions, dtype=np.int32), n_regions,
                meta=dict(seed=seed, jitter=jitter, n_bg_sites=n_bg))
    return mesh


def square_map(rects, n_regions=None) -> Mesh:
    """Map of axis-aligned rectangles [(x0, y0, x1, y1), ...]; test helper."""
    verts, idx, off = [], [], [0]
    for (x0, y0, x1, y1) in rects:
        b = len(verts)
        verts += [(x0, y0), (x0, y1), (x1, y1), (x1, y0)]
        idx += [b, b + 1, b + 2, b + 3]
        off.append(len(idx))
    R = len(rects) if n_regions is None else n_regions
    return Mesh(np.array(verts, np.float64), np.array(off, np.int32), np.array(idx, np.int32),
                np.arange(len(rects), dtype=np.int32), R)


# ----------------------------------------------------------------------------
# values
# ----------------------------------------------------------------------------

def lognormal_values(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).lognormal(0.0, sigma, size=n)


def loguniform_values(n: int, seed: int, decades: float = 6.0) -> np.ndarray:
    return 10.0 ** np.random.default_rng(seed).uniform(0.0, decades, size=n)


def random_walk_values(n: int, T: int, seed: int, sigma: float = 0.2, sigma0: float = 1.0) -> np.ndarray:
    """[T, n] log-normal random walk: log s_{t+1} = log s_t + sigma * N(0, 1)."""
    rng = np.random.default_rng(seed)
    ls = np.empty((T, n))
    ls[0] = rng.normal(0.0, sigma0, size=n)
    for t in range(1, T):
        ls[t] = ls[t - 1] + sigma * rng.normal(0.0, 1.0, size=n)
    return np.exp(ls)


# ----------------------------------------------------------------------------
# the synthetic workloads
# ----------------------------------------------------------------------------

def single_step_workload():
    """32 Voronoi regions, ~2k vertices, 256^2, 20 iterations, shape 0.5."""
    mesh = voronoi_map(32, 2000, seed=1)
    vals = lognormal_values(32, seed=1001)[None, :]
    return dict(name="voronoi32_v2k_res256_it20", mesh=mesh, values=vals, log2_res=8,
                iters=20, shapes=(0.5,))


def time_varying_workload(n_regions=200, n_verts=50_000, log2_res=10, T=24):
    """200 jittered Voronoi regions, ~50k vertices, 1024^2, 24 random-walk steps."""
    mesh = voronoi_map(n_regions, n_verts, seed=2, jitter=0.3)
    vals = random_walk_values(n_regions, T, seed=102, sigma=0.2)
    return dict(name=f"voronoi{n_regions}_v{n_verts // 1000}k_res{1 << log2_res}_T{T}_it50",
                mesh=mesh, values=vals, log2_res=log2_res, iters=50, shapes=(0.25, 0.5, 0.75))


def batched_workload(B=64, base_seed=3000, n_verts_per_region=60):
    """B independent maps: N from {256..2048}, 20-500 regions, log-normal values."""
    maps = []
    for b in range(B):
        rng = np.random.default_rng(base_seed + b)
        k = int(rng.integers(8, 12))
        R = int(rng.integers(20, 501))
        mesh = voronoi_map(R, R * n_verts_per_region, seed=base_seed + b)
        vals = rng.lognormal(0.0, 1.0, size=R)
        maps.append(dict(mesh=mesh, values=vals[None, :], log2_res=k))
    return maps


def precision_workload(n_regions=2000, n_verts=500_000, log2_res=12):
    """2000 regions, ~500k vertices, 4096^2, values log-uniform over 6 decades."""
    mesh = voronoi_map(n_regions, n_verts, seed=4)
    vals = loguniform_values(n_regions, seed=1004, decades=6.0)[None, :]
    return dict(name=f"voronoi{n_regions}_v{n_verts // 1000}k_res{1 << log2_res}_it100",
                mesh=mesh, values=vals, log2_res=log2_res, iters=100, shapes=(0.5,))
