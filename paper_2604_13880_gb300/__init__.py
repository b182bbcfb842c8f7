"""GB300 integral-image (InIm) contiguous cartograms.

Python binding of the C ABI in ``include/inim.h`` (same function names).  The
functions take numpy arrays (host memory) or torch tensors (host or CUDA) and
only marshal arguments; the cartogram iteration itself (rasterisation,
density, integral images, Eq. (2)-(3) displacement, blend, move, areas and
errors) runs in the CUDA kernels of ``libinim.so``.  Nothing here falls back
to a CPU implementation: a missing library raises.

Typical use::

    from paper_2604_13880_gb300 import synth, inim_map_create, inim_run, params
    mesh = synth.voronoi_map(200, 50_000, seed=2, jitter=0.3)
    m = inim_map_create(mesh)
    out, stats = inim_run(m, values_T_by_R, params(log2_res=10, shape=0.5))
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (INIM_CUMULATIVE, INIM_DIRECT, INIM_E_ARG, INIM_E_CAPACITY, INIM_E_CUDA,  # noqa: F401
                   INIM_E_STATE, INIM_E_TIMEOUT, INIM_E_VALUE, INIM_FIX64, INIM_FORM_FUSED, INIM_FORM_PLAIN,
                   INIM_FP32, INIM_KAHAN, InimError, inim_job, inim_params, inim_series, inim_step_stats)

__all__ = [
    "params", "inim_params_default", "inim_status_string", "inim_map_create", "inim_map_destroy",
    "inim_map_info", "inim_run", "inim_run_batch", "inim_raster", "inim_inims", "inim_displacement",
    "inim_iterate", "inim_areas", "inim_background_values", "inim_interpolate_values", "inim_run_dynamic",
    "inim_quality", "Map",
]


def inim_params_default() -> inim_params:
    p = inim_params()
    _lib.load().inim_params_default(ctypes.byref(p))
    return p


def params(**kw) -> inim_params:
    """Defaults of Sec. 4.1 with keyword overrides (log2_res, shape, ...)."""
    p = inim_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def inim_status_string(status: int) -> str:
    return _lib.load().inim_status_string(status).decode()


class Map:
    """Owner of an ``inim_map*`` handle."""

    def __init__(self, handle, n_verts, n_regions):
        self.handle = handle
        self.n_verts = n_verts
        self.n_regions = n_regions

    def close(self):
        if self.handle:
            _lib.load().inim_map_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def inim_map_create(mesh=None, *, xy=None, ring_off=None, ring_idx=None, ring_region=None,
                    n_regions=None) -> Map:
    """Create a map from a ``synth.Mesh`` or from the raw arrays."""
    if mesh is not None:
        xy, ring_off, ring_idx, ring_region, n_regions = (
            mesh.verts, mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
    xy = np.ascontiguousarray(xy, dtype=np.float32)
    ring_off = np.ascontiguousarray(ring_off, dtype=np.int32)
    ring_idx = np.ascontiguousarray(ring_idx, dtype=np.int32)
    ring_region = np.ascontiguousarray(ring_region, dtype=np.int32)
    h = ctypes.c_void_p()
    lib = _lib.load()
    _lib.check(lib.inim_map_create(xy.ctypes.data, xy.shape[0], ring_off.ctypes.data, ring_region.shape[0],
                                   ring_idx.ctypes.data, ring_region.ctypes.data, int(n_regions), 0,
                                   ctypes.byref(h)), "inim_map_create")
    return Map(h.value, xy.shape[0], int(n_regions))


def inim_map_destroy(m: Map) -> None:
    m.close()


def inim_map_info(m: Map):
    a = [ctypes.c_int32() for _ in range(4)]
    _lib.check(_lib.load().inim_map_info(m.handle, *[ctypes.byref(x) for x in a]), "inim_map_info")
    return dict(n_verts=a[0].value, n_regions=a[1].value, n_rings=a[2].value, n_edges=a[3].value)


def _stats_array(T):
    return (inim_step_stats * T)()


def inim_run(m: Map, values, p: inim_params, init_xy=None, out_xy=None, stream=None):
    """Time-varying run (values [T, R]); returns (out_xy [T, V, 2], stats list)."""
    lib = _lib.load()
    if isinstance(values, np.ndarray) or not hasattr(values, "data_ptr"):
        values = np.ascontiguousarray(np.atleast_2d(values), dtype=np.float32)
    T = int(values.shape[0]) if values.ndim == 2 else 1
    if init_xy is not None and isinstance(init_xy, np.ndarray):
        init_xy = np.ascontiguousarray(init_xy, dtype=np.float32)
    if out_xy is None:
        out_xy = np.empty((T, m.n_verts, 2), np.float32)
    st = _stats_array(T)
    s = stream if stream is not None else _lib.stream_of(values, init_xy, out_xy)
    status = _lib.check(lib.inim_run(m.handle, _lib.ptr(values), T, ctypes.byref(p), _lib.ptr(init_xy),
                                     _lib.ptr(out_xy), st, s), "inim_run")
    return out_xy, [x.as_dict() for x in st], status


def inim_run_dynamic(m: Map, values, p: inim_params, a_min: float, a_max: float, t0: int = 0, t1: int = -1,
                     init_xy=None, out_xy=None, stream=None):
    """Time-varying run with dynamic area (Eq. (Mb)): host values [T, R];
    returns (out_xy [T, V, 2], stats list, status) like inim_run."""
    lib = _lib.load()
    values = np.ascontiguousarray(np.atleast_2d(values), dtype=np.float32)
    T = int(values.shape[0])
    if init_xy is not None and isinstance(init_xy, np.ndarray):
        init_xy = np.ascontiguousarray(init_xy, dtype=np.float32)
    if out_xy is None:
        out_xy = np.empty((T, m.n_verts, 2), np.float32)
    st = _stats_array(T)
    s = stream if stream is not None else _lib.stream_of(init_xy, out_xy)
    status = _lib.check(lib.inim_run_dynamic(m.handle, _lib.ptr(values), T, ctypes.byref(p), float(a_min),
                                             float(a_max), t0, t1, _lib.ptr(init_xy), _lib.ptr(out_xy), st, s),
                        "inim_run_dynamic")
    return out_xy, [x.as_dict() for x in st], status


def inim_run_batch(jobs, stream=None):
    """jobs: list of dicts(map=Map, values, params, init_xy=None, out_xy=None)."""
    lib = _lib.load()
    n = len(jobs)
    arr = (inim_job * n)()
    stats = _stats_array(n)
    keep = []
    outs = []
    for k, j in enumerate(jobs):
        vals = j["values"]
        if isinstance(vals, np.ndarray) or not hasattr(vals, "data_ptr"):
            vals = np.ascontiguousarray(vals, dtype=np.float32).ravel()
        init = j.get("init_xy")
        if init is not None and isinstance(init, np.ndarray):
            init = np.ascontiguousarray(init, dtype=np.float32)
        out = j.get("out_xy")
        if out is None:
            out = np.empty((j["map"].n_verts, 2), np.float32)
        keep += [vals, init]
        outs.append(out)
        arr[k].map = j["map"].handle
        arr[k].values = _lib.ptr(vals)
        arr[k].init_xy = _lib.ptr(init)
        arr[k].out_xy = _lib.ptr(out)
        arr[k].params = j["params"]
        arr[k].stats = ctypes.pointer(stats[k])
    status = _lib.check(lib.inim_run_batch(arr, n, stream), "inim_run_batch")
    return outs, [s.as_dict() for s in stats], status


def inim_interpolate_values(values, frames_per_step: int):
    """[(T - 1) f + 1, R] float32 values of an animation with f frames per
    time step of the [T, R] series (Sec. 5.5); host arithmetic."""
    vals = np.ascontiguousarray(values, dtype=np.float32)
    vals = vals.reshape(1, -1) if vals.ndim == 1 else vals
    T, R = vals.shape
    out = np.empty(((T - 1) * frames_per_step + 1, R), np.float32)
    _lib.check(_lib.load().inim_interpolate_values(_lib.ptr(vals), T, R, frames_per_step, _lib.ptr(out)),
               "inim_interpolate_values")
    return out


def inim_quality(m: Map, xy_cart, log2_res: int, xy_map=None, stream=None):
    """Quality measures of Sec. 3.3 of the cartogram at xy_cart against the map
    at xy_map (None: the map's own vertices), rasterised at 2^log2_res.
    Returns (dict of tau, shape, rel_pos, adj_map, adj_cart, adj_both,
    n_present; per-region shape distortion [R] float64)."""
    def prep(a):
        if a is None or hasattr(a, "data_ptr"):
            return a
        return np.ascontiguousarray(a, dtype=np.float32)
    xc, xm = prep(xy_cart), prep(xy_map)
    out = _lib.inim_quality_out()
    per = np.empty(m.n_regions, np.float64)
    _lib.check(_lib.load().inim_quality(m.handle, _lib.ptr(xm), _lib.ptr(xc), log2_res, ctypes.byref(out),
                                        _lib.ptr(per), stream if stream is not None else _lib.stream_of(xc, xm)),
               "inim_quality")
    res = {k: getattr(out, k) for k in ("tau", "shape", "rel_pos", "adj_map", "adj_cart", "adj_both", "n_present")}
    return res, per


def inim_background_values(values, log2_res: int, a_min: float, a_max: float, t0: int = 0, t1: int = -1):
    """Background value and area fraction of every time step of a [T, R]
    value series with dynamic area (Sec. 4.3, Eq. (Mb)); host arithmetic.
    Returns (bdv [T], area_fraction [T]) as float64 arrays."""
    vals = np.ascontiguousarray(values, dtype=np.float32)
    vals = vals.reshape(1, -1) if vals.ndim == 1 else vals
    T, R = vals.shape
    bdv = np.empty(T, np.float64)
    frac = np.empty(T, np.float64)
    _lib.check(_lib.load().inim_background_values(_lib.ptr(vals), T, R, log2_res, float(a_min), float(a_max),
                                                  t0, t1, _lib.ptr(bdv), _lib.ptr(frac)),
               "inim_background_values")
    return bdv, frac


def inim_raster(m: Map, xy, log2_res: int, labels, counts, stream=None) -> int:
    """Device buffers: xy [V,2] f32, labels [N,N] u16 (int16 tensor), counts [R+1] i32."""
    ov = ctypes.c_int32(0)
    _lib.check(_lib.load().inim_raster(m.handle, _lib.ptr(xy), log2_res, _lib.ptr(labels), _lib.ptr(counts),
                                       ctypes.byref(ov), stream or _lib.stream_of(xy)), "inim_raster")
    return ov.value


def inim_inims(density, log2_res: int, precision: int, frac_bits: int, S, T, A, B, stream=None) -> None:
    _lib.check(_lib.load().inim_inims(_lib.ptr(density), log2_res, precision, frac_bits, _lib.ptr(S),
                                      _lib.ptr(T), _lib.ptr(A), _lib.ptr(B), stream or _lib.stream_of(density)),
               "inim_inims")


def inim_inims_noalloc(density, log2_res: int, S, T, A, B, stream=None) -> None:
    """FP32 integral images without any device allocation (N <= 1024).

    For callers that cannot allocate device memory (another framework owns
    the device pool, or a loop that cannot afford cudaMalloc's
    synchronisation); the library keeps its working memory in a fixed array.
    Calls that overlap on the GPU share that array and race.
    """
    _lib.check(_lib.load().inim_inims_noalloc(_lib.ptr(density), log2_res, _lib.ptr(S), _lib.ptr(T), _lib.ptr(A),
                                              _lib.ptr(B), stream or _lib.stream_of(density)),
               "inim_inims_noalloc")


def inim_displacement(density, log2_res: int, precision: int, xy, delta, stream=None) -> None:
    n = int(xy.shape[0])
    _lib.check(_lib.load().inim_displacement(_lib.ptr(density), log2_res, precision, _lib.ptr(xy), n,
                                             _lib.ptr(delta), stream or _lib.stream_of(density)),
               "inim_displacement")


def inim_iterate(m: Map, xy, values, p: inim_params, n_iters: int, stream=None):
    st = inim_step_stats()
    status = _lib.check(_lib.load().inim_iterate(m.handle, _lib.ptr(xy), _lib.ptr(values), ctypes.byref(p),
                                                 n_iters, ctypes.byref(st), stream or _lib.stream_of(xy)),
                        "inim_iterate")
    return st.as_dict(), status


def inim_areas(m: Map, xy, areas, stream=None) -> None:
    _lib.check(_lib.load().inim_areas(m.handle, _lib.ptr(xy), _lib.ptr(areas), stream or _lib.stream_of(xy)),
               "inim_areas")


def inim_profile_stages(reps: int = 20):
    """{stage name: average ms per launch} for the most recent batch."""
    lib = _lib.load()
    ms = (ctypes.c_float * 16)()
    n = ctypes.c_int32(0)
    _lib.check(lib.inim_profile_stages(reps, ms, 16, ctypes.byref(n)), "inim_profile_stages")
    return {lib.inim_stage_name(i).decode(): ms[i] for i in range(n.value)}


def inim_launch_count() -> int:
    return int(_lib.load().inim_launch_count())


def inim_set_scan_tile(log2_res: int, precision: int, large: int, band_rows: int, cols_per_thread: int,
                       threads: int) -> None:
    _lib.check(_lib.load().inim_set_scan_tile(log2_res, precision, large, band_rows, cols_per_thread, threads),
               "inim_set_scan_tile")


def inim_get_scan_tile(log2_res: int, precision: int = 0, large: int = 1):
    v = [ctypes.c_int32() for _ in range(3)]
    _lib.check(_lib.load().inim_get_scan_tile(log2_res, precision, large, *[ctypes.byref(x) for x in v]),
               "inim_get_scan_tile")
    return dict(band_rows=v[0].value, cols_per_thread=v[1].value, threads=v[2].value)


def inim_autotune_scan(job_array, reps: int = 5) -> None:
    """job_array: a ctypes (inim_job * n) array (see inim_run_batch)."""
    _lib.check(_lib.load().inim_autotune_scan(job_array, len(job_array), reps), "inim_autotune_scan")


def inim_run_series(series, stream=None):
    """series: list of dicts(map=Map, values [T, R], params, init_xy=None, out_xy=None).

    Returns (list of out_xy [T, V, 2], list of stats lists, status)."""
    lib = _lib.load()
    n = len(series)
    arr = (inim_series * n)()
    keep, outs, stats = [], [], []
    for k, x in enumerate(series):
        vals = x["values"]
        if isinstance(vals, np.ndarray) or not hasattr(vals, "data_ptr"):
            vals = np.ascontiguousarray(np.atleast_2d(vals), dtype=np.float32)
        T = int(vals.shape[0])
        init = x.get("init_xy")
        if init is not None and isinstance(init, np.ndarray):
            init = np.ascontiguousarray(init, dtype=np.float32)
        out = x.get("out_xy")
        if out is None:
            out = np.empty((T, x["map"].n_verts, 2), np.float32)
        st = _stats_array(T)
        keep += [vals, init]
        outs.append(out)
        stats.append(st)
        arr[k].map = x["map"].handle
        arr[k].values = _lib.ptr(vals)
        arr[k].T = T
        arr[k].init_xy = _lib.ptr(init)
        arr[k].out_xy = _lib.ptr(out)
        arr[k].params = x["params"]
        arr[k].stats = st
    status = _lib.check(lib.inim_run_series(arr, n, stream), "inim_run_series")
    return outs, [[s.as_dict() for s in st] for st in stats], status


def inim_set_persistent(enable: bool) -> None:
    _lib.load().inim_set_persistent(1 if enable else 0)


PERSISTENT_PHASES = ("crossings", "rows", "density", "scan_phase1", "scan_carry", "scan_phase3", "gather_move",
                     "areas_errors")


def inim_set_area_overlap(enable: bool) -> None:
    """Each iteration's area kernel beside the next raster (the default), or
    in sequence after the move."""
    _lib.check(_lib.load().inim_set_area_overlap(1 if enable else 0), "inim_set_area_overlap")


def inim_set_single_pass_scan(enable: bool) -> None:
    """Large batches scan in one pass, or with three kernels (the default)."""
    _lib.check(_lib.load().inim_set_single_pass_scan(1 if enable else 0), "inim_set_single_pass_scan")


TIMELINE_KERNELS = ("crossings", "rows", "scan_phase1", "scan_carry", "scan_phase3", "gather_move", "areas_errors")


def inim_timeline(enable: bool) -> None:
    """Record the first-block start and last-block end of every kernel launch of
    batches built from now on (global-timer ns); False switches it off."""
    _lib.check(_lib.load().inim_timeline(1 if enable else 0), "inim_timeline")


def inim_timeline_read():
    """(start_ns, end_ns): int64 arrays [8, 128] (kernel, launch slot), 0 where
    nothing ran; clears the record."""
    n = 8 * 128
    a, b = (ctypes.c_uint64 * n)(), (ctypes.c_uint64 * n)()
    _lib.check(_lib.load().inim_timeline_read(a, b, n), "inim_timeline_read")
    return (np.frombuffer(a, dtype=np.uint64).astype(np.int64).reshape(8, 128),
            np.frombuffer(b, dtype=np.uint64).astype(np.int64).reshape(8, 128))


def inim_set_wait_cap(spins: int) -> None:
    """Polls of a device-side barrier wait before it gives up (INIM_E_TIMEOUT); <= 0: the default."""
    _lib.check(_lib.load().inim_set_wait_cap(int(spins)), "inim_set_wait_cap")


def inim_persistent_phase_times(enable: bool):
    """Toggle phase timing of persistent launches; returns the ms per phase so far."""
    ms = (ctypes.c_double * 8)()
    _lib.check(_lib.load().inim_persistent_phase_times(1 if enable else 0, ms, 8), "inim_persistent_phase_times")
    return dict(zip(PERSISTENT_PHASES, list(ms)))


# ---------------------------------------------------------------------------
# learned warm start (not part of the paper): density input, network, loading
# ---------------------------------------------------------------------------
def inim_density_pooled(m: Map, xy, log2_res: int, values, pool: int, out, stream=None) -> None:
    """out[(N/pool)^2] = block averages of log(d / d0) of the map at xy (host or device arrays)."""
    if isinstance(values, np.ndarray) or not hasattr(values, "data_ptr"):
        values = np.ascontiguousarray(values, dtype=np.float32)
    _lib.check(_lib.load().inim_density_pooled(m.handle, _lib.ptr(xy), log2_res, _lib.ptr(values), pool,
                                               _lib.ptr(out), stream or _lib.stream_of(xy, out)),
               "inim_density_pooled")


class Cnn:
    """Owner of an inim_cnn handle (encoder-decoder, in_res^2 -> 64^2 x 2)."""

    def __init__(self, seed: int = 0, in_res: int = 64):
        lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check_cnn(lib.inim_cnn_create_res(seed, in_res, ctypes.byref(h)), "inim_cnn_create_res")
        self.handle = h.value
        self.n_params = int(lib.inim_cnn_num_params(self.handle))
        self.in_res = int(lib.inim_cnn_input_res(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().inim_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def inim_cnn_create(seed: int = 0, in_res: int = 64) -> Cnn:
    return Cnn(seed, in_res)


def inim_cnn_destroy(c: Cnn) -> None:
    c.close()


def inim_cnn_num_params(c: Cnn = None) -> int:
    return int(_lib.load().inim_cnn_num_params(c.handle if c else None))


def inim_cnn_get_params(c: Cnn, out=None):
    if out is None:
        out = np.empty(c.n_params, np.float32)
    _lib.check_cnn(_lib.load().inim_cnn_get_params(c.handle, _lib.ptr(out), c.n_params), "inim_cnn_get_params")
    return out


def inim_cnn_set_params(c: Cnn, blob) -> None:
    if isinstance(blob, np.ndarray) or not hasattr(blob, "data_ptr"):
        blob = np.ascontiguousarray(blob, dtype=np.float32)
    _lib.check_cnn(_lib.load().inim_cnn_set_params(c.handle, _lib.ptr(blob), c.n_params), "inim_cnn_set_params")


def _cnn_shapes(c: Cnn, x, y) -> None:
    """The C entry points take only the batch size: the binding checks the rest
    of both shapes, so that no call reads or writes past a tensor."""
    B = int(x.shape[0])
    if tuple(x.shape) != (B, c.in_res, c.in_res):
        raise ValueError(f"input of shape {tuple(x.shape)}; this network takes [B, {c.in_res}, {c.in_res}]")
    if tuple(y.shape) != (B, 64, 64, 2):
        raise ValueError(f"field of shape {tuple(y.shape)}; expected [{B}, 64, 64, 2]")
    for t in (x, y):
        if hasattr(t, "is_contiguous") and not t.is_contiguous():
            raise ValueError("tensors must be contiguous")


def inim_cnn_forward(c: Cnn, x, y, stream=None) -> None:
    """x [B, in_res, in_res] f32, y [B, 64, 64, 2] f32; device tensors."""
    _cnn_shapes(c, x, y)
    _lib.check_cnn(_lib.load().inim_cnn_forward(c.handle, _lib.ptr(x), int(x.shape[0]), _lib.ptr(y),
                                                stream or _lib.stream_of(x)), "inim_cnn_forward")


def inim_cnn_gradients(c: Cnn, x, y, grads=None, stream=None) -> float:
    """Mean squared error of the prediction for x against y; its gradient into grads [n_params]."""
    _cnn_shapes(c, x, y)
    if grads is not None and int(np.prod(grads.shape)) != c.n_params:
        raise ValueError(f"gradient buffer of {int(np.prod(grads.shape))} values; expected {c.n_params}")
    loss = ctypes.c_float()
    _lib.check_cnn(_lib.load().inim_cnn_gradients(c.handle, _lib.ptr(x), _lib.ptr(y), int(x.shape[0]),
                                                  ctypes.byref(loss), _lib.ptr(grads), stream or _lib.stream_of(x)),
                   "inim_cnn_gradients")
    return loss.value


def inim_cnn_train_step(c: Cnn, x, y, lr: float, stream=None, wait: bool = True):
    """One Adam step; returns the batch loss before the step (wait=True), or
    None without waiting for the step (wait=False; see inim_cnn_loss_mean)."""
    _cnn_shapes(c, x, y)
    loss = ctypes.c_float()
    _lib.check_cnn(_lib.load().inim_cnn_train_step(c.handle, _lib.ptr(x), _lib.ptr(y), int(x.shape[0]), lr,
                                                   ctypes.byref(loss) if wait else None,
                                                   stream or _lib.stream_of(x)),
                   "inim_cnn_train_step")
    return loss.value if wait else None


def inim_cnn_loss_mean(c: Cnn) -> float:
    """Mean loss of the training steps since the previous call (waits for them)."""
    m = ctypes.c_double()
    _lib.check_cnn(_lib.load().inim_cnn_loss_mean(c.handle, ctypes.byref(m)), "inim_cnn_loss_mean")
    return m.value


def inim_warmstart_load(blob, in_res: int = 64) -> None:
    """Install the network used by params(warm_start=1) (an f32 parameter blob
    of a network with the given input resolution)."""
    blob = np.ascontiguousarray(blob, dtype=np.float32)
    _lib.check_cnn(_lib.load().inim_warmstart_load_res(blob.ctypes.data, blob.nbytes, int(in_res)),
                   "inim_warmstart_load_res")
