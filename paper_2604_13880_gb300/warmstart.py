"""Learned warm start: data from the method itself, training, evaluation.

Training pairs come from the InIm iteration itself.  Every training map gets a
64^2 lattice of extra vertices (pixel-cell centres of a 64^2 grid) that belong
to no region: they do not change the raster or the areas, but the gather
moves them with the same displacement field as the map's vertices.  After the
solve, lattice(final) - lattice(start) is the total displacement field on the
lattice (the target, x 10); the input is log(d / d0) of the start map,
average-pooled from the 512^2 texture to the network's input resolution
(64^2, 128^2 or 256^2) by the library's density kernel.  All arithmetic runs in the library's CUDA kernels; this module only
prepares seeded inputs and marshals buffers.
"""
from __future__ import annotations

import multiprocessing as mp
import time

import numpy as np

from . import (Cnn, inim_cnn_get_params, inim_cnn_loss_mean, inim_cnn_train_step, inim_density_pooled,
               inim_map_create, inim_run_series, inim_warmstart_load, params, synth)

FIELD = 64            # lattice / CNN resolution
SCALE = 10.0          # the network predicts SCALE x the displacement
LOG2_RES = 9          # 512^2 density textures


def lattice(m: int = FIELD) -> np.ndarray:
    c = (np.arange(m) + 0.5) / m
    y, x = np.meshgrid(c, c, indexing="ij")
    return np.stack([x.ravel(), y.ravel()], 1)


def training_map(seed: int):
    """50-300 Voronoi regions, log-normal values (seeded)."""
    rng = np.random.default_rng(seed)
    R = int(rng.integers(50, 301))
    mesh = synth.voronoi_map(R, 12 * R, seed=seed)
    vals = rng.lognormal(0.0, 1.0, size=R)
    return mesh, vals


def _gen(seed):
    m, v = training_map(seed)
    return seed, m.verts, m.ring_off, m.ring_idx, m.ring_region, m.n_regions, v


def generate_maps(seeds, workers: int = 0):
    """Maps for the given seeds, in parallel (spawned workers, no CUDA)."""
    seeds = list(seeds)
    if workers <= 1 or len(seeds) < 16:
        res = [_gen(s) for s in seeds]
    else:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_gen, seeds, chunksize=max(1, len(seeds) // (4 * workers)))
    out = []
    for _, verts, off, idx, reg, R, v in res:
        out.append((synth.Mesh(verts, off, idx, reg, R), v))
    return out


def with_lattice(mesh):
    """The map plus the lattice as extra vertices that no ring uses."""
    return synth.Mesh(np.vstack([mesh.verts, lattice()]), mesh.ring_off, mesh.ring_idx, mesh.ring_region,
                      mesh.n_regions)


def pooled_density(m, xy, values, log2_res=LOG2_RES, in_res=FIELD):
    out = np.empty((in_res, in_res), np.float32)
    inim_density_pooled(m, np.ascontiguousarray(xy, dtype=np.float32), log2_res, values,
                        (1 << log2_res) // in_res, out)
    return out


def build_dataset(maps, eps_target=0.02, max_iters=300, batch=64, in_res=FIELD):
    """(inputs [n, in_res, in_res], targets [n, 64, 64, 2], stats) from the method itself."""
    Xs, Y, st = build_dataset_multi(maps, (in_res,), eps_target, max_iters, batch)
    return Xs[in_res], Y, st


def build_dataset_multi(maps, resolutions, eps_target=0.02, max_iters=300, batch=64):
    """One solve per map; the inputs at every resolution in `resolutions`
    ({res: [n, res, res]}), the targets [n, 64, 64, 2], stats."""
    Xs = {r: np.empty((len(maps), r, r), np.float32) for r in resolutions}
    Y = np.empty((len(maps), FIELD, FIELD, 2), np.float32)
    lat = lattice()
    iters = []
    for b0 in range(0, len(maps), batch):
        chunk = maps[b0:b0 + batch]
        handles, series = [], []
        for k, (mesh, vals) in enumerate(chunk):
            ml = with_lattice(mesh)
            h = inim_map_create(ml)
            handles.append(h)
            for r, X in Xs.items():
                X[b0 + k] = pooled_density(h, ml.verts, vals, in_res=r)
            series.append(dict(map=h, values=np.asarray(vals, np.float32)[None],
                               params=params(log2_res=LOG2_RES, shape=0.0, max_iters=max_iters, xi_stop=0.0,
                                               stall_window=0, eps_stop=eps_target)))
        outs, stats, _ = inim_run_series(series)
        for k, (mesh, _) in enumerate(chunk):
            V = mesh.n_verts
            disp = outs[k][0][V:] - lat.astype(np.float32)
            Y[b0 + k] = SCALE * disp.reshape(FIELD, FIELD, 2)
            iters.append(stats[k][0]["iters"])
        for h in handles:
            h.close()
    return Xs, Y, dict(iters_mean=float(np.mean(iters)), iters_max=int(np.max(iters)))


def train(X, Y, epochs=20, batch=64, lr=1e-3, seed=0, log=None):
    """Adam on the mean squared error; X [n, r, r], Y numpy arrays -> trained
    network of input resolution r.  The steps of an epoch are enqueued without
    waiting; the epoch's mean loss is read once at its end."""
    import torch
    net = Cnn(seed, int(X.shape[1]))
    Xd = torch.as_tensor(X, device="cuda")
    Yd = torch.as_tensor(Y, device="cuda")
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    t0 = time.perf_counter()
    hist = []
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device="cuda")
        cur = lr * 0.5 * (1.0 + np.cos(np.pi * ep / epochs))          # cosine decay
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb = Xd.index_select(0, idx).contiguous()
            yb = Yd.index_select(0, idx).contiguous()
            inim_cnn_train_step(net, xb, yb, cur, wait=False)
        hist.append(inim_cnn_loss_mean(net))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f}")
    secs = time.perf_counter() - t0
    return net, dict(loss=hist, seconds=secs, samples_per_s=epochs * (n // batch) * batch / secs)


def evaluate(net, maps, eps_target=0.05, max_iters=512, log2_res=LOG2_RES):
    """Iterations and wall time to reach eps_target, cold vs warm start."""
    import torch
    inim_warmstart_load(inim_cnn_get_params(net), net.in_res)
    handles = [inim_map_create(mesh) for mesh, _ in maps]
    res = {}
    for name, warm in (("cold", 0), ("warm", 1)):
        series = [dict(map=h, values=np.asarray(v, np.float32)[None],
                       params=params(log2_res=log2_res, shape=0.0, max_iters=max_iters, xi_stop=0.0,
                                       stall_window=0, eps_stop=eps_target, warm_start=warm))
                  for h, (_, v) in zip(handles, maps)]
        inim_run_series(series)                           # warm-up (allocations, graphs)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, stats, _ = inim_run_series(series)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        its = [s[0]["iters"] for s in stats]
        res[name] = dict(seconds=dt, iters_mean=float(np.mean(its)), iters_total=int(np.sum(its)),
                         reached=int(sum(s[0]["eps"] < eps_target for s in stats)))
    for h in handles:
        h.close()
    return res


def eps_curve(net, maps, ks, log2_res=LOG2_RES):
    """Mean and median eps after k plain iterations (cold) and after the warm move + k iterations."""
    inim_warmstart_load(inim_cnn_get_params(net), net.in_res)
    handles = [inim_map_create(mesh) for mesh, _ in maps]
    out = {"k": list(ks), "cold_mean": [], "warm_mean": [], "cold_median": [], "warm_median": []}
    for k in ks:
        for name, warm in (("cold", 0), ("warm", 1)):
            series = [dict(map=h, values=np.asarray(v, np.float32)[None],
                           params=params(log2_res=log2_res, shape=0.0, max_iters=k, xi_stop=0.0, stall_window=0,
                                         eps_stop=0.0, warm_start=warm))
                      for h, (_, v) in zip(handles, maps)]
            _, stats, _ = inim_run_series(series)
            e = np.array([s[0]["eps"] for s in stats])
            out[name + "_mean"].append(float(e.mean()))
            out[name + "_median"].append(float(np.median(e)))
    for h in handles:
        h.close()
    return out


def main(argv=None):
    """Train on method-generated fields, then compare warm and cold starts.

    python -m paper_2604_13880_gb300.warmstart --train 10000 --test 256 --epochs 30 --out result.json

    With several --in-res values, one network per input resolution is trained
    on the same solves and evaluated on the same held-out maps.
    """
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=10000)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eps", type=float, nargs="+", default=[0.2, 0.1, 0.05, 0.03])
    ap.add_argument("--curve", type=int, nargs="*", default=[1, 2, 4, 8, 16, 32, 64, 128, 256, 512])
    ap.add_argument("--data-eps", type=float, default=0.02)
    ap.add_argument("--data-iters", type=int, default=300)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-weights", default=None)
    ap.add_argument("--in-res", type=int, nargs="+", default=[FIELD], choices=[64, 128, 256],
                    help="input resolution(s) of the network (the 512^2 density texture pooled to it)")
    ap.add_argument("--batch", type=int, default=64, help="training batch")
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)          # noqa: E731
    t0 = time.perf_counter()
    train_maps = generate_maps(range(50000, 50000 + a.train), a.workers)
    test_maps = generate_maps(range(60000, 60000 + a.test), a.workers)
    t_gen = time.perf_counter() - t0
    log(f"maps generated in {t_gen:.1f} s")
    t0 = time.perf_counter()
    Xs, Y, dstat = build_dataset_multi(train_maps, a.in_res, eps_target=a.data_eps, max_iters=a.data_iters)
    t_data = time.perf_counter() - t0
    log(f"dataset in {t_data:.1f} s: {dstat}")
    Xts, Yt, _ = build_dataset_multi(test_maps, a.in_res, eps_target=a.data_eps, max_iters=a.data_iters)
    import torch
    from . import inim_cnn_forward
    res = dict(train_maps=a.train, test_maps=a.test, epochs=a.epochs, batch=a.batch, seconds_maps=t_gen,
               seconds_dataset=t_data, dataset=dstat, runs={})
    for r in a.in_res:
        net, tstat = train(Xs[r], Y, epochs=a.epochs, batch=a.batch, lr=a.lr, log=log)
        log(f"in_res {r}: trained in {tstat['seconds']:.1f} s ({tstat['samples_per_s']:.0f} samples/s)")
        pred = torch.empty((len(Xts[r]), FIELD, FIELD, 2), dtype=torch.float32, device="cuda")
        inim_cnn_forward(net, torch.as_tensor(Xts[r], device="cuda"), pred)
        pred = pred.cpu().numpy()
        field_err = float(np.linalg.norm(pred - Yt) / np.linalg.norm(Yt))
        evals = {str(e): evaluate(net, test_maps, eps_target=e) for e in a.eps}
        curve = eps_curve(net, test_maps, a.curve) if a.curve else None
        res["runs"][str(r)] = dict(in_res=r, train_loss=tstat["loss"], seconds_train=tstat["seconds"],
                                   train_samples_per_s=tstat["samples_per_s"], test_field_rel_err=field_err,
                                   eval=evals, eps_curve=curve)
        log(json.dumps(res["runs"][str(r)]))
        if a.save_weights:
            np.save(f"{a.save_weights}_{r}.npy", inim_cnn_get_params(net))
        net.close()
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
