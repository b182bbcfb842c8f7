"""Compare GPU precision-study results with the FP64 oracle (test tooling).

Reads the file written by ``bench.py --precision-study K --study-out F`` (the
input map, the values and the GPU vertices after K iterations in FP32, 64-bit
fixed point and compensated FP32), runs K oracle iterations (float64, the
static algorithm of Sec. 4.1) from the same float32 vertices, and prints the
vertex and area errors of each precision against it as JSON (optionally
writing the oracle's vertices for reuse).

    python -m oracle.compare_precision F [--save-oracle G]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inim_oracle as O


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study")
    ap.add_argument("--save-oracle", default=None)
    ap.add_argument("--oracle", default=None, help="reuse oracle vertices saved by --save-oracle")
    a = ap.parse_args()
    z = np.load(a.study)
    arrays = (z["ring_off"], z["ring_idx"], z["ring_region"], int(z["n_regions"]))
    K = int(z["iterations"])
    xy0 = z["verts"].astype(np.float64)
    if a.oracle:
        ora = np.load(a.oracle)["xy"]
        secs = None
    else:
        t = time.perf_counter()
        t0 = O.transform_uniform(4096)
        ora = xy0.copy()
        for _ in range(K):
            ora, _ = O.iterate(ora, arrays, z["values"].astype(np.float64), 12, 0.5, t0=t0)
        secs = time.perf_counter() - t
        if a.save_oracle:
            np.savez_compressed(a.save_oracle, xy=ora)
    oa = O.signed_areas(ora, *arrays)
    out = {"iterations": K, "oracle_seconds": secs, "oracle_moved_max": float(np.abs(ora - xy0).max())}
    for name in ("fp32", "fix64", "kahan"):
        g = z[f"gpu_{name}"].astype(np.float64)
        ga = O.signed_areas(g, *arrays)
        d = np.abs(g - ora)
        out[name] = {"vertex_max": float(d.max()), "vertex_mean": float(d.mean()),
                     "area_rel_max": float((np.abs(ga - oa) / np.abs(oa)).max()),
                     "area_err_over_mean_area": float(np.abs(ga - oa).max() / np.abs(oa).mean())}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
