"""Write paper_2007_00745_gb300/data/boundary_points.json: centres near the Mandelbrot boundary.

Renders the 1024 x 1024 full view re[-2, 1] x im[-1.5, 1.5] at iterMax 65536
with the CPU oracle only, keeps the pixels whose count is in [50, 65536) and
stores a seeded subsample of their c values.  The batched and served
workloads (and the tile-cost model's training windows) draw their centres
from this list.  Run from the repository root:  python oracle/make_boundary_manifest.py

Test infrastructure like the rest of oracle/: the package only reads the
JSON file it writes (input data, no method arithmetic), never this script.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

WINDOW = (-2.0, 1.0, -1.5, 1.5)
SIDE, ITER_MAX, KEEP, SEED = 1024, 65536, 4096, 200700745


def main():
    img = oracle.render(WINDOW, SIDE, SIDE, ITER_MAX)
    cx, cy = oracle.pixel_map(WINDOW, SIDE, SIDE)
    ii, jj = np.nonzero((img >= 50) & (img < ITER_MAX))
    rng = np.random.default_rng(SEED)
    pick = np.sort(rng.choice(len(ii), size=min(KEEP, len(ii)), replace=False))
    pts = [[float(cx[jj[k]]), float(cy[ii[k]])] for k in pick]
    out = {"window": WINDOW, "side": SIDE, "iter_max": ITER_MAX, "count_range": [50, ITER_MAX],
           "candidates": int(len(ii)), "seed": SEED, "points": pts}
    path = os.path.join(ROOT, "paper_2007_00745_gb300", "data", "boundary_points.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, len(pts), "of", len(ii))


if __name__ == "__main__":
    main()
