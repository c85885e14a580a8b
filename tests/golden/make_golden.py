"""Writes the stored expected values under tests/golden/.

closed_forms.json: constants of the mathematics, computed here with `math`:
  erf3_squared = erf(3 / sqrt 2)^2, the mass of a 2-D normal inside its
  axis-aligned 3-sigma box when rho = 0 (the Algorithm-1 box window of GSASR,
  arXiv 2501.06838, Sec. 3.1, with the 3-sigma footprint).
oracle_small.json: a regression fixture, a few pixels of a small render written
  by the FP64 oracle (oracle/ only; nothing from the CUDA path).
Run from the repository root: python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gs_synthetic as S  # noqa: E402
import oracle  # noqa: E402


def main():
    cf = {"erf3_squared": math.erf(3 / math.sqrt(2)) ** 2,
          "source": "erf(3/sqrt(2))^2: captured mass of the 3-sigma box, rho = 0"}
    with open(os.path.join(HERE, "closed_forms.json"), "w") as f:
        json.dump(cf, f, indent=1)

    rng = np.random.default_rng(1234)
    n = 16
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    p = {"mx": f32(rng.uniform(0, 12, n)), "my": f32(rng.uniform(0, 10, n)),
         "sx": f32(rng.uniform(0.3, 1.8, n)), "sy": f32(rng.uniform(0.3, 1.8, n)),
         "rho": f32(rng.uniform(-0.9, 0.9, n)), "rgb": f32(rng.uniform(0, 1, (n, 3))),
         "alpha": f32(rng.uniform(0, 1, n))}
    g = S.GaussianSet(np.stack([p["mx"], p["my"]], 1), np.stack([p["sx"], p["sy"]], 1), p["rho"],
                      p["rgb"], p["alpha"], lr_h=10, lr_w=12, ref_grid_m=0)
    view = dict(lr_h=10, lr_w=12, out_h=27, out_w=32, scale=2.7, trunc_k=3.0, norm=0)
    img = oracle.render(g, S.View(**view))
    ys = [0, 5, 13, 20, 26]
    xs = [0, 7, 16, 24, 31]
    out = {"params": {k: v.tolist() for k, v in p.items()}, "view": view,
           "probe_y": ys, "probe_x": xs,
           "values": img[:, ys, xs].tolist(),
           "source": "FP64 oracle render (regression fixture, written by make_golden.py)"}
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
