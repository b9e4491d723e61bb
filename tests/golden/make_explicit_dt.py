#!/usr/bin/env python
"""Writes explicit_dt.json: the explicit diffusion limit of each full-size workload recipe.

The limit is min over cells of dx^2 / (2 d D_cell), with D_cell the Levermore-Pomraning
coefficient (Sect. 2.2) of the recipe's initial state.  Only the oracle computes D here (its
opacity and coefficient functions on the numpy fields of ``inputs``); the recipes and the
benchmark then take the stored numbers as an input.  Run from the repository root:

    python tests/golden/make_explicit_dt.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import lp_dt  # noqa: E402
from paper_2104_03968_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "explicit_dt.json")


def main():
    out = {"_what": "explicit diffusion limit min(dx^2 / (2 d D_cell)) of each recipe's initial state, "
                    "D_cell from the oracle's Levermore-Pomraning coefficients; written by make_explicit_dt.py"}
    for n, seed in ((128, 1), (256, 2), (512, 2)):
        t = time.time()
        case = inputs.lognormal_3d(n=n, seed=seed)
        lp_dt.grid_dt(case)
        out[f"lognormal_3d_{n}_seed{seed}"] = case["dt_exp"]
        print(f"lognormal {n}^3: dt_exp {case['dt_exp']:.6e} (thick {case['dt_exp_thick']:.6e}) "
              f"{time.time() - t:.0f} s", flush=True)
        del case
    cases = lp_dt.batched_dt(inputs.batched_2d(ngrids=512, seed=3))
    out["batched_2d_512_seed3"] = [c["dt_exp"] for c in cases]
    print("batched 2-D: done", flush=True)
    case = lp_dt.columns_dt(inputs.wind_columns(ncol=4096, ncell=2048, seed=4))
    out["wind_columns_4096x2048_seed4"] = [float(v) for v in case["dt_exp"]]
    print("columns: done", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
