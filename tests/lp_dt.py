"""Explicit diffusion limits of the seeded workload recipes, for the tests.

The recipes' time step is a multiple of the explicit limit of the initial state, min over cells
of dx^2 / (2 d D_cell) with the Levermore-Pomraning D_cell (Sect. 2.2).  The recipes hold no
limiter, so the tests take D_cell from the oracle here; the full-size workloads read the limit
from ``golden/explicit_dt.json``, which ``golden/make_explicit_dt.py`` writes with the oracle.
"""
import json
import os

import numpy as np

import oracle
from paper_2104_03968_gb300 import inputs

GOLDEN_DT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "explicit_dt.json")


def _host(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def grid_D(case):
    """The oracle's cell-centred D of a grid recipe's initial state."""
    rho, eps, E = _host(case["rho"]), _host(case["eps"]), _host(case["E"])
    kap = oracle.opacity(case["phys"], rho, eps)
    return oracle.coeffs(case["grid"], case["phys"], E, rho, kap)


def grid_dt(case):
    """Set a grid recipe's dt from the oracle's D of its initial state."""
    g = case["grid"]
    return inputs.with_explicit_dt(case, inputs.explicit_dt(grid_D(case), g["dx"][0] ** 2, g["ndim"]))


def batched_dt(cases):
    for c in cases:
        grid_dt(c)
    return cases


def columns_dt(case):
    """Set a column recipe's per-column dt from the oracle's column D of its initial state."""
    col = {"r_faces": case["r_faces"], "geometry": case["geometry"], "bc": case["bc"]}
    D = np.empty_like(case["E"])
    for j in range(case["E"].shape[0]):
        kap = oracle.opacity(case["phys"], case["rho"][j], case["eps"][j])
        D[j] = oracle.column_coeffs(col, case["phys"], case["E"][j], case["rho"][j], kap,
                                    float(case["bc_lo"][j]), float(case["bc_hi"][j]))
    return inputs.with_explicit_dt(case, inputs.column_explicit_dt(D, case["r_faces"]))


def stored(key):
    """A stored explicit limit (a float, or a list for batched grids and columns)."""
    with open(GOLDEN_DT) as f:
        return json.load(f)[key]
