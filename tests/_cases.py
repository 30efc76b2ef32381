"""Seeded operator cases for the parity tests: inputs from ``synth``, the
geometry and the expected values from the oracle only."""
import numpy as np

import oracle
from paper_2506_20994_gb300 import synth

GKEYS = ("g11", "g22", "g33", "g12", "g13", "g23")


def operator_case(dims, lx, seed=0, h1_const=None):
    """dict with u, h1, g11..g23 (E,lx,lx,lx) fp64, dx, dxt and the oracle w."""
    nx, ny, nz = dims
    v = synth.box_vertices(nx, ny, nz, seed=seed)
    geo = oracle.box_geometry(v, lx)
    shape = geo["jac"].shape
    u = synth.uniform(shape, seed=seed + 1)
    h1 = (np.full(shape, float(h1_const)) if h1_const is not None
          else synth.uniform(shape, seed=seed + 2, lo=0.5, hi=2.0))
    dx, dxt = oracle.d_buffers(lx)
    case = {"u": u, "h1": h1, "dx": dx, "dxt": dxt, "lx": lx, "vertices": v}
    for k in GKEYS:
        case[k] = geo[k]
    case["w"] = oracle.ax_helm(u, dx, dxt, h1, *[geo[k] for k in GKEYS], lx)
    return case


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
