"""Helpers shared by the GPU parity tests: run the same case on the CUDA
library and on the oracle and compare fields on leaf cells."""
import numpy as np


def as_fp32_phi(case):
    c = dict(case)
    c["phi0"] = np.asarray(case["phi0"], np.float32).astype(np.float64)
    return c


def run_both(case, steps):
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    case = as_fp32_phi(case)
    g = lsb.Grid(case)
    g.step(steps)
    s = Sim(case)
    s.step(steps)
    return g, s


def rel_l2(a, b):
    den = np.sqrt((b ** 2).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / (den if den > 0 else 1.0))


def compare_levels(g, s, case_idx=0):
    """Per level: leaf mask equality and rel-L2 errors of rho-1 and u on leaf cells."""
    out = []
    for l, geom in enumerate(s.geoms):
        leaf_o = s.masks[l][0]
        tag = g.get("tag", case_idx, l).reshape(-1)
        leaf_g = (tag & 64) != 0
        rho_g = g.get("rho", case_idx, l).reshape(-1).astype(np.float64)
        u_g = g.get("u", case_idx, l).reshape(geom.D, -1).astype(np.float64)
        rho_o, u_o = s.macros(l)
        m = leaf_o
        out.append(dict(level=l, leaf_equal=bool(np.array_equal(leaf_o, leaf_g)),
                        drho=rel_l2(rho_g[m] - 1, rho_o[m] - 1), u=rel_l2(u_g[:, m], u_o[:, m]),
                        drho_abs=float(np.abs(rho_g[m] - rho_o[m]).max()) if m.any() else 0.0,
                        umax_abs=float(np.abs(u_g[:, m] - u_o[:, m]).max()) if m.any() else 0.0))
    return out
