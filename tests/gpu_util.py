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


def run_both_schedule(case, steps, schedule=None):
    """Step the library and the oracle one coarse step at a time on the same case;
    before coarse step k, schedule[k] (a dict of parameter changes, e.g. a new
    refine_dist that the next regrid applies) goes to both sides through
    lsb_set_params and the oracle's case.  Returns (g, s, refilled): refilled marks
    the finest-level cells whose phase changed during the run (oracle)."""
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    case = as_fp32_phi(case)
    g = lsb.Grid(case)
    s = Sim(case)
    refilled = np.zeros(s.geoms[-1].N, dtype=bool)
    cur = dict(case)
    for k in range(steps):
        if schedule and k in schedule:
            cur.update(schedule[k])
            s.case.update(schedule[k])
            g.set_params(cur)
        ph0 = s.phase[-1].copy()
        g.step(1)
        s.step(1)
        refilled |= s.phase[-1] != ph0
    return g, s, refilled


def block_status_equal(g, s, case_idx=0):
    return all(np.array_equal(g.get("blocks", case_idx, l), s.status[l]) for l in range(len(s.geoms)))


def interface_errors(g, s, refilled=None, case_idx=0):
    """Finest level: the interface cells (a cut incoming link) of both sides must be the
    same cells; over them and the refilled cells, the largest |u_g - u_o| relative to
    the largest |u_o| on the level's leaves, and the largest |rho_g - rho_o|."""
    L = len(s.geoms) - 1
    leaf = s.masks[L][0]
    lx, _ = s.cut_links(s.phase[L], leaf)
    iface_o = np.zeros(s.geoms[L].N, dtype=bool)
    iface_o[lx] = True
    tag = g.get("tag", case_idx, L).reshape(-1)
    iface_g = (tag & 2) != 0
    cells = iface_o | (refilled if refilled is not None else False)
    cells &= leaf
    rho_o, u_o = s.macros(L)
    rho_g = g.get("rho", case_idx, L).reshape(-1).astype(np.float64)
    u_g = g.get("u", case_idx, L).reshape(s.D, -1).astype(np.float64)
    uscale = float(np.abs(u_o[:, leaf]).max()) or 1.0
    return dict(iface_equal=bool(np.array_equal(iface_o, iface_g)), n_cells=int(cells.sum()),
                n_refilled=int((refilled & leaf).sum()) if refilled is not None else 0,
                u_rel_max=float(np.abs(u_g[:, cells] - u_o[:, cells]).max()) / uscale if cells.any() else 0.0,
                u_abs_max=float(np.abs(u_g[:, cells] - u_o[:, cells]).max()) if cells.any() else 0.0,
                drho_max=float(np.abs(rho_g[cells] - rho_o[cells]).max()) if cells.any() else 0.0)
