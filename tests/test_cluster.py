"""The nine-bubble cluster (Sec. 3.2, last example): the workload's geometry on the CPU, and
the CUDA path against the oracle on a small copy (d = 4 finest cells), one and two levels."""
import numpy as np
import pytest


def test_cluster_geometry():
    """Nine separate gas regions, each a sphere of diameter d at its stated centre, none
    touching another or a wall."""
    ndimage = pytest.importorskip("scipy.ndimage")
    from paper_2601_05936_gb300 import workloads
    d = 8
    case = workloads.bubble_cluster_3d(d=d)
    nx, ny, nz = case["base"]
    assert (nx, ny, nz) == (10 * d, 10 * d, 20 * d)
    gas = (np.asarray(case["phi0"]) >= 0).reshape(nz, ny, nx)
    lab, n = ndimage.label(gas)
    assert n == 9
    vol = 4.0 / 3.0 * np.pi * (d / 2) ** 3
    cents = np.asarray(case["centres"])
    for k in range(1, n + 1):
        zz, yy, xx = np.nonzero(lab == k)
        assert abs(len(xx) / vol - 1.0) < 0.15, (k, len(xx), vol)
        c = np.array([xx.mean(), yy.mean(), zz.mean()]) + 0.5
        assert np.min(np.linalg.norm(cents - c, axis=1)) < 0.5
        assert xx.min() > 0 and yy.min() > 0 and zz.min() > 0 and xx.max() < nx - 1 and yy.max() < ny - 1
    dist = np.linalg.norm(cents[:, None, :] - cents[None, :, :], axis=2) + np.eye(9) * 1e9
    assert dist.min() > 2.0 * d  # 2.1 d with the default spacing


def test_cluster_refined_region_holds_every_bubble():
    """With two levels the oracle's sensor refines around all nine interfaces."""
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import workloads
    case = workloads.bubble_cluster_3d(d=4, levels=2)
    s = Sim(case)
    gas = np.asarray(case["phi0"]) >= 0
    assert s.masks[-1][0][gas].all()  # every gas cell is a leaf of the finest level


@pytest.mark.gpu
@pytest.mark.parametrize("levels,steps", [(1, 4), (2, 2)])
def test_cluster_parity(levels, steps):
    from paper_2601_05936_gb300 import workloads
    from tests.gpu_util import compare_levels, run_both
    case = workloads.bubble_cluster_3d(d=4, levels=levels)
    g, s = run_both(case, steps)
    for r in compare_levels(g, s):
        assert r["leaf_equal"], r
        assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    assert np.abs(phi_g - s.phi).max() < 1e-4
    assert np.array_equal(g.get("phase").reshape(-1), s.phase[-1].astype(np.uint8))
    g.close()
