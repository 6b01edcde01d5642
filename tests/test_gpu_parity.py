"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element on leaf cells.

Tolerances: FP32 arithmetic against FP64 gives relative L2 errors of order
1e-6 on these short runs; the stratified channel carries the 1e-5 bound after
1000 steps; phases, cut masks and block statuses are compared bit-exactly (both
sides classify the same float32 level set).
"""
import numpy as np
import pytest

from tests.gpu_util import as_fp32_phi, compare_levels, interface_errors, rel_l2, run_both, run_both_schedule

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _channel(lat, H=16, nu=1 / 6, G=1e-5, wall_top=None, nx=32):
    D = 2 if lat == "D2Q9" else 3
    base = (nx, H) if D == 2 else (nx, H, 4)
    block = (32, 8) if D == 2 else (32, 4, 4)
    n = int(np.prod(base))
    wall = np.zeros((2 * D, D))
    if wall_top is not None:
        wall[3, 0] = wall_top
    bf = np.zeros(D)
    bf[0] = G
    return dict(lattice=lat, base=base, block=block, periodic=(True, False) if D == 2 else (True, False, True),
                rho_phys=(1.0, 1.0), nu=(nu, nu), body_force=bf, wall_u=wall, phi0=-np.ones(n), n_ext=0,
                reinit_every=0, ls_active=False)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_single_phase_channel(lat):
    g, s = run_both(_channel(lat), 200)
    r = compare_levels(g, s)[0]
    assert r["leaf_equal"]
    assert r["u"] < TOL and r["drho_abs"] < 1e-6, r


def test_moving_wall_channel():
    g, s = run_both(_channel("D2Q9", G=0.0, wall_top=1e-3), 200)
    r = compare_levels(g, s)[0]
    assert r["u"] < TOL, r


def test_stratified_channel_1000_steps():
    from paper_2601_05936_gb300 import workloads
    case = workloads.stratified_channel()
    g, s = run_both(case, 1000)
    r = compare_levels(g, s)[0]
    assert r["u"] < TOL, r
    ph_g = g.get("phase").reshape(-1)
    assert np.array_equal(ph_g, s.phase[-1].astype(np.uint8))


def _bubble2d(N=48, R=9.0, levels=1, sigma=5e-3, rr=10.0, nu=(0.1, 0.1), g=0.0, block=(32, 8), seed=7):
    rng = np.random.default_rng(seed)
    r = 2 ** (levels - 1)
    n = N * r
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    off = rng.random(2)
    xc, yc = (N / 2 + off[0]) * r, (N / 2 + off[1]) * r
    phi = R * r - np.sqrt((X - xc) ** 2 + (Y - yc) ** 2)
    return dict(lattice="D2Q9", base=(N, N), n_levels=levels, block=block, periodic=(False, False),
                rho_phys=(1.0, 1.0 / rr), nu=nu, sigma=sigma, gravity=(0.0, -g), x_ref=(xc, yc),
                phi0=phi.reshape(-1), refine_dist=[12.0] * (levels - 1), regrid_every=5 if levels > 1 else 0)


def test_static_bubble_levelset_parity():
    case = _bubble2d()
    g, s = run_both(case, 40)
    r = compare_levels(g, s)[0]
    assert r["u"] < 1e-4 and r["drho"] < 1e-4, r
    ie = interface_errors(g, s)
    assert ie["iface_equal"] and ie["u_rel_max"] < 1e-3 and ie["drho_max"] < 1e-5, ie
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    assert np.abs(phi_g - s.phi).max() < 1e-4
    assert np.array_equal(g.get("phase").reshape(-1), s.phase[-1].astype(np.uint8))


def test_rising_bubble_with_refill_parity():
    case = _bubble2d(N=40, R=7.0, rr=100.0, nu=(0.06, 0.6), g=2e-5, sigma=2e-3)
    g, s, refilled = run_both_schedule(case, 60)
    r = compare_levels(g, s)[0]
    assert s.stats["flipped"] > 0 and refilled.any()
    assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    # cell by cell on the interface cells and on every cell refilled during the run
    ie = interface_errors(g, s, refilled)
    assert ie["iface_equal"] and ie["u_rel_max"] < 1e-3 and ie["drho_max"] < 1e-5, ie
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    assert np.abs(phi_g - s.phi).max() < 1e-4


def test_two_level_bubble_parity():
    case = _bubble2d(N=64, R=6.0, levels=2, rr=100.0, nu=(0.06, 0.6), g=2e-5, sigma=2e-3)
    case["refine_dist"] = [8.0]
    g, s = run_both(case, 12)
    res = compare_levels(g, s)
    assert all(s.masks[l][0].any() for l in range(2)), "both levels must hold leaves"
    for r in res:
        assert r["leaf_equal"], r
        assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    for l in range(2):
        assert np.array_equal(g.get("blocks", 0, l), s.status[l]), l
    ie = interface_errors(g, s)
    assert ie["iface_equal"] and ie["u_rel_max"] < 1e-3 and ie["drho_max"] < 1e-5, ie


@pytest.mark.parametrize("lattice,n,block", [("D2Q9", (48, 24), (8, 8)), ("D3Q19", (12, 8, 12), (4, 4, 4))])
def test_two_level_coarse_cut_links_parity(lattice, n, block):
    """Interface partly on coarse leaves (refinement distance below a cell): a link into
    the other phase on a coarser level takes plain bounce-back, as in the oracle."""
    from paper_2601_05936_gb300 import workloads
    case = workloads.adjoint_window(lattice, n=n, levels=2, block=block, refine_dist=0.2)
    g, s = run_both(case, 12)
    assert s.stats["coarse_cut"] > 0
    for r in compare_levels(g, s):
        assert r["leaf_equal"], r
        assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    tag0 = g.get("tag", 0, 0).reshape(-1)
    assert ((tag0 & 128) != 0).any()


def test_cut_masks_bit_exact_on_random_level_sets():
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    rng = np.random.default_rng(11)
    for lat, base, block in (("D2Q9", (32, 16), (32, 8)), ("D3Q19", (32, 8, 8), (32, 4, 4))):
        D = len(base)
        for trial in range(3):
            phi = rng.standard_normal(int(np.prod(base))).astype(np.float32)
            phi[rng.random(phi.size) < 0.05] = 0.0  # exact zeros count as gas
            case = dict(lattice=lat, base=base, block=block, periodic=tuple([trial % 2 == 0] * D),
                        rho_phys=(1.0, 0.5), nu=(0.1, 0.1), phi0=phi.astype(np.float64), ls_active=False)
            g = lsb.Grid(case)
            s = Sim(case)
            leaf = s.masks[0][0]
            lx, lk = s.cut_links(s.phase[0], leaf)
            want = np.zeros(s.geoms[0].N, dtype=np.uint32)
            np.bitwise_or.at(want, lx, (1 << lk).astype(np.uint32))
            got = g.get("cutmask").reshape(-1)
            assert np.array_equal(got, want), (lat, trial)
            assert np.array_equal(g.get("phase").reshape(-1), s.phase[0].astype(np.uint8))
            g.close()


def test_curvature_matches_oracle_fit():
    from oracle import levelset
    case = _bubble2d(N=40, R=8.3)
    case = as_fp32_phi(case)
    from paper_2601_05936_gb300 import lsb
    from oracle.sim import Sim
    g = lsb.Grid(case)
    s = Sim(case)
    lx, lk = s.cut_links(s.phase[0], s.masks[0][0])
    cells = np.unique(lx)
    _, kap, _, _ = levelset.fit_geometry(s.geoms[0], s.phi, cells)
    kg = g.get("kappa").reshape(-1)[cells]
    assert np.abs(kg - kap).max() < 1e-5
