"""GPU parity on block-refined grids beyond two static levels: three levels
(the level recursion nested twice, Sec. 2.1 last paragraph), regrids that
refine and coarsen blocks during the run in 2D and 3D (Sec. 2.6), the paper's
signed refinement sensor (Sec. 3.2.2) and the static drop of the Laplace test
(Sec. 3.1) element by element.  The CUDA library runs through the C ABI
against the FP64 oracle on the same seeded inputs; block statuses, leaf masks,
phases and interface cells are compared bit for bit, fields on leaf cells and,
cell by cell, on the interface and refilled cells.

The refined region is steered between regrids by changing the refinement
distance with lsb_set_params (it applies at the next regrid), so that each run
crosses regrids that both add and remove blocks.

Tolerances: FP32 storage and arithmetic against FP64 after tens of finest
steps give relative L2 errors of 2e-7 to 1e-6 in u on these runs and cell by
cell at most 6e-6 of the velocity scale on interface and refilled cells; the
bounds below (1e-5 field-wide, 1e-4 cell by cell, 1e-5 in rho) leave an order
of magnitude for the accumulation over the run.  The static drop is nearly at
rest (|u| ~ 1e-7 on the coarse level, 4e-6 at most), so relative errors of u
say nothing there; its velocity error is bounded instead by the FP32
resolution of the state, 1e-6 of the largest |rho_hat - 1| (0.31 in the gas at
density ratio 1000), on every level and cell by cell.
"""
import numpy as np
import pytest

from tests.gpu_util import block_status_equal, compare_levels, interface_errors, run_both_schedule

pytestmark = pytest.mark.gpu

U_TOL = 1e-5       # field-wide relative L2 of u on leaf cells
CELL_TOL = 1e-4    # largest |u_g - u_o| on interface / refilled cells over the largest |u_o|
RHO_TOL = 1e-5     # largest |rho_g - rho_o|


def bubble_rect(nx, ny, R, levels, rr=100.0, nu=(0.06, 0.6), g=4e-5, sigma=2e-3, block=(8, 8), seed=8,
                dref=None, regrid_every=3, sensor="band"):
    """2D gas bubble (radius R base cells) at a third of the height of an nx x ny no-slip box."""
    rng = np.random.default_rng(seed)
    r = 2 ** (levels - 1)
    x = np.arange(nx * r) + 0.5
    y = np.arange(ny * r) + 0.5
    X, Y = np.meshgrid(x, y)
    off = rng.random(2)
    xc, yc = (nx / 2 + off[0]) * r, (ny / 3 + off[1]) * r
    phi = R * r - np.sqrt((X - xc) ** 2 + (Y - yc) ** 2)
    return dict(lattice="D2Q9", base=(nx, ny), n_levels=levels, block=block, periodic=(False, False),
                rho_phys=(1.0, 1.0 / rr), nu=nu, sigma=sigma, gravity=(0.0, -g), x_ref=(xc, yc),
                phi0=phi.reshape(-1), refine_dist=dref or [12.0] * (levels - 1), regrid_every=regrid_every,
                sensor=sensor, p_gas0=sigma / (R * r))


def _check(g, s, refilled, u_tol=U_TOL, at_rest=False):
    assert block_status_equal(g, s)
    res = compare_levels(g, s)
    floor = 1e-6 * max(float(np.abs(s.macros(l)[0][s.masks[l][0]] - 1.0).max()) for l in range(len(s.geoms)))
    for r in res:
        assert r["leaf_equal"], r
        assert r["drho_abs"] < RHO_TOL, r
        if at_rest:
            assert r["umax_abs"] < floor, (r, floor)
        else:
            assert r["u"] < u_tol, r
    ie = interface_errors(g, s, refilled)
    assert ie["iface_equal"], ie
    assert ie["drho_max"] < RHO_TOL, ie
    if at_rest:
        assert ie["u_abs_max"] < floor, (ie, floor)
    else:
        assert ie["u_rel_max"] < CELL_TOL, ie
    # phi within 3 cells of the interface (where the link fractions, the curvature fit and
    # the refill read it) to 1e-4; on the rest of the band to 1e-2: far from the interface
    # the reinitialisation meets the kinks of the distance function (the ridge where the
    # fronts of the periodic images meet in the static drop's box), where the HJ-WENO5
    # weights and Godunov's branch are ill-conditioned and FP32 and FP64 part by ~3e-3
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    near = np.abs(s.phi) < 3.0
    assert np.abs(phi_g - s.phi)[near].max() < 1e-4
    assert np.abs(phi_g - s.phi).max() < 1e-2
    assert np.array_equal(g.get("phase").reshape(-1), s.phase[-1].astype(np.uint8))
    print("phi near", float(np.abs(phi_g - s.phi)[near].max()), "phi max", float(np.abs(phi_g - s.phi).max()))
    print("levels", [(r["level"], r["u"], r["drho_abs"]) for r in compare_levels(g, s)], "iface", ie)
    return ie


def test_three_level_bubble_parity():
    """Three levels, regrid every 3 coarse steps; the refined band narrows after step 4
    and widens after step 8, so the regrids at steps 6 and 9 remove and add blocks on
    both finer levels (prolongation, coarsening, the ghost ring at t and t + 1/2 nested
    twice)."""
    case = bubble_rect(24, 48, 4.0, 3, dref=[16.0, 6.0])
    sched = {4: dict(refine_dist=[10.0, 3.0]), 8: dict(refine_dist=[20.0, 8.0])}
    g, s, refilled = run_both_schedule(case, 14, sched)
    assert all(s.masks[l][0].any() for l in range(3)), "every level must hold leaves"
    ie = _check(g, s, refilled)
    assert s.stats["flipped"] > 0 and ie["n_refilled"] > 0
    g.close()


def test_bubble3d_two_level_across_regrids():
    """The 32x32x64 two-level copy of the 3D rising-bubble benchmark with a regrid every
    4 coarse steps: the band narrows before the regrid at step 8 (blocks coarsened)
    and widens before the one at step 12 (blocks prolongated), then two more steps."""
    from paper_2601_05936_gb300 import workloads
    case = workloads.rising_bubble_3d(scale=0.25)
    case["regrid_every"] = 4
    sched = {4: dict(refine_dist=[5.0]), 8: dict(refine_dist=[12.0])}
    g, s, refilled = run_both_schedule(case, 14, sched)
    _check(g, s, refilled)
    g.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_signed_sensor_parity(dim):
    """The paper's AMR-study sensor (gas plus the liquid within d_ref of the interface,
    Sec. 3.2.2): block statuses and fields against the oracle's amr.sensor(..., "signed"),
    with d_ref changed between regrids (3 -> 0 -> 6 cells in 2D; 0 -> 6 -> 1 in 3D), so
    that two regrids change the block layout.  At d_ref = 0 in 2D the interface lies on
    coarse leaves of the liquid side."""
    if dim == 2:
        case = bubble_rect(32, 48, 5.0, 2, dref=[3.0], sensor="signed", regrid_every=2, block=(8, 4))
        sched = {3: dict(refine_dist=[0.0]), 6: dict(refine_dist=[6.0])}
        steps = 9
    else:
        from paper_2601_05936_gb300 import workloads
        case = workloads.paper_box_3d("I", d=8, levels=2, block=(8, 4, 4), nu_floor=0.1, sensor="signed",
                                      refine_dist=0.0, regrid_every=2)
        sched = {3: dict(refine_dist=[6.0]), 6: dict(refine_dist=[1.0])}
        steps = 9
    g, s, refilled = run_both_schedule(case, steps, sched)
    assert block_status_equal(g, s)
    assert (s.status[0] == 2).any() and (s.status[0] == 1).any()
    _check(g, s, refilled)
    g.close()


def test_static_drop_elementwise():
    """The Laplace test (config of Sec. 3.1's static drop: density ratio 1000, viscosity
    ratio 100, seeded sub-cell offset and sigma) at 32x32 base cells on two levels with a
    4-cell band, 100 coarse steps, against the oracle element by element."""
    from paper_2601_05936_gb300 import workloads
    case = workloads.static_drop(n=32, radius_base=6.0, band=4.0)
    g, s, refilled = run_both_schedule(case, 100)
    _check(g, s, refilled, at_rest=True)
    g.close()
