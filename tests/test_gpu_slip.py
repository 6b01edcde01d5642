"""Slip walls on the GPU against the oracle (forward step and adjoint).

The oracle's slip walls are pinned as mirror planes (test_oracle_slip.py);
here the library must reproduce them: a bubble rising between slip side walls
with the level set live (2D), the adjoint window with slip side walls that
its wall film meets (reflected links into the other phase), single-level in
2D and 3D and on two levels, and the frozen-interface adjoint on those
windows.  Tolerances are those of the other parity tests.
"""
import numpy as np
import pytest

from gpu_util import as_fp32_phi, compare_levels, interface_errors, rel_l2, run_both, run_both_schedule

pytestmark = pytest.mark.gpu


def _slip_window(lattice, n, levels=1, **kw):
    from paper_2601_05936_gb300 import workloads
    c = workloads.adjoint_window(lattice, n=n, levels=levels, **kw)
    D = len(n)
    c["periodic"] = (False,) * D
    c["slip"] = (True,) * (D - 1) + (False,)
    return c


def test_rising_bubble_between_slip_walls():
    rng = np.random.default_rng(8)
    N = 40
    x = np.arange(N) + 0.5
    X, Y = np.meshgrid(x, x)
    xc, yc = N / 2 + rng.random(), 12.0 + rng.random()
    phi = 7.0 - np.sqrt((X - xc) ** 2 + (Y - yc) ** 2)
    case = dict(lattice="D2Q9", base=(N, N), n_levels=1, block=(32, 8), periodic=(False, False),
                slip=(True, False), rho_phys=(1.0, 0.01), nu=(0.06, 0.6), sigma=2e-3, gravity=(0.0, -2e-5),
                x_ref=(xc, yc), phi0=phi.reshape(-1), regrid_every=0)
    g, s, refilled = run_both_schedule(case, 60)
    r = compare_levels(g, s)[0]
    assert r["u"] < 1e-4, r
    ie = interface_errors(g, s, refilled)
    assert ie["iface_equal"] and ie["u_rel_max"] < 1e-3 and ie["drho_max"] < 1e-5, ie
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    assert np.abs(phi_g - s.phi).max() < 1e-4


@pytest.mark.parametrize("lattice,n,levels,kw", [
    ("D2Q9", (32, 24), 1, {}),
    ("D3Q19", (16, 16, 14), 1, {"block": (16, 4, 4)}),
    ("D2Q9", (48, 24), 2, {"block": (8, 8), "refine_dist": 2.0}),
])
def test_slip_window_parity(lattice, n, levels, kw):
    case = _slip_window(lattice, n, levels, **kw)
    g, s = run_both(case, 12)
    for r in compare_levels(g, s):
        assert r["leaf_equal"], r
        assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    g.close()


@pytest.mark.parametrize("lattice,n,levels,kw,warmup,steps", [
    ("D2Q9", (32, 24), 1, {}, 6, 12),
    ("D3Q19", (16, 16, 14), 1, {"block": (16, 4, 4)}, 4, 6),
    ("D2Q9", (48, 24), 2, {"block": (8, 8), "refine_dist": 2.0}, 4, 8),
])
def test_slip_window_adjoint(lattice, n, levels, kw, warmup, steps):
    from oracle.adjoint import FrozenStep, gradients, params_of
    from oracle import adjoint_amr
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    case = as_fp32_phi(_slip_window(lattice, n, levels, **kw))
    D = len(n)
    a = np.random.default_rng(1).standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0
    sim = Sim(case)
    sim.step(warmup)
    if levels == 1:
        st = FrozenStep(sim)
        assert st.rcut.any()
        _, dp_o, lam_o = gradients(st, sim.f[0].copy(), params_of(sim), steps, a)
        lam_o = [lam_o]
    else:
        st = adjoint_amr.AMRFrozenStep(sim)
        _, dp_o, lam_o = adjoint_amr.gradients(st, [f.copy() for f in sim.f], params_of(sim), steps, a)
    g = lsb.Grid(case)
    g.step(warmup)
    g.record(5)
    g.step(steps)
    dp_g = g.backward(a.reshape(1, -1))[0]
    for k in range(5):
        assert abs(dp_g[k] - dp_o[k]) <= 1e-3 * abs(dp_o[k]) + 1e-9, (k, dp_g, dp_o)
    for l in range(levels):
        lam_g = g.get("adj_f", 0, l).reshape(g.Q, -1).astype(np.float64)
        assert rel_l2(lam_g, lam_o[l]) < 1e-3, (l, rel_l2(lam_g, lam_o[l]))
    g.close()


@pytest.mark.parametrize("pcase", ["I", "II"])
def test_paper_box_parity(pcase):
    """The paper's box (slip lateral walls) at d = 8 cells, level set live; viscosity floored
    at 0.1 as for the downsampled benchmark bubble (tau 0.508 at the paper's Re is unstable)."""
    from paper_2601_05936_gb300 import workloads
    case = workloads.paper_box_3d(pcase, d=8, block=(16, 4, 4), nu_floor=0.1)
    g, s = run_both(case, 16)
    r = compare_levels(g, s)[0]
    assert r["leaf_equal"], r
    assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    ie = interface_errors(g, s)
    assert ie["iface_equal"] and ie["u_rel_max"] < 1e-3 and ie["drho_max"] < 1e-5, ie
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    assert np.abs(phi_g - s.phi).max() < 1e-4
    g.close()


def test_two_layer_couette_parity():
    from paper_2601_05936_gb300 import workloads
    case = workloads.two_layer_couette(nx=32, ny=32)
    g, s = run_both(case, 150)
    r = compare_levels(g, s)[0]
    assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    g.close()
