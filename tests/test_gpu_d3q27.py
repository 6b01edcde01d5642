"""D3Q27 and the cumulant collision on the GPU against the oracle.

The oracle's cumulant operator (oracle/cumulant.py) keeps general rates and
per-cell linear solves; the library computes the rates-one case from the
relaxed second moments alone.  Parity here pins that shortcut: a periodic box
of gas with a random-ish velocity field (every population and moment active),
and the paper's own 3D setup at small size (D3Q27, BGK liquid, cumulant gas,
slip lateral walls, level set live), plus the same box with BGK in both
phases.  Tolerances as for the D3Q19 parity tests.
"""
import numpy as np
import pytest

from gpu_util import compare_levels, run_both

pytestmark = pytest.mark.gpu


def test_cumulant_gas_box_parity():
    """All-gas periodic box with a body force and a shear layer from the initial level set
    (liquid stripe): both operators side by side, every direction of D3Q27 active."""
    n = 16
    z = np.arange(n) + 0.5
    phi = np.repeat(np.abs(z - 8.3) - 3.1, n * n)  # liquid stripe |z - 8.3| < 3.1, gas elsewhere
    case = dict(lattice="D3Q27", base=(n, n, n), n_levels=1, block=(16, 4, 4), periodic=(True, True, True),
                rho_phys=(1.0, 0.5), nu=(0.05, 0.08), sigma=0.0, body_force=(2e-5, 1e-5, 0.0), phi0=phi,
                ls_active=False, n_ext=0, reinit_every=0, collision=("bgk", "cumulant"))
    g, s = run_both(case, 40)
    r = compare_levels(g, s)[0]
    assert r["u"] < 1e-4 and r["drho_abs"] < 1e-5, r
    fg = g.get("f").reshape(27, -1).astype(np.float64)
    assert np.abs(fg - s.f[0]).max() < 1e-5
    g.close()


@pytest.mark.parametrize("collision", [("bgk", "bgk"), ("bgk", "cumulant")])
def test_paper_setup_parity(collision):
    from paper_2601_05936_gb300 import workloads
    case = workloads.paper_box_3d("II", d=8, block=(16, 4, 4), nu_floor=0.1, lattice="D3Q27", collision=collision)
    g, s = run_both(case, 16)
    r = compare_levels(g, s)[0]
    assert r["leaf_equal"], r
    assert r["u"] < 1e-3 and r["drho_abs"] < 1e-5, r
    phi_g = g.get("phi").reshape(-1).astype(np.float64)
    assert np.abs(phi_g - s.phi).max() < 1e-4
    g.close()


def test_d3q27_limits():
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.paper_box_3d("I", d=8, block=(16, 4, 4), nu_floor=0.1, lattice="D3Q27",
                                  collision=("bgk", "cumulant"))
    with pytest.raises(lsb.LsbError):  # FP16 storage is not built for D3Q27
        lsb.Grid(dict(case, storage="fp16s"))
    with pytest.raises(lsb.LsbError):  # the cumulant operator needs D3Q27
        lsb.Grid(dict(case, lattice="D3Q19"))
    g = lsb.Grid(case)
    with pytest.raises(lsb.LsbError) as e:  # the adjoint transposes BGK on D2Q9 / D3Q19
        g.record(4)
    assert e.value.status == 6
    g.close()
