"""Where the reading of Eq. Sdecomp sets the method's stability limit (oracle, CPU).

The normal part of the stress jump, ([p] + sigma kappa_A) / (2 eta_bar), turns a
pressure mismatch across the interface into a jump of the strain rate, i.e. an
explicit relaxation of the mismatch whose gain grows as 1 / eta_bar.  Two
checks pin that this term is both necessary and the source of the
low-viscosity divergence the 3D rising bubble meets at the paper's Re = 35:

* a static drop started without its Laplace pressure reaches p_in - p_out =
  sigma / R with the term, and keeps no jump at all without it (so the term
  cannot be dropped: it is what enforces the Laplace law);
* at density ratio 1000 and liquid viscosity 0.02 the drop held at rest
  (interface frozen) diverges with the term within 500 steps, and stays at
  rest to round-off without it.
"""
import numpy as np
import pytest

from oracle import coupling
from oracle.lattice import CS2
from oracle.sim import Sim
from paper_2601_05936_gb300 import workloads

pytestmark = pytest.mark.slow


def _without_pressure_term(monkeypatch):
    orig = coupling.stress_jump_cc

    def no_pressure(c_i, nA, kA, Sbar, jp, jeta, eta_bar, sigma):
        return orig(c_i, nA, kA, Sbar, 0.0 * jp, jeta, eta_bar, 0.0)
    monkeypatch.setattr(coupling, "stress_jump_cc", no_pressure)


def _jump_ratio(case, s):
    rho, _ = s.macros()
    ph, phi = s.phase[-1], s.phi
    rp = np.asarray(case["rho_phys"])
    p = rp[ph] * CS2 * (rho - 1.0)
    dp = p[(ph == 1) & (phi > 3)].mean() - p[(ph == 0) & (phi < -3)].mean()
    return dp / (case["sigma"] / case["R"])


@pytest.mark.parametrize("with_term", [True, False])
def test_the_normal_stress_term_sets_the_laplace_jump(monkeypatch, with_term):
    case = workloads.static_drop(n=48, levels=1, radius_base=10.0, nu_l=0.1, rho_ratio=10.0)
    case.update(p_gas0=0.0)  # no Laplace pressure at the start
    case["phi0"] = np.asarray(case["phi0"], np.float32).astype(np.float64)
    if not with_term:
        _without_pressure_term(monkeypatch)
    s = Sim(case)
    s.step(1000)
    r = _jump_ratio(case, s)
    if with_term:
        assert abs(r - 1.0) < 0.1, r  # 0.925 after 1000 steps, 1.003 after 3000
    else:
        assert abs(r) < 1e-6, r


@pytest.mark.parametrize("with_term", [True, False])
def test_the_normal_stress_term_diverges_at_low_viscosity(monkeypatch, with_term):
    case = workloads.static_drop(n=48, levels=1, radius_base=10.0, nu_l=0.02)
    case.update(ls_active=False, n_ext=0, reinit_every=0)
    case["phi0"] = np.asarray(case["phi0"], np.float32).astype(np.float64)
    if not with_term:
        _without_pressure_term(monkeypatch)
    s = Sim(case)
    with np.errstate(all="ignore"):
        s.step(500)
        _, u = s.macros()
    umax = float(np.nanmax(np.abs(u))) if np.isfinite(u).any() else np.inf
    if with_term:
        assert not np.isfinite(u).all() or umax > 1.0, umax
    else:
        assert umax < 1e-12, umax
