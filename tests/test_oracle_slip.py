"""Pins for slip walls (specular reflection; the paper's lateral walls, Sec. 3.2).

A slip wall is a mirror plane: a periodic box of twice the width whose state
is mirror-symmetric about the wall's plane evolves exactly like the walled
half (every population that crosses the plane is replaced by its mirror
image coming the other way, which is what the reflection writes).  So the
half box with slip walls must reproduce the symmetric full box to rounding,
step by step, from a random symmetric state: a wrong mirrored direction, a
missing tangential shift or a wrong corner treatment breaks it.  The 3D case
reflects on two axes (edges and corners included) next to no-slip walls with
a body force; the two-phase case adds interface links away from the walls.
Closed-box invariants: with slip walls and no force, mass and the momentum
tangential to the walls are conserved exactly.
"""
import numpy as np
import pytest

from oracle.lattice import get as get_lattice
from oracle.lbm import equilibrium, moments
from oracle.sim import Sim


def _mirror_state(lat, f_half, dims_half, axes):
    """Full periodic state from a half (quarter) box: mirror copies along ``axes``."""
    D = lat.D
    f = f_half.reshape((lat.Q,) + tuple(reversed(dims_half)))  # (Q, [z,] y, x)
    for a in axes:
        ax = D - a  # array axis of spatial axis a
        m = 1 << a
        flipped = np.flip(f, axis=ax)[lat.mirror[:, m]]
        f = np.concatenate([f, flipped], axis=ax)
    return f.reshape(lat.Q, -1)


def _lower(lat, f_full, dims_half, axes):
    D = lat.D
    full = [n * (2 if a in axes else 1) for a, n in enumerate(dims_half)]
    f = f_full.reshape((lat.Q,) + tuple(reversed(full)))
    sl = [slice(None)] + [slice(0, dims_half[D - 1 - j]) for j in range(D)]
    return f[tuple(sl)].reshape(lat.Q, -1)


def _case(lattice, dims, periodic, slip, phi, **kw):
    D = len(dims)
    c = dict(lattice=lattice, base=dims, n_levels=1, block=dims, periodic=periodic, slip=slip,
             rho_phys=(1.0, 0.1), nu=(0.08, 0.2), sigma=0.01, phi0=phi.reshape(-1), ls_active=False,
             n_ext=0, reinit_every=0)
    c.update(kw)
    return c


def _random_state(lat, N, rng, amp=1e-2):
    rho = 1.0 + amp * rng.standard_normal(N)
    u = amp * rng.standard_normal((lat.D, N))
    return equilibrium(lat, rho, u) + 0.1 * amp * rng.standard_normal((lat.Q, N)) * lat.w[:, None]


@pytest.mark.parametrize("lattice,dims,axes,periodic,bf", [
    ("D2Q9", (12, 10), (1,), (True, False), (2e-5, 0.0)),
    ("D3Q19", (8, 6, 10), (0, 1), (False, False, False), (0.0, 0.0, -3e-5)),
])
def test_slip_walls_are_mirror_planes(lattice, dims, axes, periodic, bf):
    lat = get_lattice(lattice)
    D = lat.D
    rng = np.random.default_rng(11)
    N = int(np.prod(dims))
    slip = tuple(a in axes for a in range(D))
    per_half = tuple(False if a in axes else periodic[a] for a in range(D))
    per_full = tuple(True if a in axes else periodic[a] for a in range(D))
    full_dims = tuple(n * 2 if a in axes else n for a, n in enumerate(dims))
    half = Sim(_case(lattice, dims, per_half, slip, -np.ones(N), body_force=bf))
    full = Sim(_case(lattice, full_dims, per_full, None, -np.ones(int(np.prod(full_dims))), body_force=bf))
    f0 = _random_state(lat, N, rng)
    half.f[0] = f0.copy()
    full.f[0] = _mirror_state(lat, f0, dims, axes)
    for _ in range(15):
        half.step(1)
        full.step(1)
    err = np.abs(half.f[0] - _lower(lat, full.f[0], dims, axes)).max()
    assert err < 1e-14, err


def test_slip_wall_mirror_plane_with_an_interface():
    """Two-phase, frozen level set: a bubble in the half box, its mirror image in the full box."""
    lat = get_lattice("D2Q9")
    dims = (24, 16)
    rng = np.random.default_rng(12)
    X, Y = np.meshgrid(np.arange(dims[0]) + 0.5, np.arange(2 * dims[1]) + 0.5)
    phi_full = np.maximum(4.3 - np.hypot(X - 11.2, Y - 7.4), 4.3 - np.hypot(X - 11.2, Y - (2 * dims[1] - 7.4)))
    phi_half = phi_full[:dims[1]]
    half = Sim(_case("D2Q9", dims, (True, False), (False, True), phi_half, body_force=(1e-5, 0.0)))
    full = Sim(_case("D2Q9", (dims[0], 2 * dims[1]), (True, True), None, phi_full, body_force=(1e-5, 0.0)))
    f0 = _random_state(lat, dims[0] * dims[1], rng, amp=2e-3)
    half.f[0] = f0.copy()
    full.f[0] = _mirror_state(lat, f0, dims, (1,))
    for _ in range(12):
        half.step(1)
        full.step(1)
    err = np.abs(half.f[0] - _lower(lat, full.f[0], dims, (1,))).max()
    assert err < 1e-13, err


@pytest.mark.parametrize("lattice,dims,slip", [("D2Q9", (10, 9), (False, True)),
                                               ("D3Q19", (6, 7, 5), (True, False, True))])
def test_closed_slip_box_conserves_mass_and_tangential_momentum(lattice, dims, slip):
    lat = get_lattice(lattice)
    N = int(np.prod(dims))
    periodic = tuple(not s for s in slip)
    sim = Sim(_case(lattice, dims, periodic, slip, -np.ones(N)))
    sim.f[0] = _random_state(lat, N, np.random.default_rng(3))
    rho, u = moments(lat, sim.f[0])
    m0, j0 = rho.sum(), (rho * u).sum(1)
    sim.step(30)
    rho, u = moments(lat, sim.f[0])
    assert abs(rho.sum() - m0) < 1e-12 * m0
    j = (rho * u).sum(1)
    for a in range(lat.D):
        if not slip[a]:  # periodic axis: tangential to every wall
            assert abs(j[a] - j0[a]) < 1e-13 * N, (a, j[a], j0[a])


def test_mirror_pin_detects_a_reflection_without_the_tangential_shift(monkeypatch):
    """Planted in the oracle: reflected populations arrive back at their own cell."""
    from oracle import grid
    orig = grid.LevelGeom.pull

    def bad(self, cells, ck):
        src, face, flip = orig(self, cells, ck)
        src = np.where(flip != 0, np.asarray(cells), src)
        return src, face, flip
    monkeypatch.setattr(grid.LevelGeom, "pull", bad)
    with pytest.raises(AssertionError):
        test_slip_walls_are_mirror_planes("D2Q9", (12, 10), (1,), (True, False), (2e-5, 0.0))


def _slip_window(lattice, n):
    """The adjoint window with slip side walls: its wall film meets them, so reflected
    links cross the interface there (plain bounce-back)."""
    from paper_2601_05936_gb300 import workloads
    c = workloads.adjoint_window(lattice, n=n)
    D = len(n)
    c["periodic"] = (False,) * D
    c["slip"] = (True,) * (D - 1) + (False,)
    return c


@pytest.mark.parametrize("lattice,n", [("D2Q9", (32, 24)), ("D3Q19", (10, 10, 14))])
def test_frozen_adjoint_with_slip_walls(lattice, n):
    from oracle.adjoint import FrozenStep, params_of
    sim = Sim(_slip_window(lattice, n))
    st = FrozenStep(sim)
    assert st.rcut.any()  # reflected links into the other phase occur
    f, p = sim.f[0].copy(), params_of(sim)
    for _ in range(3):
        f = st.step(f, p)
    sim.step(3)
    assert np.abs(f - sim.f[0]).max() < 1e-15
    lat = sim.lat
    rng = np.random.default_rng(4)
    f0 = _random_state(lat, st.g.N, rng)
    v = 1e-3 * rng.standard_normal(f0.shape)
    w = rng.standard_normal(f0.shape)
    eps = 1e-4
    Jv = (st.step(f0 + eps * v, p) - st.step(f0 - eps * v, p)) / (2 * eps)
    lam, _ = st.step_adjoint(f0, p, w)
    lhs, rhs = (Jv * w).sum(), (v * lam).sum()
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs), (lhs, rhs)
