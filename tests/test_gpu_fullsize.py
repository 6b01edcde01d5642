"""The benchmark workload at its full size (128x128x256 base, two levels, D3Q19, FP32), in the
launch configuration bench.py times (library stream, TMA-staged collide-and-stream), against
the oracle on sampled outputs.

The oracle cannot step 37 M cells, but it can recompute sampled cells one by one: after the
full-size run's warm-up the state is exported, two more coarse steps run on the GPU, and for
sampled bulk cells (a cube of leaves of one phase around them, away from walls, the ghost
ring, the restriction layer and the interface) the oracle's collision and streaming redo the
same steps in float64 from the exported state on that cube alone: two steps on the coarse
level (radius 2), four on the fine one (radius 4, two fine sub-steps per coarse step).  The
cube shrinks by one cell per step, so its centre is exact.  FP32 state against float64:
populations agree to ~1e-7; the bound is 2e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _patch_steps(lat, cube, om, acc, nsteps):
    """cube: (Q, n, n, n) populations (z, y, x); nsteps BGK steps, pull streaming inside."""
    from oracle.lbm import collide
    f = cube
    for _ in range(nsteps):
        Q, n = f.shape[0], f.shape[1]
        fc = collide(lat, f.reshape(Q, -1), np.full(n ** 3, om), np.repeat(acc[:, None], n ** 3, 1)).reshape(f.shape)
        g = np.empty((Q, n - 2, n - 2, n - 2))
        for k in range(Q):
            cx, cy, cz = lat.c[k]
            g[k] = fc[k, 1 - cz:n - 1 - cz, 1 - cy:n - 1 - cy, 1 - cx:n - 1 - cx]
        f = g
    return f[:, 0, 0, 0]


def _bulk_centres(tag, dims, R, rng, m, extra=None):
    """Up to m cells whose (2R+1)^3 cube lies inside the box and is all leaves of one phase."""
    nx, ny, nz = dims
    leaf = (tag & 64) != 0
    gas = (tag & 1) != 0
    t = leaf.reshape(nz, ny, nx)
    g3 = gas.reshape(nz, ny, nx)
    out = []
    tries = 0
    while len(out) < m and tries < 200 * m:
        tries += 1
        x, y, z = (int(rng.integers(R, n - R)) for n in (nx, ny, nz))
        sl = (slice(z - R, z + R + 1), slice(y - R, y + R + 1), slice(x - R, x + R + 1))
        if not t[sl].all():
            continue
        if g3[sl].any() and not g3[sl].all():
            continue
        if extra is not None and not extra(x, y, z):
            continue
        out.append((x, y, z))
    return out


def test_bench_workload_full_size_sampled_cells():
    import torch
    from oracle.lattice import get as get_lattice
    from oracle.lbm import omega_from_nu
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.rising_bubble_3d()
    lat = get_lattice("D3Q19")
    stream = torch.cuda.Stream()
    g = lsb.Grid(case, stream=stream)
    g.step(3)
    g.sync()
    L = int(case["n_levels"])
    before = [g.get("f", 0, l).reshape(19, -1) for l in range(L)]  # float32; cubes go to float64
    tags = [g.get("tag", 0, l).reshape(-1) for l in range(L)]
    phi = g.get("phi").reshape(-1)
    g.step(2)
    after = [g.get("f", 0, l).reshape(19, -1) for l in range(L)]
    g.close()
    rng = np.random.default_rng(17)
    nu = np.asarray(case["nu"])
    grav = np.asarray(case["gravity"])
    checked = 0
    for l in range(L):
        r = 2 ** (L - 1 - l)
        dims = tuple(b * 2 ** l for b in case["base"])
        nx, ny, nz = dims
        nsteps = 2 * 2 ** l  # fine sub-steps per coarse step: 2^l
        R = nsteps
        far = None
        if l == L - 1:  # finest level: keep clear of the interface (no cut link, no refill)
            ph3 = phi.reshape(nz, ny, nx)
            far = lambda x, y, z: abs(float(ph3[z, y, x])) > R + 6
        cells = _bulk_centres(tags[l], dims, R, rng, 40, far)
        assert len(cells) >= 20, (l, len(cells))
        F = before[l].reshape(19, nz, ny, nx)
        A = after[l].reshape(19, nz, ny, nx)
        for x, y, z in cells:
            ph = int(tags[l].reshape(nz, ny, nx)[z, y, x] & 1)
            om = float(omega_from_nu(nu[ph] / r))
            acc = grav * r  # no body force in this workload
            cube = F[:, z - R:z + R + 1, y - R:y + R + 1, x - R:x + R + 1].astype(np.float64)
            exp = _patch_steps(lat, cube, om, acc, nsteps)
            err = np.abs(A[:, z, y, x].astype(np.float64) - exp).max()
            assert err < 2e-6, (l, (x, y, z), err)
            checked += 1
    assert checked >= 40
