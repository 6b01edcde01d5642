"""Seeded synthetic workloads shaped like the paper's test cases (Sec. 3).

Inputs only: case dictionaries (geometry, initial level set, lattice-unit
parameters).  None of the method's arithmetic lives here; both the CUDA
library (through lsb.Grid) and the FP64 oracle (oracle.sim.Sim) consume these
dictionaries unchanged.  Every random number comes from
numpy.random.default_rng(seed) with seed = 1000 * workload + case.

Lattice parameters from the dimensionless groups (Sec. 3.2, Table 1 and the
Re / Eo definitions): with bubble diameter d in finest cells, U = Ma c_s,
g = U^2 / d, nu_l = U d / Re, nu_g = nu_l (eta_g/eta_l)(rho_l/rho_g),
sigma = rho_l g d^2 / Eo (rho_l = 1).

Two limits of the method as implemented shape the choice of Ma and nu_l.
Both were measured on the oracle and the library alike: the explicit
normal-stress coupling of Eq. Sdecomp relaxes a pressure mismatch with a gain
of ~ q(1-q) rho c_s / (2 eta_bar), and static drops at density ratio 1000
diverge below nu_l ~ 0.05 (stable from ~0.1); and the gas, whose lattice
pressure is rho_g c_s^2 rho_hat, compresses by ~400 Ma^2 under the Laplace
pressure at density ratio 1000, so the 3D bubble at the paper's Re = 35
(nu_l = 0.021 at Ma 0.02, d = 64) diverges within 100 steps.  So nu_l is floored at ``nu_floor`` (the effective
Reynolds number U d / nu_l is stored with the case) and the gas starts at its
Laplace pressure (p_gas0 = sigma (D-1) / R).
"""
import numpy as np

CS = 1.0 / np.sqrt(3.0)
LS_DEFAULTS = dict(n_ext=8, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)


def _grid_centers(dims):
    """Cell-centre coordinates, arrays shaped dims[::-1] (x fastest)."""
    axes = [np.arange(n) + 0.5 for n in dims]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    return mesh[::-1]  # x, y[, z] each shaped (nz,) ny, nx


def bubble_params(d, Re, Eo, rho_ratio, eta_ratio, Ma=0.02, nu_floor=0.1):
    U = Ma * CS
    g = U * U / d
    nu_l = max(U * d / Re, nu_floor)
    nu_g = nu_l * (1.0 / eta_ratio) * rho_ratio
    sigma = g * d * d / Eo
    return dict(Ma=Ma, g=g, nu=(nu_l, nu_g), sigma=sigma, rho_phys=(1.0, 1.0 / rho_ratio), Re_eff=U * d / nu_l)


def stratified_channel(nx=64, ny=32, h=16.2, steps=1000, tau_heavy=0.8, rho_ratio=10.0, eta_ratio=5.0,
                       umax=0.01, block=(32, 8)):
    """Two-layer channel (Sec. 3.1): periodic x, walls at y = 0 and y = ny, interface y = h."""
    x, y = _grid_centers((nx, ny))
    nu_l = (tau_heavy - 0.5) / 3.0
    nu_g = nu_l * (1.0 / eta_ratio) * rho_ratio
    G = 8.0 * nu_l * umax / ny ** 2
    return dict(name=f"stratified_channel_{nx}x{ny}", lattice="D2Q9", base=(nx, ny), n_levels=1, block=block,
                periodic=(True, False), rho_phys=(1.0, 1.0 / rho_ratio), nu=(nu_l, nu_g), body_force=(G, 0.0),
                gravity=(0.0, 0.0), sigma=0.0, phi0=(y - h).reshape(-1), steps=steps, **LS_DEFAULTS)


def static_drop(seed=2000, n=128, levels=2, radius_base=20.0, band=4.0, rho_ratio=1000.0, eta_ratio=100.0,
                nu_l=0.1, steps=5000, block=(32, 8)):
    """Laplace test: circular gas bubble (phi > 0 inside) in a periodic box, seeded sub-cell offset and sigma."""
    rng = np.random.default_rng(seed)
    r = 2 ** (levels - 1)
    off = rng.random(2)
    sigma = float(rng.uniform(1e-3, 1e-2))
    N = n * r
    x, y = _grid_centers((N, N))
    xc = (n / 2 + off[0]) * r
    yc = (n / 2 + off[1]) * r
    R = radius_base * r
    phi = R - np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    nu_g = nu_l * (1.0 / eta_ratio) * rho_ratio
    return dict(name=f"static_drop_{n}x{n}_L{levels}", lattice="D2Q9", base=(n, n), n_levels=levels, block=block,
                periodic=(True, True), rho_phys=(1.0, 1.0 / rho_ratio), nu=(nu_l, nu_g), sigma=sigma,
                phi0=phi.reshape(-1), refine_dist=[band] * (levels - 1), sensor="band", regrid_every=0,
                R=R, p_gas0=sigma / R, steps=steps, **LS_DEFAULTS)


def rising_bubble_2d(seed=3000, nx=160, ny=320, levels=3, radius_base=40.0, rho_ratio=1000.0, eta_ratio=100.0,
                     Eo=10.0, Re=35.0, steps=3000, block=(32, 8), Ma=0.01):
    """2D rising bubble in a no-slip box, bubble at 1/4 height (Sec. 3.2 setup in 2D)."""
    rng = np.random.default_rng(seed)
    r = 2 ** (levels - 1)
    d = 2 * radius_base * r
    prm = bubble_params(d, Re, Eo, rho_ratio, eta_ratio, Ma=Ma)
    x, y = _grid_centers((nx * r, ny * r))
    off = rng.random(2) * 0.5
    xc, yc = (nx / 2 + off[0]) * r, (ny / 4 + off[1]) * r
    phi = radius_base * r - np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    dref = [3.0 * 16.0] + [16.0] * (levels - 2) if levels > 2 else [16.0] * (levels - 1)
    return dict(name=f"rising_bubble_2d_{nx}x{ny}_L{levels}", lattice="D2Q9", base=(nx, ny), n_levels=levels,
                block=block, periodic=(False, False), rho_phys=prm["rho_phys"], nu=prm["nu"],
                gravity=(0.0, -prm["g"]), sigma=prm["sigma"], x_ref=(xc, yc), phi0=phi.reshape(-1),
                p_gas0=prm["sigma"] / (d / 2), refine_dist=dref, sensor="band", regrid_every=25, steps=steps,
                Ma=prm["Ma"], Re_eff=prm["Re_eff"], **LS_DEFAULTS)


def rising_bubble_3d(seed=4000, nx=128, ny=128, nz=256, levels=2, radius_base=16.0, rho_ratio=1000.0,
                     eta_ratio=100.0, Eo=10.0, Re=35.0, steps=2000, block=(32, 4, 4), storage="fp32", scale=1.0,
                     Ma=0.005):
    """3D rising bubble (Sec. 3.2): no-slip box, gravity along -z, bubble at 1/4 height.

    scale < 1 gives the downsampled copy used for oracle parity (same physics,
    d scaled with the box)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = int(nx * scale), int(ny * scale), int(nz * scale)
    radius_base = radius_base * scale
    r = 2 ** (levels - 1)
    d = 2 * radius_base * r
    prm = bubble_params(d, Re, Eo, rho_ratio, eta_ratio, Ma=Ma)
    x, y, z = _grid_centers((nx * r, ny * r, nz * r))
    off = rng.random(3) * 0.5
    c = ((nx / 2 + off[0]) * r, (ny / 2 + off[1]) * r, (nz / 4 + off[2]) * r)
    phi = radius_base * r - np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    return dict(name=f"rising_bubble_3d_{nx}x{ny}x{nz}_L{levels}", lattice="D3Q19", base=(nx, ny, nz),
                n_levels=levels, block=block, periodic=(False, False, False), rho_phys=prm["rho_phys"],
                nu=prm["nu"], gravity=(0.0, 0.0, -prm["g"]), sigma=prm["sigma"], x_ref=c,
                phi0=phi.reshape(-1).astype(np.float32), refine_dist=[max(8.0, 16.0 * scale * 2)] * (levels - 1),
                sensor="band", regrid_every=25, steps=steps, storage=storage, fp16_scale=1024.0, Ma=prm["Ma"],
                Re_eff=prm["Re_eff"], p_gas0=2.0 * prm["sigma"] / (d / 2), **LS_DEFAULTS)


PAPER_CASES = {"I": dict(Re=35.0, Eo=10.0, rho_ratio=10.0, eta_ratio=10.0),
               "II": dict(Re=35.0, Eo=125.0, rho_ratio=1000.0, eta_ratio=100.0)}


def paper_box_3d(case="I", d=64, levels=1, seed=4100, block=(32, 4, 4), storage="fp32", steps=2000,
                 Ma=0.02, nu_floor=0.0, lattice="D3Q19", collision=("bgk", "bgk"), sensor="band", refine_dist=8.0,
                 regrid_every=25):
    """The 3D rising-bubble benchmark in the paper's own box (Sec. 3.2): width 2 d, depth 2 d,
    height 4 d (z up, gravity along -z), slip lateral walls, no-slip top and bottom, bubble
    diameter d (finest cells; the paper uses d = 64 on a uniform grid), parameter set I or II
    of the paper's table, Ma = 0.02.  The bubble starts centred laterally one diameter above
    the floor (a sub-cell random offset from ``seed``); the paper's text does not state the
    start height.  With levels > 1 the coarse grid is the box / 2^(levels-1) and the band of
    the interface is refined (``sensor`` "band": |phi| <= refine_dist; "signed": the gas plus
    the liquid within refine_dist of the interface, the paper's AMR study; refine_dist in
    finest cells).  The paper's own runs use D3Q27 with BGK in the liquid and
    the cumulant model in the gas: lattice="D3Q27", collision=("bgk", "cumulant")."""
    rng = np.random.default_rng(seed)
    prm = bubble_params(float(d), Ma=Ma, nu_floor=nu_floor, **PAPER_CASES[case])
    r = 2 ** (levels - 1)
    nf = (2 * d, 2 * d, 4 * d)
    base = tuple(n // r for n in nf)
    assert all(b * r == n for b, n in zip(base, nf)), "box not divisible by the level ratio"
    x, y, z = _grid_centers(nf)
    off = rng.random(3) * 0.5
    c = (d + off[0], d + off[1], d + off[2])
    phi = 0.5 * d - np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    tag = "" if lattice == "D3Q19" else f"_{lattice}_{'_'.join(collision)}"
    return dict(name=f"paper_box_3d_case{case}_d{d}_L{levels}{tag}", lattice=lattice, collision=tuple(collision),
                base=base, n_levels=levels,
                block=block, periodic=(False, False, False), slip=(True, True, False), rho_phys=prm["rho_phys"],
                nu=prm["nu"], gravity=(0.0, 0.0, -prm["g"]), sigma=prm["sigma"], x_ref=c,
                phi0=phi.reshape(-1).astype(np.float32), refine_dist=[float(refine_dist)] * (levels - 1),
                sensor=sensor, regrid_every=regrid_every if levels > 1 else 0, steps=steps, storage=storage,
                fp16_scale=1024.0,
                Ma=prm["Ma"], Re_eff=prm["Re_eff"], p_gas0=2.0 * prm["sigma"] / (d / 2), **LS_DEFAULTS)


def bubble_cluster_3d(case="I", d=16, levels=1, seed=4200, block=(32, 4, 4), storage="fp32", steps=2000,
                      Ma=0.02, nu_floor=0.05, spacing=1.5, sensor="band", refine_dist=8.0, regrid_every=25):
    """Cluster of nine rising bubbles (Sec. 3.2, last example): a box of 10 d x 10 d x 20 d
    (z up, gravity along -z), bubble diameter d (finest cells), parameter set I, two layers
    of five and four bubbles.  The paper gives neither the positions nor the walls; this
    reading: lower layer at height 2 d with one bubble on the vertical axis and four on the
    diagonals at (+-s, +-s), upper layer at height 2 d + s with four bubbles on the axes at
    (+-s, 0) and (0, +-s), s = spacing x d (1.5 d: neighbouring bubbles 2.1 d apart), the
    whole cluster shifted by a sub-cell offset from ``seed``; walls as in the single-bubble
    box (slip lateral walls, no-slip top and bottom).  Levels and sensor as paper_box_3d."""
    rng = np.random.default_rng(seed)
    prm = bubble_params(float(d), Ma=Ma, nu_floor=nu_floor, **PAPER_CASES[case])
    r = 2 ** (levels - 1)
    nf = (10 * d, 10 * d, 20 * d)
    base = tuple(n // r for n in nf)
    assert all(b * r == n for b, n in zip(base, nf)), "box not divisible by the level ratio"
    off = rng.random(3) * 0.5
    cx, cy, s = 5.0 * d + off[0], 5.0 * d + off[1], spacing * d
    z0 = 2.0 * d + off[2]
    centres = [(cx, cy, z0)] + [(cx + a * s, cy + b * s, z0) for a in (-1, 1) for b in (-1, 1)]
    centres += [(cx + a, cy + b, z0 + s) for a, b in ((-s, 0.0), (s, 0.0), (0.0, -s), (0.0, s))]
    x, y, z = _grid_centers(nf)
    phi = np.full(x.shape, -np.inf)
    for c in centres:  # gas inside any bubble: the largest signed distance
        phi = np.maximum(phi, 0.5 * d - np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2))
    xr = tuple(float(v) for v in np.mean(np.asarray(centres), axis=0))
    return dict(name=f"bubble_cluster_3d_case{case}_d{d}_L{levels}", lattice="D3Q19", base=base, n_levels=levels,
                block=block, periodic=(False, False, False), slip=(True, True, False), rho_phys=prm["rho_phys"],
                nu=prm["nu"], gravity=(0.0, 0.0, -prm["g"]), sigma=prm["sigma"], x_ref=xr,
                phi0=phi.reshape(-1).astype(np.float32), refine_dist=[float(refine_dist)] * (levels - 1),
                sensor=sensor, regrid_every=regrid_every if levels > 1 else 0, steps=steps, storage=storage,
                fp16_scale=1024.0, Ma=prm["Ma"], Re_eff=prm["Re_eff"], p_gas0=2.0 * prm["sigma"] / (d / 2),
                centres=centres, **LS_DEFAULTS)


def two_layer_couette(nx=2048, ny=2048, h_frac=0.5 + 1.0 / 512, U=0.01, rho=(1.0, 0.1), eta_ratio=5.0, nu_heavy=0.1,
                      block=(32, 8), steps=1000):
    """Two-layer Couette flow (Sec. 3.1): the domain [0, 2] x [-1, 1] of the paper on an
    nx x ny grid, periodic in x, a resting bottom wall and a top wall moving at U along x,
    a flat interface at height h (heavy fluid below) that stays put (u . n = 0), level set
    live.  Steady state: the piecewise-linear profile with the shear-stress jump set by the
    viscosity ratio."""
    h = h_frac * ny
    _, yy = _grid_centers((nx, ny))
    phi = yy - h
    etaA = rho[0] * nu_heavy
    nu = (nu_heavy, etaA / eta_ratio / rho[1])
    wall = np.zeros((4, 2))
    wall[3, 0] = U
    return dict(name=f"two_layer_couette_{nx}x{ny}", lattice="D2Q9", base=(nx, ny), n_levels=1, block=block,
                periodic=(True, False), rho_phys=rho, nu=nu, wall_u=wall.reshape(-1), phi0=phi.reshape(-1),
                steps=steps, regrid_every=0, **LS_DEFAULTS)


def ensemble(seed0=5000, n_cases=64, steps=2000, block=(32, 8), w_range=(96, 256), max_levels=3):
    """Uneven 2D rising bubbles: width ~ U{96..256} (even), height 2*width, levels U{1..3},
    density ratio log-uniform [10, 1000], Eo U[1, 40], Re U[10, 100], radius width/8."""
    out = []
    for k in range(n_cases):
        rng = np.random.default_rng(seed0 + k)
        w = int(rng.integers(w_range[0] // 2, w_range[1] // 2 + 1)) * 2
        L = int(rng.integers(1, max_levels + 1))
        rr = float(10 ** rng.uniform(1.0, 3.0))
        Eo = float(rng.uniform(1.0, 40.0))
        Re = float(rng.uniform(10.0, 100.0))
        r = 2 ** (L - 1)
        R = w / 8.0 * r
        prm = bubble_params(2 * R, Re, Eo, rr, 100.0, Ma=0.01)
        x, y = _grid_centers((w * r, 2 * w * r))
        off = rng.random(2) * 0.5
        xc, yc = (w / 2 + off[0]) * r, (w / 2 + off[1]) * r
        phi = R - np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
        dref = ([48.0] + [16.0] * (L - 2)) if L > 2 else [16.0] * (L - 1)
        out.append(dict(name=f"ensemble_{k}_{w}x{2 * w}_L{L}", lattice="D2Q9", base=(w, 2 * w), n_levels=L,
                        block=block, periodic=(False, False), rho_phys=prm["rho_phys"], nu=prm["nu"],
                        gravity=(0.0, -prm["g"]), sigma=prm["sigma"], x_ref=(xc, yc), phi0=phi.reshape(-1),
                        p_gas0=prm["sigma"] / R, refine_dist=dref, sensor="band", regrid_every=25, steps=steps,
                        Re_eff=prm["Re_eff"], **LS_DEFAULTS))
    return out


def uniform_box(n=128, lattice="D3Q19", storage="fp32", nu=0.05, force=1e-6):
    """Single-phase periodic box driven by a weak body force: the collide-and-stream
    kernel alone, sized for profiling captures (n = 128: 2 x 160 MB of populations)."""
    D = 3 if lattice == "D3Q19" else 2
    base = (n,) * D
    block = (32, 4, 4) if D == 3 else (32, 8)
    bf = (force,) + (0.0,) * (D - 1)
    return dict(name=f"uniform_box_{lattice}_{n}", lattice=lattice, base=base, n_levels=1, block=block,
                periodic=(True,) * D, rho_phys=(1.0, 1.0), nu=(nu, nu), body_force=bf, phi0=-np.ones(n ** D),
                ls_active=False, n_ext=0, reinit_every=0, storage=storage, fp16_scale=1024.0)


def adjoint_window(lattice="D2Q9", seed=6000, n=(32, 24), steps=20, warmup=10, levels=1, block=None,
                   refine_dist=4.0):
    """Frozen-interface window for the adjoint (level set held fixed, ls_active off):
    a gas bubble plus a one-cell gas film on the bottom wall (so that every
    bounce-back branch occurs: links whose back neighbour is the wall take the
    half-way fallback), a moving top wall, gravity, a body force along x,
    density ratio 10 and unequal viscosities.  ``warmup`` forward steps develop
    the flow before the recorded ``steps``.  With ``levels`` > 1, ``n`` is the
    coarse grid, the shapes are drawn on the finest grid (n * 2^(levels-1)) and
    blocks within ``refine_dist`` finest cells of the interface are refined,
    with no regrid (the block layout stays fixed over the window)."""
    rng = np.random.default_rng(seed)
    D = 2 if lattice == "D2Q9" else 3
    n = tuple(int(v) for v in n)
    assert len(n) == D
    nf = tuple(v * 2 ** (levels - 1) for v in n)
    cen = _grid_centers(nf)
    c = [(0.3 + 0.1 * rng.random()) * nf[0], (0.45 + 0.1 * rng.random()) * nf[1]] + \
        ([(0.45 + 0.1 * rng.random()) * nf[2]] if D == 3 else [])
    R = 0.18 * min(nf) + rng.random()
    bubble = R - np.sqrt(sum((cen[a] - c[a]) ** 2 for a in range(D)))
    h0 = 0.75 + 0.1 * rng.random()
    # phase-shifted modulations: no cell centre sits on an extremum, so no normal
    # component is exactly zero (the upwind choice of the extension has a kink there)
    film = h0 + 0.05 * np.sin(2 * np.pi * cen[0] / nf[0] + 0.37) - cen[D - 1]
    if D == 3:
        film = film + 0.03 * np.sin(2 * np.pi * cen[1] / nf[1] + 1.13)
    phi = np.maximum(bubble, film)
    wall_u = np.zeros((2 * D, D))
    wall_u[2 * D - 1, 0] = 0.02  # top wall moves along x
    grav = (0.0,) * (D - 1) + (-2e-5,)
    bf = (1e-5,) + (0.0,) * (D - 1)
    if block is None:
        block = (32, 8) if D == 2 else (32, 4, 4)
    tag = f"_L{levels}" if levels > 1 else ""
    return dict(name=f"adjoint_window_{lattice}_{'x'.join(map(str, n))}{tag}", lattice=lattice, base=n,
                n_levels=levels, block=tuple(block), periodic=(True,) * (D - 1) + (False,),
                rho_phys=(1.0, 0.1), nu=(0.08, 0.3), sigma=float(0.01 * (1 + rng.random())), gravity=grav,
                body_force=bf, wall_u=wall_u.reshape(-1), phi0=phi.reshape(-1), ls_active=False, n_ext=0,
                reinit_every=0, steps=steps, warmup=warmup, refine_dist=[float(refine_dist)] * (levels - 1),
                sensor="band", regrid_every=0)
