"""torch.autograd binding of the library's adjoint (lsb_record / lsb_backward).

``window(grid, params, nsteps)`` advances every case of ``grid`` by ``nsteps``
steps with the parameters in ``params`` (a float64 tensor, n_cases x 5:
sigma, rho_liquid, rho_gas, nu_liquid, nu_gas) and returns the observables
after the last step (n_cases x (4 + 2 D), lsb_observables order: masses,
gas volume, leaf cells, gas centroid, gas velocity).  Its backward runs the
library's reverse sweep with the incoming gradient as observable weights and
returns dJ/dparams.  The window starts from the grid's current state, which
the call advances (that state is not differentiated); the grid may hold a
frozen or a moving level set on one or several levels (lsb_backward's
conditions: FP32 storage, no cell changing phase inside the window).

``window_from(cases, params, phi0, nsteps)`` also differentiates the initial
interface: it creates a grid from ``cases`` with the initial level sets
``phi0`` (a tensor of n_cases x finest cells, or one per case), starts from
the rest state the library builds from them, and returns the observables;
backward gives dJ/dparams and dJ/dphi0.  With ``eps`` > 0 (default 1.5) the
volume, centroid and velocity are weighted by the smoothed gas indicator
(lsb_set_objective), so that a centroid objective has non-zero gradients;
a torch expression phi0(R) then gives dJ/dR (e.g. the initial radius).

All arithmetic runs in the CUDA library; this module only marshals tensors.
"""
import numpy as np
import torch

from . import lsb


class _Window(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, grid, cases, nsteps, checkpoint_every):
        p = params.detach().to("cpu", torch.float64).numpy()
        if p.shape != (len(cases), lsb.NPARAM_ADJ):
            raise ValueError("params must be n_cases x 5")
        for k, c in enumerate(cases):
            c = dict(c)
            c["sigma"] = float(p[k, 0])
            c["rho_phys"] = (float(p[k, 1]), float(p[k, 2]))
            c["nu"] = (float(p[k, 3]), float(p[k, 4]))
            grid.set_params(c, k)
        grid.record(checkpoint_every)
        grid.step(int(nsteps))
        obs = grid.observables()
        out = np.stack([np.concatenate([o["mass"], [o["volume"], o["leaf_cells"]], o["centroid"], o["velocity"]])
                        for o in obs])
        ctx.grid = grid
        ctx.device = params.device
        return torch.from_numpy(out).to(params.device)

    @staticmethod
    def backward(ctx, grad_out):
        w = grad_out.detach().to("cpu", torch.float64).numpy()
        dp = ctx.grid.backward(w)
        return torch.from_numpy(dp).to(ctx.device), None, None, None, None


def window(grid, params, nsteps, checkpoint_every=100):
    """Observables after ``nsteps`` steps, differentiable with respect to ``params``."""
    return _Window.apply(params, grid, grid.cases, nsteps, checkpoint_every)


def params_tensor(cases, requires_grad=True):
    """The n_cases x 5 parameter tensor of a list of case dicts."""
    rows = [[c.get("sigma", 0.0), c["rho_phys"][0], c["rho_phys"][1], c["nu"][0], c["nu"][1]] for c in cases]
    return torch.tensor(rows, dtype=torch.float64, requires_grad=requires_grad)


def _obs_matrix(grid):
    obs = grid.observables()
    return np.stack([np.concatenate([o["mass"], [o["volume"], o["leaf_cells"]], o["centroid"], o["velocity"]])
                     for o in obs])


def _apply_params(grid, cases, p):
    for k, c in enumerate(cases):
        c = dict(c)
        c["sigma"] = float(p[k, 0])
        c["rho_phys"] = (float(p[k, 1]), float(p[k, 2]))
        c["nu"] = (float(p[k, 3]), float(p[k, 4]))
        grid.set_params(c, k)


class _WindowFrom(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, phi0, cases, nsteps, checkpoint_every, eps, stream, device):
        p = params.detach().to("cpu", torch.float64).numpy()
        if p.shape != (len(cases), lsb.NPARAM_ADJ):
            raise ValueError("params must be n_cases x 5")
        phi = phi0.detach().to("cpu", torch.float64).numpy().reshape(len(cases), -1)
        cs = [dict(c, phi0=phi[k]) for k, c in enumerate(cases)]
        grid = lsb.Grid(cs, stream=stream, device=device)
        grid.set_objective(eps)
        _apply_params(grid, cs, p)
        grid.record(checkpoint_every)
        grid.step(int(nsteps))
        out = _obs_matrix(grid)
        ctx.grid = grid
        ctx.shape = phi0.shape
        ctx.devices = (params.device, phi0.device, phi0.dtype)
        return torch.from_numpy(out).to(params.device)

    @staticmethod
    def backward(ctx, grad_out):
        w = grad_out.detach().to("cpu", torch.float64).numpy()
        dp, dphi = ctx.grid.backward(w, want_phi=True)
        ctx.grid.close()
        pdev, fdev, fdt = ctx.devices
        g_phi = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dphi]).astype(np.float64))
        return (torch.from_numpy(dp).to(pdev), g_phi.reshape(ctx.shape).to(device=fdev, dtype=fdt),
                None, None, None, None, None, None)


def window_from(cases, params, phi0, nsteps, checkpoint_every=100, eps=1.5, stream=None, device=0):
    """Observables after ``nsteps`` steps of a grid created from ``cases`` with the initial
    level sets ``phi0``, differentiable with respect to ``params`` and ``phi0``."""
    if isinstance(cases, dict):
        cases = [cases]
    return _WindowFrom.apply(params, phi0, cases, nsteps, checkpoint_every, eps, stream, device)
