"""torch.autograd binding of the library's adjoint (lsb_record / lsb_backward).

``window(grid, params, nsteps)`` advances every case of ``grid`` by ``nsteps``
steps with the parameters in ``params`` (a float64 tensor, n_cases x 5:
sigma, rho_liquid, rho_gas, nu_liquid, nu_gas) and returns the observables
after the last step (n_cases x (4 + 2 D), lsb_observables order: masses,
gas volume, leaf cells, gas centroid, gas velocity).  Its backward runs the
library's reverse sweep with the incoming gradient as observable weights and
returns dJ/dparams.  The level set must be frozen (ls_active off), the grid
single-level with FP32 storage; the window starts from the grid's current
state, which the call advances (state is not differentiated).

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
