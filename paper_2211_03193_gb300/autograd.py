"""Torch hand-off: V(G(s)) as a differentiable function and L-BFGS drivers.

``AMHEnergy`` wraps ``amh_grad`` (one CUDA launch computes V and dV/ds for a
batch of torsion vectors); its backward scales the stored gradient by the
incoming one.  The drivers pair AMH with L-BFGS as the abstract and Sec. 3
describe: ``lbfgs_refine`` minimises a batch of states (the paper's
pyrosetta ``lbfgs_armijo_nonmonotone`` is not available; torch's L-BFGS with
a strong-Wolfe line search stands in), and ``lbfgs_with_local_mh``
alternates L-BFGS runs with localized-MH sweeps (Sec. 3: "L-BFGS w/
localized MH", 80 L-BFGS samples then 20 local-MH samples).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _amh


class AMHEnergy(torch.autograd.Function):
    """E[b] = V(G(theta[b])) for theta of shape [batch, 2L] on the GPU."""

    @staticmethod
    def forward(ctx, theta, sampler, protein: int = 0):
        th = theta.detach().contiguous()
        E, g = sampler.grad(protein, th)
        ctx.save_for_backward(g)
        return E

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return (gE.to(g.dtype)[:, None] * g), None, None


def energy(sampler, theta, protein: int = 0):
    return AMHEnergy.apply(theta, sampler, protein)


def lbfgs_refine(sampler, theta0, iterations: int = 500, protein: int = 0, history: int = 20,
                 lr: float = 1.0):
    """L-BFGS on a batch of states (the batch's energies are summed; the
    states are independent, so each keeps its own gradient).  Returns the
    final torsions (wrapped to (-pi, pi]) and their energies."""
    theta = theta0.detach().clone().requires_grad_(True)
    opt = torch.optim.LBFGS([theta], lr=lr, max_iter=iterations, max_eval=int(iterations * 1.25),
                            history_size=history, line_search_fn="strong_wolfe",
                            tolerance_grad=1e-12, tolerance_change=1e-14)

    def closure():
        opt.zero_grad()
        E = energy(sampler, theta, protein).sum()
        E.backward()
        return E

    opt.step(closure)
    with torch.no_grad():
        th = torch.remainder(theta + np.pi, 2 * np.pi) - np.pi
        E, _ = sampler.grad(protein, th.contiguous())
    return th.detach(), E


def lbfgs_with_local_mh(sampler, cycles: int, n_lbfgs: int = 80, n_local: int = 20,
                        window: int = 5, T: float = 0.1, sigma_rad: float = 0.07,
                        seed: int = 1, on_cycle=None):
    """Alternate L-BFGS (n_lbfgs iterations) on every chain of a single-protein
    sampler with n_local localized-MH sweeps (window d), starting from the
    chains' current states.  on_cycle(cycle, handed, t0, after), if given,
    receives the torsions L-BFGS handed to the sampler, the proposal counter
    the local sweeps started at and the torsions they ended with (host
    float32 [chains, 2L]).  Returns the chains' final energies."""
    if len(sampler.proteins) != 1:
        raise ValueError("one protein per sampler")
    # amh_grad takes the context's precision
    dt = torch.float64 if sampler.precision == 64 else torch.float32
    for cyc in range(cycles):
        th = torch.tensor(sampler.torsions(0), device="cuda", dtype=dt)
        th, _ = lbfgs_refine(sampler, th, iterations=n_lbfgs)
        sampler.set_state(th.float().contiguous())
        if on_cycle is not None:
            handed, t0 = sampler.torsions(0), sampler.counter(0)
        if n_local:
            sampler.sweeps(_amh.AMH_LOCAL, window, T, sigma_rad, n_local, seed, accepted=False)
        if on_cycle is not None:
            on_cycle(cyc, handed, t0, sampler.torsions(0))
    return sampler.energy()
