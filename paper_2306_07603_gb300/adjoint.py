"""Gradients of the kinetic energy after T steps with respect to (n, Re, theta).

``KineticEnergy.apply(params, spec, T, every)`` advances one cavity T steps
from rest in FP64 (staged kernels) and returns the kinetic energy of
Eq. (5.1); its backward pass runs the library's hand-written discrete
adjoint (``ifdlbm_adjoint_step``) in reverse, recomputing the states of each
segment of ``every`` steps from a checkpoint kept on the device. All
arithmetic happens in libifdlbm.so; this module only orders the calls.
"""
from __future__ import annotations

import torch

from . import capi
from .solver import Solver, cavity


def _state_buffer(h, stream):
    with torch.cuda.stream(stream):
        return torch.empty(capi.ifdlbm_state_bytes(h) // 8, dtype=torch.float64, device="cuda")


class KineticEnergy(torch.autograd.Function):
    """J(n, Re, theta) = kinetic energy after T steps; params = tensor([n, Re, theta_deg])."""

    @staticmethod
    def forward(ctx, params, nx, ny, T, every, U_lid=0.1, L=1.0, H=1.0, eta_b=0.5):
        n, Re, theta = (float(v) for v in params.detach().cpu().tolist())
        s = Solver([cavity(nx, ny, Re, n, theta_deg=theta, U_lid=U_lid, L=L, H=H)],
                   precision="fp64", kernel="staged", eta_b=eta_b)
        ckpt = {}
        for t0 in range(0, T, every):
            buf = _state_buffer(s.h, s.stream)
            capi.ifdlbm_save_state_dev(s.h, buf)
            ckpt[t0] = buf
            s.step(min(every, T - t0))
        final = _state_buffer(s.h, s.stream)
        capi.ifdlbm_save_state_dev(s.h, final)
        J = float(s.residual()[0][3])
        ctx.solver, ctx.ckpt, ctx.final, ctx.T, ctx.every = s, ckpt, final, T, every
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        s, T, every = ctx.solver, ctx.T, ctx.every
        with torch.cuda.stream(s.stream):
            dparams = torch.zeros(3, dtype=torch.float64, device="cuda")
        adj = _state_buffer(s.h, s.stream)
        capi.ifdlbm_adjoint_seed_energy(s.h, ctx.final, adj, dparams)
        for t0 in sorted(ctx.ckpt, reverse=True):
            t1 = min(t0 + every, T)
            states = [ctx.ckpt[t0]]
            capi.ifdlbm_load_state_dev(s.h, ctx.ckpt[t0])
            for _ in range(t0 + 1, t1):             # recompute the segment
                capi.ifdlbm_step(s.h, 1)
                buf = _state_buffer(s.h, s.stream)
                capi.ifdlbm_save_state_dev(s.h, buf)
                states.append(buf)
            for t in range(t1 - 1, t0 - 1, -1):
                capi.ifdlbm_adjoint_step(s.h, states[t - t0], adj, dparams)
        s.sync()
        grad = dparams.cpu() * gJ
        s.close()
        return (grad,) + (None,) * 8


def energy_and_gradient(n, Re, theta_deg, nx, ny, T, every=100, **kw):
    """(J, dJ/dn, dJ/dRe, dJ/dtheta_deg) through the adjoint."""
    p = torch.tensor([n, Re, theta_deg], dtype=torch.float64, requires_grad=True)
    J = KineticEnergy.apply(p, nx, ny, T, every, *(kw.get(k, d) for k, d in
                                                   (("U_lid", 0.1), ("L", 1.0), ("H", 1.0),
                                                    ("eta_b", 0.5))))
    J.backward()
    return float(J), *(float(v) for v in p.grad)
