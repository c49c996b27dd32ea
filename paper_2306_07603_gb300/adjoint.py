"""Gradients of scalar objectives after T steps with respect to (n, Re, theta).

Two objectives of one cavity advanced T steps from rest in FP64 (staged
kernels):

* ``KineticEnergy``: the kinetic energy of Eq. (5.1);
* ``PsiMin``: psi_min, the stream function at the primary eddy's node (the
  strength of the primary vortex), differentiable wherever that node does not
  change under the perturbation.

The forward pass keeps a device checkpoint of the state every ``every``
steps; the backward pass seeds the adjoint of the final state with the
library's seed for the objective, then runs the hand-written discrete adjoint
in reverse, segment by segment: it recomputes the segment's steps from its
checkpoint, keeping each step's output state and forward intermediates
(``ifdlbm_save_intermediates_dev``, 27 planes per step), and feeds them to
``ifdlbm_adjoint_step_saved``, so that no step is formed twice. A segment
holds ``every`` x (state + intermediates) bytes of device memory (~2 GB for
100 steps of a 257^2 cavity). With ``every = 1`` the forward pass itself keeps
every state and every step's intermediates (T x ~20 MB at 257^2) and the
backward pass recomputes nothing. All arithmetic happens in libifdlbm.so; this
module only orders the calls. Sensitivities are taken at a fixed time step: the runs use
the grid time-step rule, whose dt does not depend on theta.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .solver import Solver, cavity


def _state_buffer(h, stream):
    with torch.cuda.stream(stream):
        return torch.empty(capi.ifdlbm_state_bytes(h) // 8, dtype=torch.float64, device="cuda")


def _forward(params, nx, ny, T, every, U_lid, L, H, eta_b):
    n, Re, theta = (float(v) for v in params.detach().cpu().tolist())
    s = Solver([cavity(nx, ny, Re, n, theta_deg=theta, U_lid=U_lid, L=L, H=H)],
               precision="fp64", kernel="staged", eta_b=eta_b, dt_mode="grid")
    ckpt, inter = {}, None
    if every == 1:                      # keep every state and every step's intermediates
        inter = []
        nb = capi.ifdlbm_intermediate_bytes(s.h)
    for t0 in range(0, T, every):
        buf = _state_buffer(s.h, s.stream)
        capi.ifdlbm_save_state_dev(s.h, buf)
        ckpt[t0] = buf
        if inter is None:
            s.step(min(every, T - t0))
        else:
            capi.ifdlbm_step(s.h, 1)
            with torch.cuda.stream(s.stream):
                inter.append(torch.empty(nb // 8, dtype=torch.float64, device="cuda"))
            capi.ifdlbm_save_intermediates_dev(s.h, inter[-1])
    final = _state_buffer(s.h, s.stream)
    capi.ifdlbm_save_state_dev(s.h, final)
    return s, ckpt, final, inter
    return s, ckpt, final


def _backward(ctx, seed, gJ):
    """Adjoint sweep: `seed(h, final, adj, dparams)` writes dJ/d(final state)."""
    s, T, every = ctx.solver, ctx.T, ctx.every
    with torch.cuda.stream(s.stream):
        dparams = torch.zeros(3, dtype=torch.float64, device="cuda")
    adj = _state_buffer(s.h, s.stream)
    seed(s.h, ctx.final, adj, dparams)
    if ctx.inter is not None:                    # every == 1: nothing to recompute
        for t in range(T - 1, -1, -1):
            nxt = ctx.final if t == T - 1 else ctx.ckpt[t + 1]
            capi.ifdlbm_adjoint_step_saved(s.h, ctx.ckpt[t], nxt, ctx.inter[t], adj, dparams)
        s.sync()
        grad = dparams.cpu() * gJ
        s.close()
        return (grad,) + (None,) * 8
    nb = capi.ifdlbm_intermediate_bytes(s.h)
    states, inter = [], []                       # reused across segments
    for t0 in sorted(ctx.ckpt, reverse=True):
        t1 = min(t0 + every, T)
        capi.ifdlbm_load_state_dev(s.h, ctx.ckpt[t0])
        for t in range(t0, t1):                  # recompute the segment, keeping step t's
            capi.ifdlbm_step(s.h, 1)             # output state and intermediates
            k = t - t0
            if k == len(states):
                states.append(_state_buffer(s.h, s.stream))
                with torch.cuda.stream(s.stream):
                    inter.append(torch.empty(nb // 8, dtype=torch.float64, device="cuda"))
            capi.ifdlbm_save_state_dev(s.h, states[k])
            capi.ifdlbm_save_intermediates_dev(s.h, inter[k])
        for t in range(t1 - 1, t0 - 1, -1):
            k = t - t0
            prev = ctx.ckpt[t0] if k == 0 else states[k - 1]
            capi.ifdlbm_adjoint_step_saved(s.h, prev, states[k], inter[k], adj, dparams)
    s.sync()
    grad = dparams.cpu() * gJ
    s.close()
    return (grad,) + (None,) * 8


class KineticEnergy(torch.autograd.Function):
    """J(n, Re, theta) = kinetic energy after T steps; params = tensor([n, Re, theta_deg])."""

    @staticmethod
    def forward(ctx, params, nx, ny, T, every, U_lid=0.1, L=1.0, H=1.0, eta_b=0.5):
        s, ckpt, final, inter = _forward(params, nx, ny, T, every, U_lid, L, H, eta_b)
        J = float(s.residual()[0][3])
        ctx.solver, ctx.ckpt, ctx.final, ctx.T, ctx.every = s, ckpt, final, T, every
        ctx.inter = inter
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        return _backward(ctx, capi.ifdlbm_adjoint_seed_energy, gJ)


class PsiMin(torch.autograd.Function):
    """J(n, Re, theta) = min over interior nodes of psi after T steps."""

    @staticmethod
    def forward(ctx, params, nx, ny, T, every, U_lid=0.1, L=1.0, H=1.0, eta_b=0.5):
        s, ckpt, final, inter = _forward(params, nx, ny, T, every, U_lid, L, H, eta_b)
        e = s.eddies(0)[0]
        psi = np.zeros((ny, nx))
        capi.ifdlbm_batch_macros(s.h, 0, None, None, None, psi)
        ctx.node = (e.i, e.j)
        ctx.solver, ctx.ckpt, ctx.final, ctx.T, ctx.every = s, ckpt, final, T, every
        ctx.inter = inter
        return torch.tensor(float(psi[e.j, e.i]), dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        node = ctx.node
        return _backward(
            ctx, lambda h, st, adj, dp: capi.ifdlbm_adjoint_seed_psi(h, st, [node], adj, dp), gJ)


_OBJECTIVES = {"energy": KineticEnergy, "psi_min": PsiMin}


def objective_and_gradient(objective, n, Re, theta_deg, nx, ny, T, every=100, **kw):
    """(J, dJ/dn, dJ/dRe, dJ/dtheta_deg) through the adjoint; objective in
    {"energy", "psi_min"}."""
    p = torch.tensor([n, Re, theta_deg], dtype=torch.float64, requires_grad=True)
    J = _OBJECTIVES[objective].apply(p, nx, ny, T, every,
                                     *(kw.get(k, d) for k, d in (("U_lid", 0.1), ("L", 1.0),
                                                                 ("H", 1.0), ("eta_b", 0.5))))
    J.backward()
    return float(J), *(float(v) for v in p.grad)


def energy_and_gradient(n, Re, theta_deg, nx, ny, T, every=100, **kw):
    """(J, dJ/dn, dJ/dRe, dJ/dtheta_deg) of the kinetic energy through the adjoint."""
    return objective_and_gradient("energy", n, Re, theta_deg, nx, ny, T, every, **kw)
