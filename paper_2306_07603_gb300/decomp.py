"""Decomposition of one cavity over several ranks: eta-strips with halo exchange.

One time step (Sec. 4, Steps 2-7) chains two stencils of radius 2 along eta
(Eqs. 3.6-3.7 with the five-point mixed differences of Eqs. 2.5-2.7): the
full step at row j reads f(t+dt/2) on rows j-2..j+2, and f(t+dt/2) on row k
reads f-bar^+ on rows k-2..k+2, which is pointwise in the state of row k. So
row j of f-hat(t+dt) depends on the state (f-hat and the previous lambda) of
rows j-4..j+4 only. A rank that owns rows [r0, r1) of the cavity therefore
advances a padded strip of rows [r0 - 4, r1 + 4) (clipped at the real walls)
with the ordinary single-cavity step and keeps rows [r0, r1): every value it
keeps is formed by the same operations on the same inputs as in the
undivided cavity. The rows the padded step treats as its edges (the
first-order near-wall differences at its rows 1 and -2, the wall rule on its
rows 0 and -1) are halo rows whose results are discarded; the real walls
(the bottom on the first rank, the lid on the last) are where the undivided
cavity has them.

Per step each rank sends its first and last `halo` owned rows of the ten
planes (nine populations and lambda) to its neighbours and receives theirs:
one exchange of 2 x halo x nx x 10 values per neighbour, through
torch.distributed point-to-point calls (gloo for host tensors, NCCL for
device tensors; no one-sided access to a peer's memory). The residuals of
Eq. (2.19) are sums and maxima over the owned nodes, combined by one
all-reduce of the sums and one of the maxima.

The halo depth is a parameter: a step of the same scheme needs 4; a caller
that exchanges after each of the two stencil stages could use 2 twice.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist

STEP_HALO = 4  # rows of dependence of one step: two chained radius-2 stencils


@dataclass(frozen=True)
class Strip:
    """Rows of one rank: owned [r0, r1) of the cavity's ny rows, held as the
    padded range [p0, p1) = [max(r0 - halo, 0), min(r1 + halo, ny))."""
    rank: int
    world: int
    ny: int
    r0: int
    r1: int
    p0: int
    p1: int

    @property
    def rows(self) -> int:
        return self.p1 - self.p0

    @property
    def own(self) -> slice:
        """The owned rows as a slice of the padded strip."""
        return slice(self.r0 - self.p0, self.r1 - self.p0)

    @property
    def has_bottom_wall(self) -> bool:
        return self.r0 == 0

    @property
    def has_lid(self) -> bool:
        return self.r1 == self.ny


def strip_partition(ny: int, world: int, halo: int = STEP_HALO) -> list[Strip]:
    """Balanced eta-strips: rank k owns ny // world rows, the first ny % world
    ranks one more. Each owned range must hold at least `halo` rows, so that a
    rank's halo comes from its two neighbours only."""
    if world < 1 or halo < 0:
        raise ValueError("world >= 1 and halo >= 0 required")
    base, extra = divmod(ny, world)
    if base < max(halo, 1):
        raise ValueError(f"{ny} rows over {world} ranks leave fewer than {max(halo, 1)} rows a rank")
    out, r = [], 0
    for k in range(world):
        n = base + (1 if k < extra else 0)
        out.append(Strip(k, world, ny, r, r + n, max(r - halo, 0), min(r + n + halo, ny)))
        r += n
    return out


class HaloExchange:
    """Per-step halo exchange of a rank's padded strip (planes along dim 0,
    rows along dim -2). Works on any tensors torch.distributed can send (host
    tensors over gloo, device tensors over NCCL)."""

    def __init__(self, strip: Strip, halo: int = STEP_HALO, group=None):
        self.s = strip
        self.halo = halo
        self.group = group

    def exchange(self, planes: torch.Tensor) -> None:
        """Overwrites the halo rows of `planes` (shape (..., rows, nx), rows =
        strip.rows) with the neighbours' owned rows, in place."""
        s, h = self.s, self.halo
        if h == 0 or s.world == 1:
            return
        own = s.own
        ops = []
        recv = []
        if s.rank > 0:      # neighbour below: its top owned rows are my bottom halo
            lo = s.r0 - s.p0                      # = h unless clipped (it is not: rank > 0)
            buf = torch.empty_like(planes[..., 0:lo, :]).contiguous()
            ops.append(dist.P2POp(dist.isend, planes[..., own.start:own.start + h, :].contiguous(),
                                  s.rank - 1, self.group))
            ops.append(dist.P2POp(dist.irecv, buf, s.rank - 1, self.group))
            recv.append((slice(0, lo), buf))
        if s.rank < s.world - 1:  # neighbour above: its bottom owned rows are my top halo
            hi = s.p1 - s.r1
            buf = torch.empty_like(planes[..., 0:hi, :]).contiguous()
            ops.append(dist.P2POp(dist.isend, planes[..., own.stop - h:own.stop, :].contiguous(),
                                  s.rank + 1, self.group))
            ops.append(dist.P2POp(dist.irecv, buf, s.rank + 1, self.group))
            recv.append((slice(own.stop, own.stop + hi), buf))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for sl, buf in recv:
            planes[..., sl, :] = buf


def allreduce_residual(sums: torch.Tensor, maxima: torch.Tensor, group=None):
    """Combines per-rank partials of Eq. (2.19) over the owned nodes: `sums`
    (sum |du|^2, sum |u|^2, sum dP^2, sum P^2, ...) by addition and `maxima`
    (max |du|^2, max |u|^2, ...) by maximum, in place on every rank."""
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(maxima, op=dist.ReduceOp.MAX, group=group)
    return sums, maxima


def residuals_from_partials(sums, maxima):
    """E(u), E(P) of Eq. (2.19) and the max-norm velocity residual from the
    combined partials (sum du2, sum u2, sum dP2, sum P2) and (max du2, max u2)."""
    du2, u2, dP2, P2 = (float(v) for v in sums[:4])
    mdu2, mu2 = (float(v) for v in maxima[:2])
    return (du2 / u2) ** 0.5, (dP2 / P2) ** 0.5, (mdu2 / mu2) ** 0.5


class StripStepper:
    """Advances one rank's strip: exchange the halo, run the single-cavity
    step on the padded strip, keep the owned rows.

    `local_step(state) -> state` advances a padded strip by one step; the
    state is a tensor of shape (10, rows, nx): the nine populations f-hat
    and the previous relaxation time. Which implementation runs the step is
    the caller's choice (the CUDA library on a device strip; any other
    implementation of the same step on the host)."""

    def __init__(self, strip: Strip, local_step, halo: int = STEP_HALO, group=None):
        if halo < STEP_HALO:
            raise ValueError(f"one step needs a halo of {STEP_HALO} rows")
        self.s = strip
        self.xchg = HaloExchange(strip, halo, group)
        self.local_step = local_step

    def step(self, state: torch.Tensor) -> torch.Tensor:
        self.xchg.exchange(state)
        new = self.local_step(state)
        out = state.clone()
        out[:, self.s.own, :] = new[:, self.s.own, :]
        return out


def trapezoid_strip_corners(L: float, H: float, theta_deg: float, ny: int, p0: int, p1: int):
    """Corners (bottom-left, bottom-right, top-left, top-right) of the rows
    [p0, p1) of an ny-row trapezoid cavity. The map of Eq. (3.8.1), with the
    lid's left end at x = 0, x = H cot(theta) + L xi + H cot(theta) (2 xi - 1)
    eta, y = H eta, is bilinear in (xi, eta), so the strip is the
    quadrilateral of these corners, and its own uniform grid of p1 - p0 rows
    falls on the cavity's rows p0..p1-1."""
    import math
    cot = 0.0 if theta_deg == 90.0 else 1.0 / math.tan(math.radians(theta_deg))

    def xy(xi, eta):
        return (H * cot + L * xi + H * cot * (2.0 * xi - 1.0) * eta, H * eta)

    e0, e1 = p0 / (ny - 1), (p1 - 1) / (ny - 1)
    return (xy(0.0, e0), xy(1.0, e0), xy(0.0, e1), xy(1.0, e1))


class LibraryStripStep:
    """`local_step` of StripStepper on the CUDA library: the padded strip of
    rows [p0, p1) of a trapezoid cavity, held by a handle of its own as the
    quadrilateral cavity of its rows (trapezoid_strip_corners), FP64 on the
    staged kernels, at the undivided cavity's time step `dt` and reference
    length H. The handle applies its wall rule and near-wall differences at
    all four edges of the strip; at a strip edge inside the cavity those land
    on halo rows, which StripStepper discards. The state crosses the host
    (set_state / get_state: the nine f-hat planes and lambda), so that the
    exchange can run over any torch.distributed backend."""

    def __init__(self, strip: Strip, nx: int, Re: float, n: float, theta_deg: float, dt: float,
                 U_lid: float = 0.1, L: float = 1.0, H: float = 1.0, **options):
        from .solver import Solver, quad_cavity
        corners = trapezoid_strip_corners(L, H, theta_deg, strip.ny, strip.p0, strip.p1)
        self.solver = Solver([quad_cavity(nx, strip.rows, corners, Re, n, U_lid=U_lid, H=H)],
                             precision="fp64", kernel="staged", dt=dt, **options)

    def __call__(self, state: torch.Tensor) -> torch.Tensor:
        import numpy as np
        s = state.detach().to("cpu", torch.float64).numpy()
        self.solver.set_state(0, np.ascontiguousarray(s[:9]), np.ascontiguousarray(s[9]))
        self.solver.step(1)
        f, lam = self.solver.get_state(0)
        return torch.from_numpy(np.concatenate([f, lam[None]])).to(state.device)

    def close(self):
        self.solver.close()
