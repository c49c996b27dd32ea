"""One cavity over several ranks (eta-strips, 4-row halo): host-side logic on CPU.

Two or three gloo ranks each advance their strip of a developed 33^2 cavity
through paper_2306_07603_gb300.decomp (partition, halo exchange, residual
all-reduce), with the oracle's step as the local step. After 10 steps the
assembled field must equal the undivided oracle run bit for bit, and the
all-reduced Eq. (2.19) residuals must equal the undivided ones to rounding.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

N, RE, NPL, TH, DEV_STEPS, STEPS = 33, 400.0, 0.75, 60.0, 20, 10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _strip_grid(g, s):
    """The global grid's rows [p0, p1) as a grid of its own (metrics of the
    global eta rows; the real walls where the strip has them)."""
    import dataclasses

    rows = slice(s.p0, s.p1)
    zx = np.zeros(g.nx)
    wall_u = dict(bottom=g.wall_u["bottom"] if s.has_bottom_wall else (zx, zx),
                  top=g.wall_u["top"] if s.has_lid else (zx, zx),
                  left=tuple(a[rows] for a in g.wall_u["left"]),
                  right=tuple(a[rows] for a in g.wall_u["right"]))
    return dataclasses.replace(g, ny=s.rows, cxi=g.cxi[:, rows], ceta=g.ceta[:, rows],
                               J=g.J[rows], x_eta=g.x_eta[rows], y_eta=g.y_eta[rows],
                               wall_u=wall_u, x=g.x[rows], y=g.y[rows])


def _developed():
    import oracle as O
    run = O.cavity_run(N, RE, NPL, theta_deg=TH)
    run.advance(DEV_STEPS)
    return run


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle as O
    from paper_2306_07603_gb300 import decomp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    run = _developed()
    s = decomp.strip_partition(N, world)[rank]
    g = _strip_grid(run.g, s)

    def local_step(state):
        f, lam = O.step(state[:9].numpy(), state[9].numpy(), g, run.prm)
        return torch.from_numpy(np.concatenate([f, lam[None]]))

    st = torch.from_numpy(np.concatenate([run.fhat, run.lam[None]])[:, s.p0:s.p1].copy())
    stepper = decomp.StripStepper(s, local_step)
    for k in range(STEPS):
        prev = st[:, s.own].clone()
        st = stepper.step(st)
    # Eq. (2.19) partials of the last step over the owned nodes
    u1, v1, P1 = O.macros(st[:9, s.own].numpy())
    u0, v0, P0 = O.macros(prev[:9].numpy())
    du2 = (u1 - u0) ** 2 + (v1 - v0) ** 2
    u2 = u1 ** 2 + v1 ** 2
    sums = torch.tensor([du2.sum(), u2.sum(), ((P1 - P0) ** 2).sum(), (P1 ** 2).sum()],
                        dtype=torch.float64)
    maxima = torch.tensor([du2.max(), u2.max()], dtype=torch.float64)
    decomp.allreduce_residual(sums, maxima)
    q.put((rank, s.r0, s.r1, st[:, s.own].numpy(),
           decomp.residuals_from_partials(sums, maxima)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_strips_equal_the_undivided_cavity_bit_for_bit(world):
    import oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    run = _developed()
    run.advance(STEPS - 1)
    run.advance(1, record=True)
    ref = np.concatenate([run.fhat, run.lam[None]])
    asm = np.empty_like(ref)
    for rank, r0, r1, own, _ in got:
        asm[:, r0:r1] = own
    assert np.array_equal(asm, ref)                 # bit for bit
    Eu, EP, Rinf = run.history[-1]
    for _, _, _, _, (eu, ep, rinf) in got:          # every rank holds the combined residuals
        assert abs(eu - Eu) <= 1e-13 * Eu and abs(ep - EP) <= 1e-13 * EP
        assert rinf == Rinf


def test_strip_partition_rows_and_halos():
    from paper_2306_07603_gb300 import decomp
    for ny, world in ((33, 2), (33, 3), (257, 8), (1025, 7), (9, 2)):
        strips = decomp.strip_partition(ny, world)
        assert strips[0].r0 == 0 and strips[-1].r1 == ny
        for a, b in zip(strips, strips[1:]):
            assert a.r1 == b.r0
        sizes = [s.r1 - s.r0 for s in strips]
        assert max(sizes) - min(sizes) <= 1
        for s in strips:
            assert s.p0 == max(s.r0 - 4, 0) and s.p1 == min(s.r1 + 4, ny)
            assert s.has_bottom_wall == (s.rank == 0) and s.has_lid == (s.rank == world - 1)
    with pytest.raises(ValueError):
        decomp.strip_partition(12, 4)               # 3 rows a rank: less than the halo
    with pytest.raises(ValueError):
        decomp.StripStepper(decomp.strip_partition(33, 2)[0], None, halo=2)


def test_a_halo_of_two_rows_is_not_enough():
    """The dependence is four rows deep: with only two halo rows (and no
    exchange between the stencil stages) the owned rows next to the cut
    differ from the undivided step. Single process: the neighbour rows are
    copied in from the global state directly."""
    import oracle as O
    from paper_2306_07603_gb300 import decomp
    run = _developed()
    ref, _ = O.step(run.fhat, run.lam, run.g, run.prm)
    full = np.concatenate([run.fhat, run.lam[None]])
    for halo, equal in ((4, True), (2, False)):
        s = decomp.strip_partition(N, 2, halo=halo)[0]
        g = _strip_grid(run.g, s)
        f, _ = O.step(full[:9, s.p0:s.p1], full[9, s.p0:s.p1], g, run.prm)
        assert np.array_equal(f[:, s.own], ref[:, s.r0:s.r1]) == equal, halo


@pytest.mark.parametrize("theta", [45.0, 60.0, 90.0])
def test_strip_corners_are_the_cavity_grid_points(theta):
    """trapezoid_strip_corners: the corners of rows [p0, p1) are the cavity's
    grid points (oracle map of Eq. 3.8.1) at those rows' ends."""
    import oracle as O
    from paper_2306_07603_gb300 import decomp
    run = O.cavity_run(N, RE, NPL, theta_deg=theta, ny=29)
    g = run.g
    for p0, p1 in ((0, 29), (0, 12), (7, 19), (15, 29)):
        c = decomp.trapezoid_strip_corners(1.0, 1.0, theta, 29, p0, p1)
        want = ((g.x[p0, 0], g.y[p0, 0]), (g.x[p0, -1], g.y[p0, -1]),
                (g.x[p1 - 1, 0], g.y[p1 - 1, 0]), (g.x[p1 - 1, -1], g.y[p1 - 1, -1]))
        assert np.allclose(np.array(c), np.array(want), rtol=0, atol=1e-14), (p0, p1, c, want)
