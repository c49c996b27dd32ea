"""One cavity over several ranks with the strips' steps on the device.

Two and three gloo ranks share one GPU. Each advances the padded strip of its
rows of a 33 x 41 trapezoid cavity (theta = 60 deg), developed from rest by the
library, through decomp.StripStepper (4 halo rows exchanged per step). The
local step is decomp.LibraryStripStep: the strip as the quadrilateral of its
rows, on a library handle of its own (FP64, staged kernels, the undivided
cavity's dt). The ranks' kernels never wait on one another. Each rank's step
is its own launches, and the exchange runs over gloo on the host between
steps.

After 10 steps the owned rows must equal the undivided cavity's run (one
quadrilateral handle of the whole trapezoid, same dt):
- f-hat to 1e-12 of each plane's largest value;
- lambda to 1e-9 of its largest value.
The strips' per-node metrics come from their own corners and so agree with
the undivided ones to rounding, not bit for bit. lambda carries that rounding
amplified near the zero-shear clamp (Eqs. 2.12-2.14, 1.4).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu

NX, NY, RE, NPL, TH, DT, DEV, STEPS = 33, 41, 100.0, 0.75, 60.0, 0.0125, 300, 10


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_2306_07603_gb300 import decomp
    from paper_2306_07603_gb300.solver import Solver, quad_cavity
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        corners = decomp.trapezoid_strip_corners(1.0, 1.0, TH, NY, 0, NY)
        full = Solver([quad_cavity(NX, NY, corners, RE, NPL, H=1.0)], precision="fp64",
                      kernel="staged", dt=DT)
        full.step(DEV)
        f0, l0 = full.get_state(0)
        full.step(STEPS)
        fr, lr = full.get_state(0)
        full.close()
        s = decomp.strip_partition(NY, world)[rank]
        local = decomp.LibraryStripStep(s, NX, RE, NPL, TH, DT)
        st = torch.from_numpy(np.concatenate([f0, l0[None]])[:, s.p0:s.p1].copy())
        stepper = decomp.StripStepper(s, local)
        for _ in range(STEPS):
            st = stepper.step(st)
        local.close()
        got = st[:, s.own].numpy()
        ref = np.concatenate([fr, lr[None]])[:, s.r0:s.r1]
        err_f = max(float(np.abs(got[k] - ref[k]).max() / np.abs(fr[k]).max()) for k in range(9))
        err_l = float(np.abs(got[9] - ref[9]).max() / np.abs(lr).max())
        moved = float(np.abs(got[:9] - f0[:, s.r0:s.r1]).max())
        q.put((rank, err_f, err_l, moved, None))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, None, None, None, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_library_strips_reproduce_the_undivided_cavity(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for rank, err_f, err_l, moved, exc in sorted(res):
        assert exc is None, f"rank {rank}: {exc}"
        assert moved > 0.0                      # the strip did advance
        assert err_f <= 1e-12, (rank, err_f)
        assert err_l <= 1e-9, (rank, err_l)
