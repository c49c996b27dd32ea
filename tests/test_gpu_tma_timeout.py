"""The fused kernel's bounded TMA waits, made to run out on purpose.

With the test hook ifdlbm_inject_tma_timeout the fused kernel issues no TMA row
loads, so that every wait for one has nothing to complete it. Each warp gives
up after its bounded wait (about a second), records the timeout in the status
word and waits no more; the next synchronising call reports
IFDLBM_ERR_TIMEOUT. No fault, no hang: the same process then runs a new
handle whose step still equals the oracle's.
"""
import time

import numpy as np
import pytest

import oracle as O
from test_gpu_parity import cav, oracle_run, rel, solver

pytestmark = pytest.mark.gpu


def test_tma_wait_that_runs_out_is_reported_and_the_context_survives():
    from paper_2306_07603_gb300 import capi
    s = solver([cav(33, 29, 100.0, 0.75, 60.0)], precision="fp32dev", kernel="fused",
               fused_threads=64, fused_rows=16, graph_chunk=0)
    s.step(2)
    s.sync()
    capi.ifdlbm_inject_tma_timeout(s.h, True)
    t0 = time.time()
    s.step(1)
    with pytest.raises(capi.IfdlbmError) as e:
        s.sync()
    assert e.value.code == capi.IFDLBM_ERR_TIMEOUT, str(e.value)
    assert time.time() - t0 < 60.0          # bounded: the warps gave up
    s.close()
    # a fresh handle in the same context steps as before
    run = oracle_run(33, 29, 100.0, 0.75, 60.0)
    run.advance(10)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    fo, _ = O.step(f0, l0, run.g, run.prm)
    s = solver([cav(33, 29, 100.0, 0.75, 60.0)], precision="fp32dev", kernel="fused",
               fused_threads=64, fused_rows=16)
    s.set_state(0, f0, l0)
    s.step(1)
    fg, _ = s.get_state(0)
    ug, vg, _ = O.macros(fg)
    uo, vo, _ = O.macros(fo)
    assert rel(ug, uo) < 1e-5 and rel(vg, vo) < 1e-5
    s.close()


def test_hook_refuses_the_staged_kernels():
    from paper_2306_07603_gb300 import capi
    s = solver([cav(17, 17, 100.0, 0.75, 60.0)], kernel="staged")
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_inject_tma_timeout(s.h, True)
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG
    s.close()
