"""The allocation-free residual entry point (ifdlbm_residual_fields_static).

It serves callers that must not allocate device memory. Here it is called
through the C ABI on device fields taken from a cavity before and after a
step, twice in a row, and must agree with the handle's own residual
(ifdlbm_residual) within the residual tolerance of the parity tests; around
the second call neither PyTorch's allocator nor the device's free memory may
change. A call on a field of exactly the array's capacity uses every slot of
the static scratch and is checked against a float64 reduction of Eq. (2.19).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-9  # the parity tests' tolerance for Eq. (2.19) residuals of one step


def test_static_residual_matches_handle_residual_on_two_calls():
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import Solver, cavity

    nx, ny = 67, 45
    s = Solver([cavity(nx, ny, 100.0, 0.75, theta_deg=60.0)])
    s.step(30)
    stream = s.stream

    def fields():
        rho, u, v = (torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3))
        capi.ifdlbm_macros_dev(s.h, 0, rho, u, v, None)
        with torch.cuda.stream(stream):
            P = (rho - 1.0) / 3.0          # P = (rho - rho0) c_s^2, rho0 = 1, c = 1
        return u, v, P

    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        u0, v0, p0 = fields()
        s.step(1)
        ref = s.residual()[0][:3]          # the existing entry point (synchronises)
        u1, v1, p1 = fields()
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
                  torch.cuda.mem_get_info()[0])
        capi.ifdlbm_residual_fields_static(nx, ny, u1, v1, p1, u0, v0, p0, out,
                                           stream.cuda_stream)
        stream.synchronize()
        after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
                 torch.cuda.mem_get_info()[0])
        if call == 1:                      # the first call was the set-up on this device
            assert after[:2] == before[:2], (before, after)
            assert after[2] >= before[2], (before, after)   # no device memory taken
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), (call, got)
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0, err_msg=f"call {call}")
    s.close()


def test_static_residual_on_a_field_of_the_full_capacity():
    """nx * ny = IFDLBM_STATIC_MAX_NODES: every partial slot of the array."""
    import torch

    from paper_2306_07603_gb300 import capi

    nx, ny = 2048, capi.IFDLBM_STATIC_MAX_NODES // 2048
    assert nx * ny == capi.IFDLBM_STATIC_MAX_NODES
    g = torch.Generator(device="cuda").manual_seed(2306)
    u0, v0, p0 = (torch.randn(ny, nx, dtype=torch.float64, device="cuda", generator=g)
                  for _ in range(3))
    u1, v1, p1 = (a + 1e-3 * torch.randn(ny, nx, dtype=torch.float64, device="cuda", generator=g)
                  for a in (u0, v0, p0))
    u1[ny // 2, nx - 1] += 0.5             # the maximum sits in the last slot's neighbourhood
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        capi.ifdlbm_residual_fields_static(nx, ny, u1, v1, p1, u0, v0, p0, out, 0)
        torch.cuda.synchronize()
        du2 = (u1 - u0) ** 2 + (v1 - v0) ** 2
        u2 = u1 ** 2 + v1 ** 2
        ref = [torch.sqrt(du2.sum() / u2.sum()).item(),
               torch.sqrt(((p1 - p0) ** 2).sum() / (p1 ** 2).sum()).item(),
               torch.sqrt(du2.max() / u2.max()).item()]
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=0)


def test_static_residual_rejects_fields_beyond_its_scratch():
    """The C entry point itself refuses sizes beyond its array (before any
    launch, so the 1-element buffers below are never read)."""
    import ctypes

    import torch

    from paper_2306_07603_gb300 import capi

    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    n = capi.IFDLBM_STATIC_MAX_NODES
    rc = capi.load_library().ifdlbm_residual_fields_static(n + 1, 1, p, p, p, p, p, p, p,
                                                           ctypes.c_void_p(0))
    assert rc == capi.IFDLBM_ERR_INVALID_ARG
    assert "exceed" in capi.ifdlbm_last_error()
    # the binding refuses it as well, before the library sees it
    with pytest.raises(ValueError):
        capi.ifdlbm_residual_fields_static(n + 1, 1, t, t, t, t, t, t, t, 0)
