"""The allocation-free residual entry point (ifdlbm_residual_fields_static).

It serves callers that must not allocate device memory. Here it is called
through the C ABI on device fields taken from a cavity before and after a
step, twice in a row, and must agree with the handle's own residual
(ifdlbm_residual) within the residual tolerance of the parity tests.
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
        capi.ifdlbm_residual_fields_static(nx, ny, u1, v1, p1, u0, v0, p0, out,
                                           stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), (call, got)
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0, err_msg=f"call {call}")


def test_static_residual_rejects_fields_beyond_its_scratch():
    import torch

    from paper_2306_07603_gb300 import capi

    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = capi.IFDLBM_STATIC_MAX_NODES
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_residual_fields_static(n + 1, 1, t, t, t, t, t, t, t, 0)
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG and "exceed" in str(e.value)
