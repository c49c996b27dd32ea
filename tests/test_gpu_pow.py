"""The FP64 power of the power-law viscosity (Eq. 1.4) against CUDA's pow.

The library evaluates max(q, gamma_min^2)^((n-1)/2) with a table-driven
method (Tang, ACM TOMS 1989/1990). Over the range the power law meets
(q = |gamma-dot|^2 in [1e-12, 1e8], exponents (n-1)/2 for n in (0, 3]) its
relative error from CUDA's pow must stay within the bound derived from its
roundings, 5e-16 + 2.2e-16 |m log2 x| (log2 x and m log2 x are single
doubles), and the Newtonian exponent 0 must give exactly 1.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    from paper_2306_07603_gb300.solver import Solver, cavity
    s = Solver([cavity(9, 9, 100.0, 0.75)])
    yield s
    s.close()


def _run(s, x, m):
    import torch

    from paper_2306_07603_gb300 import capi
    xd = torch.as_tensor(x, dtype=torch.float64, device="cuda")
    fast = torch.empty_like(xd)
    ref = torch.empty_like(xd)
    capi.ifdlbm_selftest_pow(s.h, xd, m, fast, ref)
    s.stream.synchronize()
    return fast.cpu().numpy(), ref.cpu().numpy()


@pytest.mark.parametrize("m", [-0.5, -0.375, -0.25, -0.125, 0.125, 0.25, 0.5, 0.73, 1.0])
def test_pow_fast_relative_error(handle, m):
    rng = np.random.default_rng(12345)
    x = 10.0 ** rng.uniform(-12, 8, size=200000)
    # table-cell boundaries and exact powers of two
    j = np.arange(256)
    edges = np.concatenate([1 + j / 256.0, 1 + (j + 0.5) / 256.0, np.nextafter(1 + j / 256.0, 0)])
    x = np.concatenate([x, edges, edges * 2.0 ** -20, 2.0 ** np.arange(-40, 27)])
    fast, ref = _run(handle, x, m)
    bound = 5e-16 + 2.2e-16 * np.abs(m * np.log2(x))
    rel = np.abs(fast - ref) / np.abs(ref)
    assert np.all(rel <= bound), (m, (rel / bound).max(), x[np.argmax(rel / bound)])
    rel_np = np.abs(fast - np.power(x, m)) / np.power(x, m)
    assert np.all(rel_np <= bound + 2.3e-16)


def test_pow_fast_newtonian_exponent_is_exactly_one(handle):
    x = 10.0 ** np.linspace(-12, 8, 1001)
    fast, _ = _run(handle, x, 0.0)
    assert np.all(fast == 1.0)


@pytest.mark.parametrize("m", [-0.5, -0.375, -0.25, -0.125, 0.125, 0.25, 0.5, 0.73, 1.0])
def test_pow_f32_relative_error(handle, m):
    """The FP32 power of the FP32-deviation form: relative error from the
    exact float(x)^float(m) within 3e-7 + 1.3e-7 |m log2 x| (the roundings of
    log2 x and of m log2 x, and the ulps of log2f and exp2f)."""
    import torch

    from paper_2306_07603_gb300 import capi
    rng = np.random.default_rng(23456)
    x = 10.0 ** rng.uniform(-12, 8, size=200000)
    x = np.concatenate([x, 2.0 ** np.arange(-40, 27), 1.0 + np.arange(256) / 256.0])
    xf = x.astype(np.float32).astype(np.float64)
    mf = float(np.float32(m))
    xd = torch.as_tensor(xf, dtype=torch.float64, device="cuda")
    out = torch.empty_like(xd)
    capi.ifdlbm_selftest_pow_f32(handle.h, xd, m, out)
    handle.stream.synchronize()
    got = out.cpu().numpy()
    exact = np.power(xf, mf)
    rel = np.abs(got - exact) / exact
    bound = 3e-7 + 1.3e-7 * np.abs(mf * np.log2(xf))
    assert np.all(rel <= bound), (m, (rel / bound).max(), xf[np.argmax(rel / bound)])


def test_pow_f32_newtonian_exponent_is_exactly_one(handle):
    import torch

    from paper_2306_07603_gb300 import capi
    xd = torch.as_tensor((10.0 ** np.linspace(-12, 8, 1001)).astype(np.float32).astype(np.float64),
                         device="cuda")
    out = torch.empty_like(xd)
    capi.ifdlbm_selftest_pow_f32(handle.h, xd, 0.0, out)
    handle.stream.synchronize()
    assert np.all(out.cpu().numpy() == 1.0)


# n of the FP32-deviation handles below: power-law indices of the paper's
# sweeps and beyond (m = (n - 1)/2 from -0.45 to 1)
POW_TAB_N = [0.1, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0, 3.0]


def _exact_power(xf, m, C):
    """C xf^m to ~40 significant digits (the decimal module's ln and exp)."""
    import decimal

    ctx = decimal.Context(prec=45)
    D = decimal.Decimal                         # exact value of a binary double
    return np.array([float(ctx.multiply(D(C), ctx.exp(ctx.multiply(D(m), ctx.ln(D(float(v)))))))
                     for v in xf])


@pytest.mark.parametrize("n", POW_TAB_N)
def test_pow_tab_relative_error(n):
    """The FP64 power the FP32-deviation form applies to its FP32 strain rate
    (Eq. 1.4, lambda = K/c_s^2 q^((n-1)/2)): within 6e-16 of the exact value
    (the table roundings, three FP64 roundings and the truncated series),
    and within that plus 3 ulp of C * CUDA's pow; every float argument of the
    cavity's range, table-cell boundaries and exact powers of two included."""
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import Solver, cavity
    s = Solver([cavity(9, 9, 100.0, n)], precision="fp32dev")
    info = s.info(0)
    rng = np.random.default_rng(34567)
    x = 10.0 ** rng.uniform(-12, 8, size=200000)
    j = np.arange(256)
    edges = np.concatenate([1 + j / 256.0, 1 + (j + 0.5) / 256.0, 1 + (j + 1) / 256.0 - 2.0 ** -23])
    x = np.concatenate([x, edges, edges * 2.0 ** -20, edges * 2.0 ** 13, 2.0 ** np.arange(-40, 27),
                        [np.finfo(np.float32).tiny, 3.0e38]])
    xf = x.astype(np.float32).astype(np.float64)
    xd = torch.as_tensor(xf, device="cuda")
    out = torch.empty(2 * len(xf), dtype=torch.float64, device="cuda")
    capi.ifdlbm_selftest_pow_tab(s.h, 0, xd, out)
    s.stream.synchronize()
    o = out.cpu().numpy()
    got, ref = o[:len(xf)], o[len(xf):]
    m = (n - 1.0) / 2.0
    # the library's C = K / c_s^2 (K = U^(2-n) H^n / Re): its reference at x = 1,
    # where CUDA's pow(1, m) = 1 exactly
    C = float(ref[np.flatnonzero(xf == 1.0)[0]])
    K = 0.1 ** (2.0 - n) / 100.0
    assert abs(C / (3.0 * K) - 1.0) < 1e-15 and info.nx == 9
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.all(rel <= 6e-16 + 3.4e-16), (n, rel.max(), xf[np.argmax(rel)])
    idx = np.concatenate([np.arange(0, 200000, 97), np.arange(200000, len(xf))])
    exact = _exact_power(xf[idx], m, C)
    rel_x = np.abs(got[idx] - exact) / exact
    assert np.all(rel_x <= 6e-16), (n, rel_x.max(), xf[idx][np.argmax(rel_x)])
    if n == 1.0:
        assert np.all(got == C)
    s.close()
