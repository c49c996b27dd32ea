"""Pins of the oracle's implicit relaxation time (the implicit form of
Eq. 2.14: the strain rate taken at the lam being solved for).

With gamma-dot(lam) = a / (2 lam + dt), the equation
lam = C max(gamma-dot(lam), gamma_min)^(n-1) (C = K / c_s^2) has closed
forms: n = 1 gives lam = C; n = 2 gives 2 lam^2 + dt lam - C a = 0; n = 1/2
gives lam^2 - (2 C^2 / a) lam - C^2 dt / a = 0; and the clamped branch gives
lam = C gamma_min^(n-1). a is recovered from the lagged functions (Eqs.
2.12-2.13, 2.18), which are pinned on their own, as a = gamma-dot(lam') (2
lam' + dt) for any lam'. The implicit root is also the fixed point of the
lagged map: lagging with lam_prev = the root returns the root.
"""
import numpy as np
import pytest

import oracle as O


def _state(n, Re=400.0, steps=30):
    run = O.cavity_run(33, Re, n, theta_deg=60.0)
    run.advance(steps)
    f = run.fhat
    ux, uy, P = O.macros(f)
    return run, f, O.equilibrium(P, ux, uy)


def _lagged_gdot(f, feq, lam_p, dt):
    fl = O.f_from_fhat(f, feq, lam_p, dt)
    return O.shear_rate(*O.strain_rate(fl, feq, lam_p))


def _a_and_its_rounding(f, feq, lam, dt):
    """a = gamma-dot(lam') (2 lam' + dt), recovered through the lagged functions.
    f^ne = f - f^eq is a difference of O(w_i) numbers, so it carries an
    absolute rounding of about eps max|f-hat| per population, and f^ne is
    2 lam'/(2 lam' + dt) of f-hat - f^eq: a's rounding is bounded by
    32 eps max|f-hat| / c_s^2 times (2 lam' + dt)/(2 lam')."""
    a = _lagged_gdot(f, feq, lam, dt) * (2.0 * lam + dt)
    return a, 32.0 * np.finfo(float).eps * np.abs(f).max() * 3.0 * (2.0 * lam + dt) / (2.0 * lam)


def test_newtonian_limit_is_K_over_cs2():
    run, f, feq = _state(1.0)
    p = run.prm
    lam = O.relaxation_time_implicit(f, feq, p.dt, p.K, 1.0, p.gamma_min)
    assert np.abs(lam - p.K * 3.0).max() <= 1e-15 * p.K * 3.0


@pytest.mark.parametrize("n", [2.0, 0.5])
def test_closed_forms_n2_and_n_half(n):
    run, f, feq = _state(0.75)
    p = run.prm
    C, dt = p.K * 3.0, p.dt
    a, da = _a_and_its_rounding(f, feq, run.lam, dt)
    lam = O.relaxation_time_implicit(f, feq, dt, p.K, n, p.gamma_min)
    if n == 2.0:
        ref = (-dt + np.sqrt(dt * dt + 8.0 * C * a)) / 4.0
    else:
        b = C * C / np.maximum(a, 1e-300)
        ref = b + np.sqrt(b * b + b * dt)
    free = a / (2.0 * ref + dt) > p.gamma_min * (1 + 1e-9)
    clamped = ~free & (a / (2.0 * C * p.gamma_min ** (n - 1) + dt) <= p.gamma_min)
    assert free.sum() > 100 and clamped.sum() > 0
    # d ln lam / d ln a is (2 lam + dt)/(4 lam + dt) <= 1 (n = 2) or <= 1/2 (n = 1/2)
    bound = 1e-13 * ref + ref * da / np.maximum(a, 1e-300)
    assert np.all(np.abs(lam - ref)[free] <= bound[free])
    assert np.median(np.abs(lam - ref)[free] / ref[free]) <= 1e-12
    assert np.allclose(lam[clamped], C * p.gamma_min ** (n - 1), rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [0.5, 0.75, 1.5])
def test_implicit_root_is_the_fixed_point_of_the_lagged_map(n):
    run, f, feq = _state(n)
    p = run.prm
    lam = O.relaxation_time_implicit(f, feq, p.dt, p.K, n, p.gamma_min)
    lagged = O.relaxation_time(_lagged_gdot(f, feq, lam, p.dt), p.K, n, p.gamma_min)
    a, da = _a_and_its_rounding(f, feq, lam, p.dt)
    bound = 1e-13 * lam + abs(n - 1.0) * lam * da / np.maximum(a, 1e-300)
    assert np.all(np.abs(lagged - lam) <= bound)
    assert np.median(np.abs(lagged - lam) / lam) <= 1e-13


def test_rest_state_takes_the_clamp():
    run = O.cavity_run(17, 100.0, 0.75, theta_deg=60.0)
    ux, uy, P = O.macros(run.fhat)
    feq = O.equilibrium(P, ux, uy)
    p = run.prm
    lam = O.relaxation_time_implicit(run.fhat, feq, p.dt, p.K, 0.75, p.gamma_min)
    inner = lam[1:-1, 1:-1]
    assert np.allclose(inner, p.K * 3.0 * p.gamma_min ** (-0.25), rtol=1e-14, atol=0)


def test_implicit_step_runs_and_differs_from_lagged_only_in_transient():
    """The implicit and lagged runs share steady states; during the start-up
    they differ (lam follows the shear at once instead of one step late)."""
    a = O.cavity_run(17, 100.0, 0.75, theta_deg=60.0, implicit_lambda=True)
    b = O.cavity_run(17, 100.0, 0.75, theta_deg=60.0)
    a.advance(20)
    b.advance(20)
    assert a.prm.implicit_lambda and not b.prm.implicit_lambda
    assert np.all(np.isfinite(a.fhat)) and 0 < np.abs(a.lam - b.lam).max() < 0.5 * np.abs(b.lam).max()
