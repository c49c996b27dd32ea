"""The oracle at theta = 90 deg against a separately written Cartesian step.

At theta = 90 deg the map of Eq. (3.8.1) is the identity (cot theta = 0
exactly), every metric term of Eqs. (3.2)-(3.4) is 0 or 1, and Eqs. (3.6)-(3.7)
are the Cartesian evolution equations. ``oracle/cartesian.py`` writes that
Cartesian step again from the paper's equations, sharing no function with
``oracle.step``; the two must agree to rounding over many steps of a developed
cavity. A transposed metric, a wrong sign of x_eta, a swapped (xi, eta) axis or
a contravariant velocity that is not c e_i on the square would all break it.
"""
import numpy as np

import oracle as O
from oracle.cartesian import feq_cart, moments_cart, step_cart


def test_cartesian_pieces_agree_with_the_general_oracle_pieces():
    rng = np.random.default_rng(7)
    P, ux, uy = rng.normal(0, 1e-3, 5), rng.normal(0, 0.05, 5), rng.normal(0, 0.05, 5)
    a = np.stack(feq_cart(P, ux, uy))
    b = O.equilibrium(P, ux, uy)
    assert np.abs(a - b).max() < 1e-16
    m = moments_cart(list(a))
    assert np.abs(m[0] - ux).max() < 1e-16 and np.abs(m[1] - uy).max() < 1e-16
    assert np.abs(m[2] - P).max() < 1e-15


def test_theta90_step_equals_cartesian_step_over_100_steps():
    N, Re, n = 33, 100.0, 0.75
    run = O.cavity_run(N, Re, n, theta_deg=90.0)
    run.advance(200)                                    # a developed, non-trivial state
    prm = run.prm
    fa, la = run.fhat.copy(), run.lam.copy()
    fb, lb = fa.copy(), la.copy()
    scale = np.abs(fa).max()
    for _ in range(100):
        fa, la = O.step(fa, la, run.g, prm)
        fb, lb = step_cart(fb, lb, 0.1, prm.K, prm.n, prm.dt, prm.eta_b, prm.gamma_min)
    assert np.abs(fa - fb).max() <= 1e-13 * scale
    # lambda: where the shear nears the zero-shear clamp, the rounding of
    # f - f^eq is amplified by |n - 1| / (lam c_s^2 gamma-dot) (Eqs. 2.12-2.14);
    # measured 7e-13 of max lambda, while f-hat agrees to 2e-15
    assert np.abs(la - lb).max() <= 1e-11 * np.abs(la).max()
    # the flow is developed: the lid has set up a velocity field
    ux, uy, _ = O.macros(fa)
    assert np.sqrt(ux ** 2 + uy ** 2)[1:-1, 1:-1].max() > 0.02


def test_cartesian_step_detects_a_skewed_grid():
    """At theta = 75 deg the two differ at first order: the comparison above
    is not vacuous."""
    N = 17
    run = O.cavity_run(N, 100.0, 1.0, theta_deg=75.0)
    run.advance(20)
    prm = run.prm
    fa, _ = O.step(run.fhat, run.lam, run.g, prm)
    fb, _ = step_cart(run.fhat, run.lam, 0.1, prm.K, prm.n, prm.dt, prm.eta_b, prm.gamma_min)
    assert np.abs(fa - fb).max() > 1e-6
