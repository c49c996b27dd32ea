"""Pins of the oracle's lattice-level pieces against what the paper and the
mathematics fix (closed forms, moment identities, Chapman-Enskog relations).

None of these retypes the oracle's formula: each checks it against an
independent statement (a moment of Eq. (A1), a defining relation of
Eqs. (2.3)-(2.4), a lattice-isotropy identity, a textbook special case).
"""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(20230607)


def _rand_macros(shape, c=1.0):
    P = 1e-2 * RNG.standard_normal(shape)
    ux = 0.1 * c * RNG.standard_normal(shape)
    uy = 0.1 * c * RNG.standard_normal(shape)
    return P, ux, uy


@pytest.mark.parametrize("c,rho0", [(1.0, 1.0), (2.0, 1.0), (1.0, 0.7)])
def test_equilibrium_moments_eqA1(c, rho0):
    """Eq. (A1): sum f^eq = rho0, sum c f^eq = u, sum c c f^eq = (P + c_s^2 rho0) I + u u."""
    P, ux, uy = _rand_macros((50,), c)
    fe = O.equilibrium(P, ux, uy, rho0, c)
    cs2 = c * c / 3.0
    ex = (O.EX * c)[:, None]
    ey = (O.EY * c)[:, None]
    np.testing.assert_allclose(fe.sum(0), rho0, rtol=0, atol=1e-14)
    np.testing.assert_allclose((ex * fe).sum(0), ux, rtol=0, atol=1e-14)
    np.testing.assert_allclose((ey * fe).sum(0), uy, rtol=0, atol=1e-14)
    np.testing.assert_allclose((ex * ex * fe).sum(0), P + cs2 * rho0 + ux * ux, rtol=0, atol=1e-14)
    np.testing.assert_allclose((ey * ey * fe).sum(0), P + cs2 * rho0 + uy * uy, rtol=0, atol=1e-14)
    np.testing.assert_allclose((ex * ey * fe).sum(0), ux * uy, rtol=0, atol=1e-14)


def test_equilibrium_third_moment_is_isotropic_velocity_term():
    """Eq. (A1), third moment: sum c_a c_b c_g f^eq = c_s^2 (u_a d_bg + u_b d_ag + u_g d_ab)."""
    P, ux, uy = _rand_macros((20,))
    fe = O.equilibrium(P, ux, uy)
    cs2 = 1.0 / 3.0
    ex, ey = O.EX[:, None], O.EY[:, None]
    np.testing.assert_allclose((ex ** 3 * fe).sum(0), 3 * cs2 * ux, atol=1e-14)
    np.testing.assert_allclose((ex ** 2 * ey * fe).sum(0), cs2 * uy, atol=1e-14)
    np.testing.assert_allclose((ex * ey ** 2 * fe).sum(0), cs2 * ux, atol=1e-14)
    np.testing.assert_allclose((ey ** 3 * fe).sum(0), 3 * cs2 * uy, atol=1e-14)


def test_weights_eq29():
    """Eq. (2.9): the weights sum to one; wbar sums to zero, so P carries no mass."""
    assert abs(O.OMEGA.sum() - 1.0) < 1e-16
    assert abs(O.OMEGA_BAR.sum()) < 1e-16
    # second-order lattice isotropy: sum w c c = c_s^2 I
    assert abs((O.OMEGA * O.EX * O.EX).sum() - 1 / 3) < 1e-16
    assert abs((O.OMEGA * O.EX * O.EY).sum()) < 1e-16


@pytest.mark.parametrize("c", [1.0, 2.0])
def test_macros_invert_equilibrium(c):
    """Eqs. (2.10)-(2.11) applied to f^eq(P, u) return (u, P)."""
    P, ux, uy = _rand_macros((30,), c)
    ux2, uy2, P2 = O.macros(O.equilibrium(P, ux, uy, 1.0, c), 1.0, c)
    np.testing.assert_allclose(ux2, ux, atol=1e-15)
    np.testing.assert_allclose(uy2, uy, atol=1e-15)
    np.testing.assert_allclose(P2, P, atol=1e-15)


def test_macros_agree_for_fhat_f_fbar():
    """Eqs. (2.10)-(2.11): u and P are the same from f, f-bar and f-hat."""
    P, ux, uy = _rand_macros((40,))
    fe = O.equilibrium(P, ux, uy)
    fhat = fe + 1e-3 * RNG.standard_normal(fe.shape)
    uxh, uyh, Ph = O.macros(fhat)
    feq = O.equilibrium(Ph, uxh, uyh)
    lam, dt = 0.01 + RNG.random(40) * 0.1, 0.0078
    for F in (O.f_from_fhat(fhat, feq, lam, dt), O.fbar_plus(fhat, feq, lam, dt),
              O.fhat_plus(fhat, feq, lam, dt)):
        a, b, p = O.macros(F)
        np.testing.assert_allclose(a, uxh, atol=1e-15)
        np.testing.assert_allclose(b, uyh, atol=1e-15)
        np.testing.assert_allclose(p, Ph, atol=1e-15)


@pytest.mark.parametrize("dt", [0.0078125, 0.1])
def test_transforms_match_bgk_definitions_eq23_24(dt):
    """Eqs. (2.15)-(2.18) against the defining relations Eqs. (2.3)-(2.4) with
    the BGK operator Omega = -(f - f^eq)/lam of Eq. (2.0):

    f-hat = f - dt/2 Omega, f-hat^+ = f + dt/2 Omega,
    f-bar = f - dt/4 Omega, f-bar^+ = f + dt/4 Omega.
    """
    shape = (9, 25)
    f = 0.1 + RNG.random(shape)
    feq = 0.1 + RNG.random(shape)
    lam = 0.001 + RNG.random(25)
    omega = -(f - feq) / lam
    fhat = f - 0.5 * dt * omega
    fhat_p = f + 0.5 * dt * omega
    fbar = f - 0.25 * dt * omega
    fbar_p = f + 0.25 * dt * omega
    np.testing.assert_allclose(O.f_from_fhat(fhat, feq, lam, dt), f, rtol=1e-13)
    np.testing.assert_allclose(O.fhat_plus(fhat, feq, lam, dt), fhat_p, rtol=1e-12)
    np.testing.assert_allclose(O.fbar_plus(fhat, feq, lam, dt), fbar_p, rtol=1e-12)
    np.testing.assert_allclose(O.f_from_fbar(fbar, feq, lam, dt), f, rtol=1e-13)


def test_strain_rate_recovers_velocity_gradient_chapman_enskog():
    """Eq. (2.12) with f^ne = -lam c_i.grad f^eq (first Chapman-Enskog order,
    Eq. (A6.2) for a steady linear, divergence-free velocity field) returns
    grad u + grad u^T exactly (Eq. (A11), fourth-order lattice isotropy)."""
    for _ in range(5):
        a, b, d = RNG.standard_normal(3) * 0.01  # grad u = [[a, b], [d, -a]]
        lam = 0.003 + 0.01 * RNG.random()
        # c_i.grad (c_i.u) = c_i c_i : grad u, only the linear term of f^eq varies
        cc_gradu = (O.EX * O.EX * a + O.EX * O.EY * (b + d) - O.EY * O.EY * a)
        fne = -lam * O.OMEGA * cc_gradu / (1.0 / 3.0)
        feq = O.equilibrium(np.zeros(1), np.zeros(1), np.zeros(1))
        f = feq + fne[:, None]
        Sxx, Sxy, Syy = O.strain_rate(f, feq, lam)
        np.testing.assert_allclose(Sxx, 2 * a, atol=1e-15)
        np.testing.assert_allclose(Sxy, b + d, atol=1e-15)
        np.testing.assert_allclose(Syy, -2 * a, atol=1e-15)


def test_shear_rate_textbook_cases():
    """|gamma-dot| = sqrt(2 D:D): simple shear u = (g y, 0) gives |g|; planar
    extension u = (e x, -e y) gives 2|e| (textbook kinematics)."""
    g = 0.37
    assert abs(O.shear_rate(0.0, g, 0.0) - g) < 1e-16
    e = 0.21
    assert abs(O.shear_rate(2 * e, 0.0, -2 * e) - 2 * e) < 1e-16


def test_relaxation_time_newtonian_and_clamp():
    """Eq. (2.14): n = 1 gives the Newtonian lam = nu / c_s^2 for every shear
    rate; below the clamp the shear-rate dependence stops."""
    gd = np.array([0.0, 1e-6, 0.3, 5.0])
    lam = O.relaxation_time(gd, 0.02, 1.0, 1e-4)
    np.testing.assert_allclose(lam, 0.02 * 3.0, rtol=1e-15)
    lam = O.relaxation_time(np.array([0.0, 1e-5, 1e-4]), 0.02, 0.5, 1e-4)
    assert lam[0] == lam[1] == lam[2]
    # shear thinning: lam decreases with shear for n < 1, increases for n > 1
    l_thin = O.relaxation_time(np.array([0.01, 0.1]), 0.02, 0.5, 1e-4)
    l_thick = O.relaxation_time(np.array([0.01, 0.1]), 0.02, 1.5, 1e-4)
    assert l_thin[1] < l_thin[0] and l_thick[1] > l_thick[0]
    # one decade of shear changes mu by a factor 10^(n-1)
    np.testing.assert_allclose(l_thin[1] / l_thin[0], 10 ** (-0.5), rtol=1e-14)


def test_consistency_coefficient_newtonian_reynolds():
    """Eq. (2.15.1) at n = 1 is the Newtonian Re = U H / nu."""
    assert abs(O.consistency_coefficient(100.0, 1.0, 0.1, 1.0) - 0.1 * 1.0 / 100.0) < 1e-18
    # dimensional consistency: K scales as H^n at fixed U, Re
    k1 = O.consistency_coefficient(100.0, 0.75, 0.1, 1.0)
    k2 = O.consistency_coefficient(100.0, 0.75, 0.1, 2.0)
    assert abs(k2 / k1 - 2 ** 0.75) < 1e-14


def test_half_step_collision_is_inverted_pointwise():
    """The half step's collision, f(t + dt/2) = f_from_fbar(f-bar, f^eq(f-bar))
    (Eq. 2.17), keeps u and P, so f^eq of f(t + dt/2) is f^eq of f-bar and
    f-bar = (f - bh f^eq) / ah with ah = 4 lam / (4 lam + dt), bh = dt /
    (4 lam + dt): the pointwise recovery the adjoint of the half step uses
    instead of evaluating the stencil again. Checked on the stages of one
    oracle step of a developed cavity, at its interior nodes."""
    import oracle as O
    run = O.cavity_run(25, 400.0, 0.75, theta_deg=60.0, ny=21)
    run.advance(30)
    _, _, st = O.step(run.fhat, run.lam, run.g, run.prm, return_stages=True)
    fbar, fh, lam, dt = st["fbar_half"], st["f_half"], st["lam"], run.prm.dt
    inner = (slice(None), slice(1, -1), slice(1, -1))
    ub, vb, Pb = O.macros(fbar)
    uh, vh, Ph = O.macros(fh)
    # the moments agree to the rounding of the populations they are summed from
    for a, b in ((ub, uh), (vb, vh), (Pb, Ph)):
        assert np.abs(a[1:-1, 1:-1] - b[1:-1, 1:-1]).max() <= 1e-15 * np.abs(fh).max()
    feq = O.equilibrium(Ph, uh, vh)
    ah, bh = 4.0 * lam / (4.0 * lam + dt), dt / (4.0 * lam + dt)
    rec = (fh - bh * feq) / ah
    assert np.abs(rec[inner] - fbar[inner]).max() <= 1e-14 * np.abs(fbar[inner]).max()
    # a wrong weight (bh and ah swapped) is caught
    bad = (fh - ah * feq) / bh
    assert np.abs(bad[inner] - fbar[inner]).max() > 1e-6 * np.abs(fbar[inner]).max()
