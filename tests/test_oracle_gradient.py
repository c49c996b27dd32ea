"""The oracle's reference gradient: complex-step differentiation of the
kinetic energy (Eq. 5.1) after T steps with respect to n, Re and theta.

The oracle takes every branch (upwind side, clamps) on real parts, so a
complex perturbation i h of a parameter carries the exact derivative of its
discrete map in the imaginary part (Squire & Trapp 1998). It is pinned here
against central finite differences of the real oracle, an independent
method."""
import numpy as np
import pytest

import oracle as O


def energy(n, Re, theta, N=21, T=25):
    run = O.cavity_run(N, Re, n, theta_deg=theta, dt_mode="grid")  # dt fixed under theta
    run.advance(T)
    ux, uy, _ = O.macros(run.fhat)
    return O.kinetic_energy(ux, uy, run.g)


def complex_step(fun, x, k, h=1e-30):
    xs = [complex(v) for v in x]
    xs[k] += 1j * h
    return np.imag(fun(*xs)) / h


@pytest.mark.parametrize("k", [0, 1, 2])
def test_complex_step_gradient_matches_central_differences(k):
    x = [0.75, 400.0, 60.0]
    g_cs = complex_step(energy, x, k)
    hk = 1e-5 * abs(x[k])
    xp, xm = list(x), list(x)
    xp[k] += hk
    xm[k] -= hk
    g_fd = (energy(*xp) - energy(*xm)) / (2 * hk)
    assert g_cs != 0.0
    assert abs(g_cs - g_fd) <= 1e-6 * abs(g_cs), (g_cs, g_fd)
    # the real part of the complex run is the real energy
    xs = [complex(v) for v in x]
    xs[k] += 1e-30j
    assert abs(np.real(energy(*xs)) - energy(*x)) <= 1e-15 * energy(*x)
