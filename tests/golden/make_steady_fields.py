"""Writes the oracle's steady fields of the 65 x 65 cavity to a compressed .npz.

Cavity: theta = 60 deg, n = 0.75, Re = 100, U = 0.1, L = H = 1 (the FP64
validation case of Sec. 5.1's parameters), advanced from rest by the FP64
oracle for STEPS steps (default contravariant time-step rule), by which the
per-step max-norm residual is about 1e-11. The
file holds u, v, P, psi (Eqs. 2.10-2.11; psi integrated along xi lines) and
the residuals of Eq. (2.19) of the last step. Only the oracle is called.

    python tests/golden/make_steady_fields.py      # ~13 min on one core
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

N, RE, N_POW, THETA = 65, 100.0, 0.75, 60.0
STEPS = 130000
OUT = os.path.join(HERE, "steady_65_theta60_n075_re100.npz")


def main():
    run = O.cavity_run(N, RE, N_POW, theta_deg=THETA)
    run.advance(STEPS - 1)
    run.advance(1, record=True)
    f = run.fields()
    Eu, EP, Rinf = run.history[-1]
    np.savez_compressed(OUT, u=f["u"], v=f["v"], P=f["P"], psi=f["psi"], steps=STEPS,
                        last_residual=np.array([Eu, EP, Rinf]),
                        case=np.array([N, N, RE, N_POW, THETA]))
    print(OUT, STEPS, Eu, EP, Rinf)


if __name__ == "__main__":
    main()
