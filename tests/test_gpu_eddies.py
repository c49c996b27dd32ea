"""Tables 1-3 of the paper, reproduced: steady Re = 100 eddy centres in the
trapezoidal cavity for theta in {75, 60, 45} deg and n in {1.5, 1, 0.75, 0.5}.

All twelve cavities run as one batch on a 257^2 grid (the paper's 256^2
cells) in FP32-deviation storage for 300k steps from rest (the centres move
by less than 2e-4 between 300k and 400k steps); ifdlbm_eddies locates the
centres. The paper's values (tests/golden/eddy_centres_re100.txt) come from
its own solver on its own grid, so the bar is in grid spacings of this grid:
dx = (L + 2 H cot theta)/256 (the widest row), dy = H/256.

* primary eddy: within 1 spacing for n >= 0.75 (measured <= 0.65), within
  3.5 for n = 0.5 (measured <= 2.9; the strongly shear-thinning cases, where
  the zero-shear clamp, which the paper does not give, shapes the slow core);
* bottom-corner eddies, where the tables give them: found, within 2 spacings.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, STEPS = 257, 300000


def test_tables_1_to_3_eddy_centres(golden_dir):
    from paper_2306_07603_gb300.solver import Solver, cavity
    rows = np.loadtxt(os.path.join(golden_dir, "eddy_centres_re100.txt"))
    s = Solver([cavity(N, N, 100.0, float(r[1]), theta_deg=float(r[0])) for r in rows],
               precision="fp32dev")
    s.step(STEPS)
    bad = []
    for k, r in enumerate(rows):
        th, n = float(r[0]), float(r[1])
        dx = (1.0 + 2.0 / math.tan(math.radians(th))) / (N - 1)
        dy = 1.0 / (N - 1)
        e = s.eddies(k)
        lim = 1.0 if n >= 0.75 else 3.5
        p = e[0]
        if not (p.found and abs(p.x - r[2]) <= lim * dx and abs(p.y - r[3]) <= lim * dy):
            bad.append(("primary", th, n, p.x, p.y, r[2], r[3]))
        for side, (cx, cy) in ((1, (r[4], r[5])), (2, (r[6], r[7]))):
            if np.isnan(cx):
                continue
            q = e[side]
            if not (q.found and abs(q.x - cx) <= 2 * dx and abs(q.y - cy) <= 2 * dy):
                bad.append(("corner", side, th, n, q.found, q.x, q.y, cx, cy))
    s.close()
    assert not bad, bad
