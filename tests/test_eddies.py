"""Eddy-centre finder (Tables 1-3): oracle pins and the library's host finder.

The oracle's finder (``oracle.eddy_centres``, NumPy least squares) is pinned
on fields whose extrema are known in closed form: a quadratic bowl (the
least-squares quadratic is then exact, so the centre is recovered to
rounding), corner bumps, and the map of Eq. (3.8.1). The library's
``ifdlbm_find_eddies`` (host C++, orthogonal-basis projections) must agree
with it on the same fields and on the oracle's steady 65^2 cavity. No GPU is
needed: the finder is host code.
"""
import os

import numpy as np
import pytest

import oracle as O


def _grid(nx, ny):
    return np.linspace(0, 1, nx)[None, :], np.linspace(0, 1, ny)[:, None]


def _bowl(nx, ny, xc, yc):
    xi, eta = _grid(nx, ny)
    return 3 * (xi - xc) ** 2 + 2 * (eta - yc) ** 2 + 0.5 * (xi - xc) * (eta - yc) - 1.0


def _with_corner_eddies(nx, ny, left=(0.13, 0.07), right=(0.83, 0.11), amp=1e-3):
    """A bowl plus two positive quadratic caps centred at `left` and `right`."""
    xi, eta = _grid(nx, ny)
    psi = _bowl(nx, ny, 0.5, 0.6) * 1e-2 - 1e-2
    for (xc, yc) in (left, right):
        r2 = ((xi - xc) / 0.05) ** 2 + ((eta - yc) / 0.04) ** 2
        psi = np.where(r2 < 1.0, amp * (1.0 - r2), psi)
    return psi


def test_oracle_finder_recovers_off_node_minimum_exactly():
    e = O.eddy_centres(_bowl(41, 31, 0.4123, 0.6311), 1.0, 1.0, 60.0)
    p = e[0]
    assert p["refined"]
    assert abs(p["xi"] - 0.4123) < 1e-12 and abs(p["eta"] - 0.6311) < 1e-12
    x, y = O.trapezoid_xy(0.4123, 0.6311, 1.0, 1.0, 60.0)
    assert abs(p["x"] - x) < 1e-12 and abs(p["y"] - y) < 1e-12
    assert abs(p["psi"] + 1.0) < 1e-12
    assert e[1] is None and e[2] is None


def test_oracle_finder_corner_eddies():
    e = O.eddy_centres(_with_corner_eddies(101, 81), 1.0, 1.0, 75.0)
    # quadratic caps: their maxima are exact quadratics near the centre
    assert abs(e[1]["xi"] - 0.13) < 1e-9 and abs(e[1]["eta"] - 0.07) < 1e-9
    assert abs(e[2]["xi"] - 0.83) < 1e-9 and abs(e[2]["eta"] - 0.11) < 1e-9
    assert e[1]["psi"] == pytest.approx(1e-3, rel=1e-9)


def test_oracle_finder_ignores_upper_half_and_negative_maxima():
    psi = _with_corner_eddies(101, 81, left=(0.13, 0.8), right=(0.83, 0.11), amp=-1e-4)
    e = O.eddy_centres(psi, 1.0, 1.0, 60.0)
    assert e[1] is None and e[2] is None


def _lib_eddies(psi, theta):
    from paper_2306_07603_gb300 import capi
    ny, nx = psi.shape
    return capi.ifdlbm_find_eddies(nx, ny, (1.0, 1.0, theta), np.ascontiguousarray(psi))


def _agree(lib, orc, tol):
    assert bool(lib.found) == (orc is not None)
    if orc is None:
        return
    assert (lib.i, lib.j, bool(lib.refined)) == (orc["i"], orc["j"], orc["refined"])
    for k in ("x", "y", "xi", "eta"):
        assert abs(getattr(lib, k) - orc[k]) <= tol, (k, getattr(lib, k), orc[k])
    assert abs(lib.psi - orc["psi"]) <= tol * max(abs(orc["psi"]), 1e-30) + 1e-18


@pytest.mark.parametrize("field,theta", [("bowl", 60.0), ("corners", 75.0), ("corners", 45.0)])
def test_library_finder_matches_oracle_on_synthetic_fields(field, theta):
    psi = _bowl(41, 31, 0.4123, 0.6311) if field == "bowl" else _with_corner_eddies(101, 81)
    lib = _lib_eddies(psi, theta)
    orc = O.eddy_centres(psi, 1.0, 1.0, theta)
    for a, b in zip(lib, orc):
        _agree(a, b, 1e-12)


def test_library_finder_matches_oracle_on_steady_cavity(golden_dir):
    d = np.load(os.path.join(golden_dir, "steady_65_theta60_n075_re100.npz"))
    lib = _lib_eddies(d["psi"], 60.0)
    orc = O.eddy_centres(d["psi"], 1.0, 1.0, 60.0)
    assert lib[0].found and lib[0].refined
    for a, b in zip(lib, orc):
        _agree(a, b, 1e-10)


def test_library_finder_rejects_bad_input():
    from paper_2306_07603_gb300 import capi
    psi = np.zeros((2, 5))
    with pytest.raises(capi.IfdlbmError):
        capi.ifdlbm_find_eddies(5, 2, (1.0, 1.0, 60.0), psi)
    psi = np.zeros((5, 5))
    psi[2, 2] = np.nan
    with pytest.raises(capi.IfdlbmError):
        capi.ifdlbm_find_eddies(5, 5, (1.0, 1.0, 60.0), psi)
