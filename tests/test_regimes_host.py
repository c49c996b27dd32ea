"""Host-side statistics of the unsteady-flow time series (regimes.py): the
regime rule on series whose spectra are known in closed form. No GPU."""
import numpy as np

from paper_2306_07603_gb300.regimes import classify, spectrum

DT = 0.05
T = np.arange(20000) * DT


def test_constant_series_is_steady():
    assert classify(1.0 + 1e-9 * np.sin(T), DT)["regime"] == "steady"


def test_harmonic_series_is_periodic_with_its_fundamental():
    f0 = 0.37
    E = 1.0 + 0.01 * np.sin(2 * np.pi * f0 * T) + 0.004 * np.sin(2 * np.pi * 2 * f0 * T + 0.3)
    c = classify(E, DT)
    df = 1.0 / (len(T) * DT)
    assert c["regime"] == "periodic" and abs(c["f0"] - f0) <= df
    assert abs(c["period"] - 1 / f0) <= 2 * df / f0 ** 2


def test_two_incommensurate_frequencies_are_quasi_periodic():
    E = 1.0 + 0.01 * np.sin(2 * np.pi * 0.37 * T) + 0.006 * np.sin(2 * np.pi * 0.37 * np.sqrt(2) * T)
    assert classify(E, DT)["regime"] == "quasi-periodic"


def test_broadband_series_is_turbulent():
    """A stationary AR(1) fluctuation (correlation time 20 samples): a
    Lorentzian, broadband spectrum."""
    rng = np.random.default_rng(1)
    x = np.zeros(len(T))
    a = np.exp(-1.0 / 20.0)
    for k in range(1, len(T)):
        x[k] = a * x[k - 1] + rng.standard_normal()
    c = classify(1.0 + 1e-3 * x, DT)
    assert c["regime"] == "turbulent" and c["concentration"] < 0.8


def test_trend_is_removed_and_slow_settling_is_drifting():
    f0 = 0.37
    E = 1.0 + 0.001 * T + 0.01 * np.sin(2 * np.pi * f0 * T)
    c = classify(E, DT)
    assert c["regime"] == "periodic" and abs(c["f0"] - f0) <= 1.0 / (len(T) * DT)
    E = 1.0 + 0.05 * np.exp(-T / 400.0)          # still settling over the record
    c = classify(E, DT)
    assert c["regime"] == "drifting" and c["drift"] < 0


def test_spectrum_peak_at_the_signal_frequency():
    f, p = spectrum(np.sin(2 * np.pi * 1.25 * T), DT)
    assert abs(f[np.argmax(p)] - 1.25) <= 1.0 / (len(T) * DT)
