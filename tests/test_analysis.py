"""Host-side spectrum analysis helpers against closed forms."""
import numpy as np

from paper_2101_06187_gb300 import analysis


def test_compensated_spectrum_is_flat_on_the_power_law():
    k = np.arange(0, 40, dtype=float)
    E = np.zeros_like(k)
    E[1:] = 3.0 * k[1:] ** (-5.0 / 3.0)
    np.testing.assert_allclose(analysis.compensated(E), 3.0, rtol=1e-14)


def test_fit_slope_recovers_exponent():
    k = np.arange(0, 30, dtype=float)
    E = np.zeros_like(k)
    E[1:] = 0.7 * k[1:] ** -2.0
    slope, intercept = analysis.fit_slope(E, 2, 12)
    assert abs(slope + 2.0) < 1e-12 and abs(intercept - np.log(0.7)) < 1e-12


def test_decorrelated_mean_uses_the_stride():
    rng = np.random.default_rng(0)
    s = rng.normal(size=(1000, 3))
    m, se = analysis.decorrelated_mean(s, 10)
    np.testing.assert_allclose(m, s[::10].mean(axis=0))
    np.testing.assert_allclose(se, s[::10].std(axis=0, ddof=1) / np.sqrt(100))
