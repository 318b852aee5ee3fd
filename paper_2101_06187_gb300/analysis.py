"""Host-side analysis of the spectra the library returns (Sec. 4, Sec. 5,
App. C): these act on small arrays of shell energies, not on the lattice.

* compensated(E, slope): k^{-slope} E(k) for k >= 1 -- the paper's "spectrum
  divided by the expected slope" (Kolmogorov's -5/3, Sec. 4), flat where the
  power law holds.
* fit_slope(E, kmin, kmax): least-squares slope of log E against log k over
  the shells kmin <= k <= kmax (the inertial range below the driven band).
* decorrelated_mean(samples, stride): time mean and standard error of E(k)
  samples taken every step, keeping every stride-th sample so that the
  samples are decorrelated (App. C chooses the stride from the agreement of
  the averages across strides).
"""
from __future__ import annotations

import numpy as np

KOLMOGOROV = -5.0 / 3.0


def compensated(E, slope: float = KOLMOGOROV) -> np.ndarray:
    """k^{-slope} E(k) for k = 1 .. len(E)-1 (shell 0 is dropped)."""
    E = np.asarray(E, dtype=np.float64)
    k = np.arange(1, len(E), dtype=np.float64)
    return E[1:] * k ** (-slope)


def fit_slope(E, kmin: int, kmax: int):
    """(slope, intercept) of log E(k) = slope * log k + intercept over kmin..kmax."""
    E = np.asarray(E, dtype=np.float64)
    k = np.arange(kmin, kmax + 1, dtype=np.float64)
    e = E[kmin:kmax + 1]
    if np.any(e <= 0) or len(k) < 2:
        raise ValueError("need at least two shells with positive energy")
    slope, intercept = np.polyfit(np.log(k), np.log(e), 1)
    return float(slope), float(intercept)


def decorrelated_mean(samples, stride: int):
    """(mean, standard error) over every stride-th row of samples (n, nshells)."""
    s = np.asarray(samples, dtype=np.float64)[::max(1, int(stride))]
    if len(s) < 2:
        raise ValueError("need at least two decorrelated samples")
    return s.mean(axis=0), s.std(axis=0, ddof=1) / np.sqrt(len(s))
