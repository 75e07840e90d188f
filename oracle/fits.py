"""Rate and frequency fits on diagnostic histories (test infrastructure only).

These read the field-energy or Fourier-mode histories that the oracle (or the
CUDA path) records and turn them into the quantities the paper's tests compare
with linear theory (Sec. 3.1 plasma oscillation, Sec. 3.2 two-stream growth,
Sec. 3.3 Landau damping).  numpy's FFT and least squares are the only library
steps.
"""
from __future__ import annotations

import numpy as np


def mode(E_hist, m: int):
    """Complex Fourier coefficient m of every row of a (steps, nx) field history."""
    E_hist = np.asarray(E_hist, dtype=np.float64)
    return np.fft.rfft(E_hist, axis=1)[:, m] / E_hist.shape[1]


def local_maxima(t, y, t_min=-np.inf, t_max=np.inf):
    """Parabola-refined interior local maxima of y(t) inside [t_min, t_max]."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out_t, out_y = [], []
    for i in range(1, len(y) - 1):
        if y[i] > y[i - 1] and y[i] >= y[i + 1] and t_min <= t[i] <= t_max:
            y0, y1, y2 = y[i - 1], y[i], y[i + 1]
            den = y0 - 2 * y1 + y2
            off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
            h = t[i + 1] - t[i]
            out_t.append(t[i] + off * h)
            out_y.append(y1 - 0.25 * (y0 - y2) * off)
    return np.array(out_t), np.array(out_y)


def exp_rate(t, y):
    """Least-squares slope of log(y) against t."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    A = np.vstack([t, np.ones_like(t)]).T
    slope, _ = np.linalg.lstsq(A, np.log(y), rcond=None)[0]
    return float(slope)


def damping_rate(t, W, t_min, t_max):
    """gamma from the peaks of a field energy W ~ exp(2 gamma t) cos^2(...)."""
    pt, py = local_maxima(t, W, t_min, t_max)
    if len(pt) < 3:
        raise ValueError("fewer than three peaks in the fit window")
    return 0.5 * exp_rate(pt, py)


def growth_rate(t, amp, t_min, t_max):
    """gamma from a mode amplitude |E_m| ~ exp(gamma t) inside [t_min, t_max]."""
    t = np.asarray(t)
    sel = (t >= t_min) & (t <= t_max)
    return exp_rate(t[sel], np.asarray(amp)[sel])


def zero_crossings(t, y):
    """Linearly interpolated times at which y changes sign."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s = np.signbit(y)
    idx = np.nonzero(s[1:] != s[:-1])[0]
    return t[idx] - y[idx] * (t[idx + 1] - t[idx]) / (y[idx + 1] - y[idx])


def oscillation_omega(t, y):
    """Angular frequency of y(t) ~ cos(omega t) from its zero crossings."""
    zc = zero_crossings(t, y)
    if len(zc) < 3:
        raise ValueError("fewer than three zero crossings")
    half_period = np.polyfit(np.arange(len(zc)), zc, 1)[0]
    return float(np.pi / half_period)
