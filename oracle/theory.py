"""Closed-form linear theory used to pin the oracle (test infrastructure only).

* Cold plasma oscillation under leapfrog (Sec. 3.1): omega = (2/dt) asin(dt/2).
* Cold two-stream dispersion (Sec. 3.2): two beams of density 1/2 each
  (per-beam plasma frequency squared 1/2) at +-v0; the unstable root of
  1 - wb^2/(w + k v0)^2 - wb^2/(w - k v0)^2 = 0 is purely growing with rate
  sqrt(wb sqrt(wb^2 + 4 k^2 v0^2) - k^2 v0^2 - wb^2), whose maximum over k is
  wb/2 at k v0 = (sqrt(3)/2) wb.
* Warm (Maxwellian) beams and Landau damping: roots of the kinetic dielectric
  1 + sum_b (n_b / (k^2 s_b^2)) (1 + zeta_b Z(zeta_b)), zeta_b = (w - k v_b)/(sqrt(2) k s_b),
  with the plasma dispersion function Z(zeta) = i sqrt(pi) w(zeta) and w the
  Faddeeva function, written here from its textbook definitions: the power
  series w(z) = sum_n (iz)^n / Gamma(n/2 + 1) for small |z|, Laplace's
  continued fraction w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...))))
  for large |z| in the upper half plane, and w(z) = 2 exp(-z^2) - w(-z) below
  the real axis.
"""
from __future__ import annotations

import cmath
import math

_SQRT_PI = math.sqrt(math.pi)


def leapfrog_omega(dt: float, omega0: float = 1.0) -> float:
    """Frequency of x'' = -omega0^2 x integrated by leapfrog with step dt."""
    return (2.0 / dt) * math.asin(omega0 * dt / 2.0)


def faddeeva(z: complex) -> complex:
    """Faddeeva function w(z) = exp(-z^2) erfc(-i z)."""
    z = complex(z)
    if z.imag < 0.0:
        return 2.0 * cmath.exp(-z * z) - faddeeva(-z)
    if abs(z) < 4.0:
        # power series: sum_n (i z)^n / Gamma(n/2 + 1)
        iz = 1j * z
        total = 0j
        term_pow = 1 + 0j
        for n in range(0, 400):
            term = term_pow / math.gamma(n / 2.0 + 1.0)
            total += term
            if n > 10 and abs(term) < 1e-17 * max(1.0, abs(total)):
                break
            term_pow *= iz
        return total
    # Laplace continued fraction, evaluated from the bottom up
    depth = 400
    frac = z
    for n in range(depth, 0, -1):
        frac = z - (n / 2.0) / frac
    return (1j / _SQRT_PI) / frac


def plasma_Z(zeta: complex) -> complex:
    """Plasma dispersion function Z(zeta) = i sqrt(pi) w(zeta)."""
    return 1j * _SQRT_PI * faddeeva(zeta)


def kinetic_dielectric(omega: complex, k: float, beams) -> complex:
    """1 + sum over Maxwellian beams (density n, drift u, thermal spread s)."""
    eps = 1.0 + 0j
    for n, u, s in beams:
        zeta = (omega - k * u) / (math.sqrt(2.0) * k * s)
        eps += (n / (k * k * s * s)) * (1.0 + zeta * plasma_Z(zeta))
    return eps


def _secant(f, x0: complex, x1: complex, tol=1e-14, maxit=200) -> complex:
    f0, f1 = f(x0), f(x1)
    for _ in range(maxit):
        if f1 == f0:
            break
        x2 = x1 - f1 * (x1 - x0) / (f1 - f0)
        x0, f0 = x1, f1
        x1, f1 = x2, f(x2)
        if abs(x1 - x0) < tol * max(1.0, abs(x1)):
            return x1
    return x1


def landau_root(k: float) -> complex:
    """Least-damped root omega of the unit-Maxwellian (omega_p = 1) dielectric."""
    guess = complex(math.sqrt(1.0 + 3.0 * k * k), -0.05)
    f = lambda w: kinetic_dielectric(w, k, [(1.0, 0.0, 1.0)])
    return _secant(f, guess, guess * (1 + 1e-3) + 1e-3j)


def cold_two_stream_rate(k: float, v0: float, wb2: float = 0.5) -> float:
    """Growth rate of the cold symmetric two-stream mode (0 if stable)."""
    wb = math.sqrt(wb2)
    a2 = (k * v0) ** 2
    g2 = wb * math.sqrt(wb2 + 4.0 * a2) - a2 - wb2
    return math.sqrt(g2) if g2 > 0 else 0.0


def warm_two_stream_rate(k: float, v0: float, sigma: float, wb2: float = 0.5) -> float:
    """Growth rate of two Maxwellian beams (density wb2 each, spread sigma)."""
    beams = [(wb2, v0, sigma), (wb2, -v0, sigma)]
    g0 = cold_two_stream_rate(k, v0, wb2)
    if g0 <= 0:
        raise ValueError("cold mode is stable at this k")
    f = lambda w: kinetic_dielectric(w, k, beams)
    root = _secant(f, complex(0.0, g0), complex(0.0, 0.98 * g0))
    return root.imag
