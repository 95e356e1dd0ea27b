"""Ritz-value machinery for the oracle (TEST INFRASTRUCTURE ONLY).

Carson 2019, Section 4:
  eq. (T)     Lanczos tridiagonal T_i built from the CG coefficients alpha, beta
  eq. (lit)   its Cholesky factor L_i^T: zeta_j = 1/sqrt(alpha_j), eta_j = sqrt(beta_j/alpha_j)
  eq. (lest)  lmax = ||L_i||^2, lmin = ||L_i^{-1}||^{-2}
  Alg. 3      incremental estimate of ||L_i||^2 (Meurant-Tichy)
  Alg. 4      incremental estimate of ||L_i^{-1}||^{-2} (Meurant-Tichy)
  ExactRitz   the extremal eigenvalues of T_i themselves (the exact Ritz
              values that Algs. 3-4 estimate), after every CG iteration

Readings.  Alg. 3 prints "xi_{l+1}^2" in a_l; the matching entry of T is
eta_l^2 + zeta_{l+1}^2, so xi is read as zeta (reading C1).  sign(0) = +1; when
chi = 0 the 2x2 problem is already diagonal: omega is kept, h = 1, g = 0
(reading C3).  The argument of a square root that should lie in [0, 1] is
clamped to it.
"""
from __future__ import annotations

import math

import numpy as np


def lanczos_t(alpha, beta) -> np.ndarray:
    """T_i of eq. (T) from alpha_0..alpha_{i-1} and beta_0..beta_{i-2}."""
    i = len(alpha)
    T = np.zeros((i, i))
    for j in range(i):
        T[j, j] = 1.0 / alpha[j] + (beta[j - 1] / alpha[j - 1] if j >= 1 else 0.0)
        if j + 1 < i:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(beta[j]) / alpha[j]
    return T


def cholesky_lt(alpha, beta):
    """(zeta, eta) of eq. (lit): the diagonal and superdiagonal of L_i^T."""
    zeta = [1.0 / math.sqrt(a) for a in alpha]
    eta = [math.sqrt(beta[j] / alpha[j]) for j in range(len(alpha) - 1)]
    return zeta, eta


def _clamp01(v: float) -> float:
    return 0.0 if v < 0.0 else (1.0 if v > 1.0 else v)


def _sign(v: float) -> float:
    return -1.0 if v < 0.0 else 1.0


class NormL:
    """Algorithm 3: running estimate omega of ||L_i||^2 (= lmax of eq. lest)."""

    def __init__(self, zeta0: float):
        self.omega = zeta0 * zeta0
        self.h = 1.0

    def step(self, zeta_l: float, eta_l: float, zeta_l1: float) -> float:
        d = zeta_l * zeta_l * eta_l * eta_l * self.h
        a = eta_l * eta_l + zeta_l1 * zeta_l1
        chi = math.sqrt((self.omega - a) ** 2 + 4.0 * d)
        if chi == 0.0:
            self.h = 1.0
            return self.omega
        self.h = _clamp01(0.5 * (1.0 - (self.omega - a) / chi))
        self.omega = self.omega + chi * self.h
        return self.omega


class NormLinv:
    """Algorithm 4: running estimate omega of ||L_i^{-1}||^2; lmin = 1/omega."""

    def __init__(self, zeta0: float):
        self.omega = 1.0 / (zeta0 * zeta0)
        self.a = self.omega
        self.d = 0.0
        self.g = 0.0
        self.h = 1.0

    def step(self, zeta_l: float, eta_l: float, zeta_l1: float) -> float:
        d1 = -(eta_l / zeta_l1) * (self.g * self.d + self.h * self.a)
        a1 = (eta_l * eta_l * self.a + 1.0) / (zeta_l1 * zeta_l1)
        chi = math.sqrt((self.omega - a1) ** 2 + 4.0 * d1 * d1)
        if chi == 0.0:
            h, g = 1.0, 0.0
        else:
            h2 = _clamp01(0.5 * (1.0 - (self.omega - a1) / chi))
            self.omega = self.omega + chi * h2
            h = math.sqrt(h2)
            g = math.sqrt(_clamp01(1.0 - h2))
        self.h = abs(h) * _sign(d1)
        self.g = g
        self.d = d1
        self.a = a1
        return 1.0 / self.omega


def mt_estimates(alpha, beta):
    """(lmin, lmax) after running Algs. 3 and 4 from scratch on alpha, beta.

    Uses zeta_0..zeta_{i-1} and eta_0..eta_{i-2}, i = len(alpha).
    """
    zeta, eta = cholesky_lt(alpha, beta[: len(alpha) - 1])
    up, lo = NormL(zeta[0]), NormLinv(zeta[0])
    lmax, lmin = up.omega, 1.0 / lo.omega
    for l in range(len(alpha) - 1):
        lmax = up.step(zeta[l], eta[l], zeta[l + 1])
        lmin = lo.step(zeta[l], eta[l], zeta[l + 1])
    return lmin, lmax


class RitzTracker:
    """Incremental Algs. 3-4 fed one CG iteration at a time (Alg. 5, Section 4).

    ``push(alpha_i, beta_{i-1})`` after the i-th alpha is known.  After the
    first push both estimates equal 1/alpha_0; each later push runs one loop
    step of each algorithm with zeta_{i-1}, eta_{i-1}, zeta_i.
    """

    def __init__(self):
        self.n = 0
        self.lmin = None
        self.lmax = None
        self._zeta_prev = None
        self._alpha_prev = None

    def push(self, alpha: float, beta_prev: float | None):
        zeta = 1.0 / math.sqrt(alpha)
        if self.n == 0:
            self._up, self._lo = NormL(zeta), NormLinv(zeta)
            self.lmax, self.lmin = self._up.omega, 1.0 / self._lo.omega
        else:
            eta = math.sqrt(beta_prev / self._alpha_prev)
            self.lmax = self._up.step(self._zeta_prev, eta, zeta)
            self.lmin = self._lo.step(self._zeta_prev, eta, zeta)
        self._zeta_prev = zeta
        self._alpha_prev = alpha
        self.n += 1
        return self.lmin, self.lmax


class ExactRitz:
    """The extremal eigenvalues of T_i (eq. T) after every CG iteration, in
    place of the estimates of Algs. 3-4: the same ``push(alpha_i, beta_{i-1})``
    interface, T grown by one row per push (diagonal 1/alpha_i +
    beta_{i-1}/alpha_{i-1}, off-diagonal sqrt(beta_{i-1})/alpha_{i-1}), and its
    smallest and largest eigenvalues from LAPACK's tridiagonal bisection
    (scipy.linalg.eigvalsh_tridiagonal)."""

    def __init__(self):
        self.n = 0
        self.lmin = None
        self.lmax = None
        self.d: list[float] = []
        self.e: list[float] = []
        self._alpha_prev = None

    def push(self, alpha: float, beta_prev: float | None):
        from scipy.linalg import eigvalsh_tridiagonal
        if self.n == 0:
            self.d.append(1.0 / alpha)
        else:
            self.d.append(1.0 / alpha + beta_prev / self._alpha_prev)
            self.e.append(math.sqrt(beta_prev) / self._alpha_prev)
        self._alpha_prev = alpha
        self.n += 1
        if self.n == 1:
            self.lmin = self.lmax = self.d[0]
        else:
            d, e = np.array(self.d), np.array(self.e)
            self.lmin = float(eigvalsh_tridiagonal(d, e, select="i", select_range=(0, 0))[0])
            self.lmax = float(eigvalsh_tridiagonal(d, e, select="i", select_range=(self.n - 1, self.n - 1))[0])
        return self.lmin, self.lmax
