"""s-step basis construction for the oracle (TEST INFRASTRUCTURE ONLY).

Paper references (Carson 2019, Section 2):
  eq. (cg-krylovbasis)  P = [rho_0(A)p .. rho_s(A)p],  R = [rho_0(A)r .. rho_{s-1}(A)r]
  eq. (rho)             rho_0 = 1, rho_1 = (z - theta_0) rho_0 / gamma_0,
                        rho_l = ((z - theta_{l-1}) rho_{l-1} - mu_{l-2} rho_{l-2}) / gamma_{l-1}
  eq. (AVVB), (B)       A Ybar = Y B,  B = diag(B_{s+1}, B_s)
  eq. (newtbasis)       Newton basis with Leja-ordered shifts
  eq. (chebbasis)       "simplified" Chebyshev basis

Column order.  The paper writes Y = [P, R].  Here Y is stored interleaved,
Y = [P_0, R_0, P_1, R_1, ..., P_{s-1}, R_{s-1}, P_s], so that the basis
Y_l = {P_0..P_l, R_0..R_{l-1}} of the first l inner steps (eq. reqsub) is the
leading 2l+1 columns and its Gram matrix the leading principal submatrix
(reading C9).  B is permuted to the same order.
"""
from __future__ import annotations

import math

import numpy as np

MONOMIAL, NEWTON, CHEBYSHEV = 0, 1, 2
BASIS_NAMES = {"monomial": MONOMIAL, "newton": NEWTON, "chebyshev": CHEBYSHEV}


def p_index(l: int) -> int:
    """Interleaved column of P_l."""
    return 2 * l


def r_index(l: int) -> int:
    """Interleaved column of R_l."""
    return 2 * l + 1


# ----------------------------------------------------------------------------
# Leja points (eq. newtbasis), on the reference interval [-1, 1]
# ----------------------------------------------------------------------------

def _leja_dlog(t: float, pts) -> float:
    """d/dt of sum_m log|t - t_m|: strictly decreasing between two neighbours.

    Summed left to right in plain binary64 (Python's built-in sum() of floats
    is compensated since 3.12; plain order keeps the bisection's decisions a
    function of the IEEE operations alone)."""
    acc = 0.0
    for tm in pts:
        acc = acc + 1.0 / (t - tm)
    return acc


def _leja_logprod(t: float, pts) -> float:
    acc = 0.0
    for tm in pts:
        acc = acc + math.log(abs(t - tm))
    return acc


def leja_points(s: int) -> np.ndarray:
    """First s Leja points of [-1, 1] with t_0 = 1, t_1 = -1 (eq. newtbasis).

    t_l maximises prod_{m<l} |t - t_m| over [-1, 1].  Between two neighbouring
    points the log of the product is concave, so its maximiser there is the
    unique zero of its derivative; that zero is found by bisection until the
    bracket stops shrinking (reading C7).  The gap whose maximiser gives the
    largest product wins; products within 1e-13 (in log) count as a tie, and a
    tie goes to the smaller t (reading C7).
    """
    pts = [1.0, -1.0][:s]
    while len(pts) < s:
        srt = sorted(pts)
        best_t, best_v = None, -math.inf
        for a, b in zip(srt[:-1], srt[1:]):
            lo, hi = a, b
            while True:
                mid = 0.5 * (lo + hi)
                if mid <= lo or mid >= hi:
                    break
                dv = _leja_dlog(mid, pts)
                if dv == 0.0:
                    lo = hi = mid
                    break
                if dv > 0.0:
                    lo = mid
                else:
                    hi = mid
            t = 0.5 * (lo + hi)
            v = _leja_logprod(t, pts)
            if v > best_v + 1e-13:
                best_t, best_v = t, v
            elif abs(v - best_v) <= 1e-13 and t < best_t:
                best_t, best_v = t, max(v, best_v)
        pts.append(best_t)
    return np.array(pts, dtype=np.float64)


# ----------------------------------------------------------------------------
# basis parameters theta, gamma, mu
# ----------------------------------------------------------------------------

def basis_params(kind: int, s: int, lmin: float | None, lmax: float | None,
                 newton_scale: str = "capacity", cheb_params: str = "standard"):
    """Recurrence coefficients (theta[0..s-1], gamma[0..s-1], mu[0..s-1]) of eq. (rho).

    mu[l] multiplies rho_l in the recurrence for rho_{l+2}; mu[s-1] is unused.
    Monomial (Section 2): theta = 0, gamma = 1, mu = 0; also used while no
    Ritz estimates exist.
    Newton (eq. newtbasis): theta = Leja points of [lmin, lmax] starting with
    lmax, lmin; mu = 0; gamma = 1 as printed (``newton_scale='paper_unit'``) or
    the interval's logarithmic capacity (lmax - lmin)/4 (``'capacity'``,
    reading C6).
    Chebyshev: ``cheb_params='standard'`` gives rho_l(z) = T_l((z - c)/h) with
    c = (lmax + lmin)/2, h = (lmax - lmin)/2: theta = c, gamma_0 = h,
    gamma_l = h/2 (l >= 1), mu = h/2 (reading C5); ``'paper_printed'`` takes
    eq. (chebbasis) literally: theta = c, mu = 2 (lmax - lmin),
    gamma_0 = lmax - lmin, gamma_l = (lmax - lmin)/2.
    """
    theta = np.zeros(s)
    gamma = np.ones(s)
    mu = np.zeros(s)
    if kind == MONOMIAL or lmin is None:
        return theta, gamma, mu
    c = 0.5 * (lmax + lmin)
    h = 0.5 * (lmax - lmin)
    if kind == NEWTON:
        theta = c + h * leja_points(s)
        if newton_scale == "capacity":
            gamma = np.full(s, (lmax - lmin) / 4.0)
        elif newton_scale != "paper_unit":
            raise ValueError(newton_scale)
        return theta, gamma, mu
    if kind == CHEBYSHEV:
        theta = np.full(s, c)
        if cheb_params == "standard":
            gamma = np.full(s, 0.5 * h)
            gamma[0] = h
            mu = np.full(s, 0.5 * h)
        elif cheb_params == "paper_printed":
            gamma = np.full(s, 0.5 * (lmax - lmin))
            gamma[0] = lmax - lmin
            mu = np.full(s, 2.0 * (lmax - lmin))
        else:
            raise ValueError(cheb_params)
        return theta, gamma, mu
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# the basis matrix Y and the change-of-basis matrix B
# ----------------------------------------------------------------------------

def krylov_basis(A, p: np.ndarray, r: np.ndarray, s: int, theta, gamma, mu,
                 store32: bool = False) -> np.ndarray:
    """Y (N x (2s+1), interleaved) by the three-term recurrence eq. (rho).

    P_{l+1} = ((A - theta_l I) P_l - mu_{l-1} P_{l-1}) / gamma_l (no mu term for l = 0),
    the same for R, which stops at R_{s-1} (eq. cg-krylovbasis).
    store32: every column is rounded to binary32 when it is stored, and the
    recurrence continues from the stored (rounded) columns in binary64
    arithmetic (the FP32-stored-basis variant).
    """
    N = p.shape[0]
    Y = np.zeros((N, 2 * s + 1))

    def put(c, v):
        Y[:, c] = v.astype(np.float32).astype(np.float64) if store32 else v

    put(p_index(0), p)
    put(r_index(0), r)
    for l in range(s):
        for chain_len, index in ((s, p_index), (s - 1, r_index)):
            if l + 1 > chain_len:
                continue
            v = Y[:, index(l)]
            w = A @ v - theta[l] * v
            if l >= 1:
                w = w - mu[l - 1] * Y[:, index(l - 1)]
            put(index(l + 1), w / gamma[l])
    return Y


def b_matrix(s: int, theta, gamma, mu) -> np.ndarray:
    """B with A Ybar = Y B (eq. AVVB, eq. B), in the interleaved column order.

    In the paper's order B = diag(B_{s+1}, B_s); B_i has theta_0..theta_{i-2}
    on the diagonal, gamma_0..gamma_{i-2} below it, mu_0..mu_{i-3} above it,
    and a zero last column (Ybar has the last P and last R columns zeroed).
    """
    n = 2 * s + 1
    B = np.zeros((n, n))
    for chain_len, index in ((s + 1, p_index), (s, r_index)):
        for l in range(chain_len - 1):
            B[index(l), index(l)] = theta[l]
            B[index(l + 1), index(l)] = gamma[l]
            if l >= 1:
                B[index(l - 1), index(l)] = mu[l - 1]
    return B


def y_bar(Y: np.ndarray, s: int) -> np.ndarray:
    """Y with its last P column (P_s) and last R column (R_{s-1}) set to zero."""
    Yb = Y.copy()
    Yb[:, p_index(s)] = 0.0
    Yb[:, r_index(s - 1)] = 0.0
    return Yb
