"""The paper's delta_tol sparsity pattern in plain FP64 (TEST INFRASTRUCTURE ONLY;
see oracle/__init__.py).

Algorithm 1 and Sec. 4 ("Computing the kernel matrix with a k-d tree") keep an entry
(i, j) of a kernel matrix only where its value exceeds a tolerance delta_tol:

    K^(ij) = exp(-||x_i - x_j||^2 / (eps^2 rho_i rho_j))   kept iff  K^(ij) > delta_tol,

with rho = b for the density kernel K_eps and rho = 2 psi^beta for the operator kernel
K_eps,beta.  The k-d tree version first gathers the points inside the radius
R^2 = -eps^2 b_max^2 log(delta_tol) (a superset, for speed) and then applies the same
per-entry test; the pattern is that of the brute-force Algorithm 1.  Because the kept
set depends on eps, a self-tuning sweep over eps_xi^2 = 2^xi has one pattern per grid
point (Eq. (bandwidth sensitivity) summed over that pattern).

Readings of the paper this module takes:
  R11 the test exp(-t) > delta_tol is taken as t < tau with tau = -log(delta_tol)
      computed once in FP64 (exp is strictly decreasing, so the two agree up to the
      rounding of exp; the threshold form is the one two implementations can evaluate
      identically), t = d2 / (eps^2 (rho_i rho_j)): the product rho_i rho_j first, so
      t_ij = t_ji bit for bit and the pattern is symmetric.
  R12 the diagonal is kept (t = 0 < tau for delta_tol < 1), as in R3.
  R13 in the sweep, grid point xi keeps the pairs with t / 2^xi < tau and sums
      exp(-t / 2^xi) over them.

The brute force below evaluates every pair (O(n^2 m)), for the sizes the tests use.
"""
from __future__ import annotations

import math

import numpy as np

from . import knn as _knn
from .method import Pattern


def tau_of(delta_tol: float) -> float:
    """R11: the threshold on t = d2 / (eps^2 rho_i rho_j), -log(delta_tol)."""
    if not (0.0 < delta_tol < 1.0):
        raise ValueError("delta_tol must lie in (0, 1)")
    return -math.log(delta_tol)


def _t_rows(x: np.ndarray, rho: np.ndarray, eps2: float, r0: int, r1: int):
    """t for rows [r0, r1) against every column, and the canonical d2."""
    x64 = np.asarray(x, dtype=np.float32).astype(np.float64)
    acc = None
    for r in range(x64.shape[1]):
        dl = x64[r0:r1, None, r] - x64[None, :, r]   # RN difference of exact FP64 copies
        s = dl * dl
        acc = s if acc is None else acc + s          # ascending coordinate order (canonical)
    rr = rho[r0:r1, None] * rho[None, :]             # rho_i rho_j first (R11)
    return acc / (eps2 * rr), acc


def radius_pattern(x: np.ndarray, rho: np.ndarray, eps2: float, delta_tol: float, block: int = 512) -> Pattern:
    """Algorithm 1: every (i, j), diagonal included (R12), with t_ij < tau (R11).
    Rows sorted by column; d2 holds the canonical squared distances."""
    n = x.shape[0]
    rho = np.asarray(rho, dtype=np.float64)
    tau = tau_of(delta_tol)
    rows, cols, d2s = [], [], []
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        t, d2 = _t_rows(x, rho, eps2, r0, r1)
        ii, jj = np.nonzero(t < tau)
        rows.append(ii.astype(np.int64) + r0)
        cols.append(jj.astype(np.int64))
        d2s.append(d2[ii, jj])
    row = np.concatenate(rows)
    col = np.concatenate(cols)
    d2 = np.concatenate(d2s)
    row_ptr = np.searchsorted(row, np.arange(n + 1, dtype=np.int64)).astype(np.int64)
    return Pattern(n=n, row_ptr=row_ptr, col=col, row=row, d2=d2)


def radius_sweep(x: np.ndarray, rho: np.ndarray, scale: float, xi: np.ndarray, delta_tol: float,
                 block: int = 512) -> np.ndarray:
    """Eq. (bandwidth sensitivity) with the delta_tol pattern of every grid point (R13):
    chi_xi = sum over (i, j) with t_ij / 2^xi < tau of exp(-t_ij / 2^xi),
    t_ij = d2_ij / (scale (rho_i rho_j)); returns chi over the grid."""
    n = x.shape[0]
    rho = np.asarray(rho, dtype=np.float64)
    tau = tau_of(delta_tol)
    chi = np.zeros(len(xi), dtype=np.float64)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        t, _ = _t_rows(x, rho, scale, r0, r1)
        for g, xg in enumerate(xi):
            u = t / 2.0 ** xg
            keep = u < tau
            chi[g] += np.sum(np.exp(-u[keep]))
    return chi


def critical_radius2(eps2: float, rho: np.ndarray, delta_tol: float) -> float:
    """Sec. 4: the search radius R^2 = -eps^2 b_max^2 log(delta_tol), a ball that holds
    every kept pair of every row."""
    return eps2 * float(np.max(rho)) ** 2 * tau_of(delta_tol)


def pattern_pairs(p: Pattern) -> set:
    """The off-diagonal entries of a pattern as a set of (i, j), i < j."""
    m = p.row < p.col
    return set(zip(p.row[m].tolist(), p.col[m].tolist()))


def pair_d2(x: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Canonical FP64 squared distances (the C oracle's), for cross-checks."""
    return _knn.pair_d2(x, a, b)
