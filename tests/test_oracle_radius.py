"""Pins of the oracle's delta_tol pattern (Algorithm 1, Sec. 4; CPU only).

Each check comes from outside the oracle's own formula:
  * with a constant bandwidth the pattern is a fixed-radius neighbour graph, which
    scipy's k-d tree finds independently (query_pairs);
  * with a variable bandwidth it is what the paper's k-d tree variant keeps: the pairs
    inside the critical radius R^2 = -eps^2 b_max^2 log(delta_tol), filtered by the
    literal test exp(-d^2 / (eps^2 rho_i rho_j)) > delta_tol;
  * it lies between the constant-bandwidth graphs at the smallest and largest bandwidth;
  * on a 1-D lattice the row lengths have a closed form;
  * the limits delta_tol -> 1 (the diagonal) and delta_tol -> 0 (every pair), where the
    per-grid-point sweep equals the dense all-pairs sweep of Sec. 2.3.
"""
import math

import numpy as np
import pytest

from oracle import method as M
from oracle import radius as R

cKDTree = pytest.importorskip("scipy.spatial").cKDTree


def _cloud(n, m, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (n, m)).astype(np.float32)


def test_constant_bandwidth_is_a_fixed_radius_graph():
    x = _cloud(1500, 3, 1)
    eps2, delta = 0.01, 1e-2
    p = R.radius_pattern(x, np.ones(x.shape[0]), eps2, delta)
    r = math.sqrt(eps2 * -math.log(delta))
    ref = cKDTree(x.astype(np.float64)).query_pairs(r)
    assert R.pattern_pairs(p) == ref
    assert np.all(p.row_ptr[1:] - p.row_ptr[:-1] >= 1)                   # the diagonal
    assert np.sum(p.row == p.col) == x.shape[0]


def test_variable_bandwidth_matches_the_kd_tree_variant():
    x = _cloud(1200, 2, 2)
    rho = np.random.default_rng(3).uniform(0.5, 2.0, x.shape[0])
    eps2, delta = 0.004, 1e-3
    p = R.radius_pattern(x, rho, eps2, delta)
    # Sec. 4: the ball of the critical radius, then the per-entry test in its literal form
    R2 = R.critical_radius2(eps2, rho, delta)
    cand = np.array(sorted(cKDTree(x.astype(np.float64)).query_pairs(math.sqrt(R2) * 1.000001)))
    i, j = cand[:, 0], cand[:, 1]
    d2 = R.pair_d2(x, i, j)
    kval = np.exp(-d2 / (eps2 * rho[i] * rho[j]))
    keep = kval > delta
    near = np.abs(kval - delta) <= 1e-12 * delta                          # rounding of exp at the edge
    got = R.pattern_pairs(p)
    want = set(zip(i[keep & ~near].tolist(), j[keep & ~near].tolist()))
    drop = set(zip(i[~keep & ~near].tolist(), j[~keep & ~near].tolist()))
    assert want <= got and not (drop & got)
    assert len(got - want) <= int(near.sum())
    assert p.d2.max() <= R2                                               # inside the critical radius


def test_bounded_by_the_extreme_bandwidths():
    x = _cloud(1000, 3, 4)
    rho = np.random.default_rng(5).uniform(0.7, 1.6, x.shape[0])
    eps2, delta = 0.02, 1e-2
    got = R.pattern_pairs(R.radius_pattern(x, rho, eps2, delta))
    tree = cKDTree(x.astype(np.float64))
    tau = -math.log(delta)
    inner = tree.query_pairs(math.sqrt(eps2 * tau) * rho.min() * (1 - 1e-9))
    outer = tree.query_pairs(math.sqrt(eps2 * tau) * rho.max() * (1 + 1e-9))
    assert inner <= got <= outer
    assert len(inner) < len(got) < len(outer)


@pytest.mark.parametrize("K", [1, 3, 7])
def test_lattice_row_lengths(K):
    N, h = 60, 0.5
    x = (h * np.arange(N, dtype=np.float32))[:, None]
    delta = math.exp(-((K + 0.5) * h) ** 2)          # eps = rho = 1: keep |i - j| h < (K + 1/2) h
    p = R.radius_pattern(x, np.ones(N), 1.0, delta)
    i = np.arange(N)
    want = np.minimum(i, K) + np.minimum(N - 1 - i, K) + 1
    assert np.array_equal(p.row_ptr[1:] - p.row_ptr[:-1], want)


def test_symmetric_sorted_and_limits():
    x = _cloud(400, 4, 6)
    rho = np.random.default_rng(7).uniform(0.5, 2.0, x.shape[0])
    p = R.radius_pattern(x, rho, 0.05, 0.05)
    pairs = set(zip(p.row.tolist(), p.col.tolist()))
    assert all((j, i) in pairs for i, j in pairs)
    for i in range(p.n):
        c = p.col[p.row_ptr[i]:p.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    # delta_tol -> 1: the diagonal only; delta_tol -> 0: every pair
    d = R.radius_pattern(x, rho, 0.05, 1.0 - 1e-15)
    assert d.nnz == x.shape[0] and np.all(d.row == d.col)
    f = R.radius_pattern(x, rho, 0.05, 1e-300)
    assert f.nnz == x.shape[0] ** 2


def test_sweep_limits_and_monotone_in_delta():
    x = _cloud(300, 2, 8)
    rho = np.random.default_rng(9).uniform(0.8, 1.25, x.shape[0])
    xi = M.xi_grid()
    # nothing dropped at any grid point: the dense all-pairs sweep of Sec. 2.3
    full = R.radius_sweep(x, rho, 1.0, xi, 1e-300)
    ref = M.sweep(M.full_pattern(x), rho, 1.0, xi).chi
    assert np.allclose(full, ref, rtol=1e-12, atol=0)
    # a larger tolerance drops entries, each below the tolerance: the sum falls by less than
    # (number of pairs) x delta_tol and never rises
    for delta in (1e-6, 1e-3, 1e-1):
        chi = R.radius_sweep(x, rho, 1.0, xi, delta)
        assert np.all(chi <= full) and np.all(full - chi <= x.shape[0] ** 2 * delta)
    # constant bandwidth: at every grid point the kept off-diagonal entries are the k-d tree's
    # pairs within sqrt(2^xi (-log delta_tol)); their kernel values plus the n diagonal ones
    for delta in (0.5, 1e-2):
        chi = R.radius_sweep(x, np.ones(x.shape[0]), 1.0, xi, delta)
        tree = cKDTree(x.astype(np.float64))
        for g in (0, 8, 16, 24, 40):
            pr = np.array(sorted(tree.query_pairs(math.sqrt(2.0 ** xi[g] * -math.log(delta)))), dtype=np.int64)
            want = float(x.shape[0])
            if len(pr):
                want += 2.0 * np.sum(np.exp(-R.pair_d2(x, pr[:, 0], pr[:, 1]) / 2.0 ** xi[g]))
            assert abs(chi[g] - want) <= 1e-12 * want, (delta, g)
