"""Pins of the oracle's formulas (CPU only).

Each check is fixed by the paper or by the mathematics, not by re-running the
oracle's own code:
  * the sparse pipeline equals the dense all-pairs matrix algebra of Sec. 2
    (Algorithm 1 with every pair kept) when k = n - 1;
  * the invariants of the construction (Markov rows, L-hat symmetric,
    L-hat = S L S^-1, constants in the null space, eigenvalues <= 0,
    S-orthonormal eigenvectors);
  * closed forms: densities 1/(2 pi) on the circle, 1/(4 pi) on S^2 and the
    von Mises-Fisher law; spectra -j^2 on the circle, -l(l+1) clusters of
    size 2l + 1 on S^2, -1/sqrt2 and -1/sqrt3 pairs for the 4-D Gaussian;
    the dimension estimate on S^2; the manufactured 4-D solve of Sec. 5.1.2.
The kernel matrix keeps its diagonal (Algorithm 1 starts the inner loop at
j = i), which biases density and spectrum by the self weight; the closed-form
checks remove exactly that term.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import method as M
from paper_2104_15124_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _self_weight(B):
    p = B.pattern
    dg = p.row == p.col
    return float(np.mean(B.op.Kt[dg] / B.op.D))


def _psi_without_self(B):
    # psi_i minus its own diagonal term 1 / w_i, w_i = n (pi eps^2 b_i^2)^(d/2)
    w = B.pattern.n * (math.pi * B.den.eps2 * B.b ** 2) ** (B.d / 2.0)
    return B.psi - 1.0 / w


def test_alpha_matches_paper_example():
    g = GOLD["alpha_example"]
    assert M.alpha_from(g["c"], g["d"], g["beta"]) == g["alpha"]


def test_grid():
    xi = M.xi_grid()
    assert xi.shape == (57,) and xi[0] == -10.0 and xi[-1] == 4.0 and xi[1] - xi[0] == 0.25


def test_bandwidth_on_equally_spaced_line():
    # points at h * j on a line: the middle point's 2s nearest are at h, h, 2h, 2h, ..., s h, s h
    h = 0.125
    x = (h * np.arange(41, dtype=np.float32))[:, None]
    from oracle import knn as K
    _, d2 = K.knn(x, 8)
    b = M.bandwidth(d2, 8)
    assert b[20] == math.sqrt(2 * h * h * (1 + 4 + 9 + 16))
    # an end point sees h, 2h, ..., 8h on one side only
    assert b[0] == math.sqrt(h * h * sum(j * j for j in range(1, 9)))


@pytest.mark.parametrize("d,c", [(2, 1.0), (2, 0.0)])
def test_sparse_equals_dense_all_pairs(d, c):
    x = W.gaussian(120, 2, seed=11)
    n = x.shape[0]
    B = M.build(x, n - 1, d=d, c=c, k_bw=10)
    R = M.dense_all_pairs(x, 10, d=d, c=c)
    p = B.pattern
    assert p.nnz == n * n
    np.testing.assert_allclose(B.b, R["b"], rtol=1e-12)
    np.testing.assert_allclose(B.den.chi, R["chi_den"], rtol=1e-12)
    assert B.den.g_star == R["g_den"] and B.xi_c == R["xi_c"] and B.op_sweep.g_star == R["g_op"]
    np.testing.assert_allclose(B.op_sweep.chi, R["chi_op"], rtol=1e-12)
    np.testing.assert_allclose(B.psi, R["psi"], rtol=1e-12)
    for key in ("q", "D", "S"):
        np.testing.assert_allclose(getattr(B.op, key), R[key], rtol=1e-12)
    dense = lambda v: v.reshape(n, n)
    np.testing.assert_allclose(dense(B.op.Kt), R["Kt"], rtol=1e-12)
    np.testing.assert_allclose(dense(B.op.Lhat), R["Lhat"], rtol=1e-10, atol=1e-9 * np.abs(R["Lhat"]).max())
    np.testing.assert_allclose(dense(B.op.L), R["L"], rtol=1e-10, atol=1e-9 * np.abs(R["L"]).max())


@pytest.fixture(scope="module")
def circle_build():
    return M.build(W.circle(2000, 1), 32, d=1, c=0.0)


def test_invariants(circle_build):
    B = circle_build
    p, op = B.pattern, B.op
    # D^-1 K~ is a Markov matrix (Sec. 2.2)
    np.testing.assert_allclose(M.row_sum(p, op.Kt / op.D[p.row]), 1.0, rtol=0, atol=1e-13)
    L = B.lhat_csr()
    # L-hat symmetric
    assert abs(L - L.T).max() <= 1e-12 * abs(L).max()
    # L-hat = S L S^-1 entrywise
    np.testing.assert_allclose(op.Lhat, op.S[p.row] * op.L / op.S[p.col], rtol=1e-12,
                               atol=1e-12 * np.abs(op.Lhat).max())
    # constants are in the null space: L 1 = 0, L-hat (S 1) = 0
    assert np.abs(M.row_sum(p, op.L)).max() <= 1e-10 * np.abs(op.L).max()
    assert np.abs(L @ op.S).max() <= 1e-10 * np.abs(op.Lhat).max() * op.S.max()
    # ellipticity: with d = 1, c = 0 the parameter relation gives alpha = 0.625
    assert M.alpha_from(0.0, 1, -0.25) == 0.625


def test_circle_spectrum_and_density(circle_build):
    B = circle_build
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, 16)
    lam = e.evals
    assert abs(lam[0]) <= 1e-8 * abs(lam[1])
    assert np.all(lam[1:] < 0)
    # S-orthonormality of phi (Eq. inner product)
    G = e.phi.T @ (B.op.S[:, None] ** 2 * e.phi) / e.phi.shape[0]
    np.testing.assert_allclose(G, np.eye(17), atol=1e-9)
    # Laplace-Beltrami on the unit circle: -j^2, each twice; the diagonal of the
    # Markov kernel scales every eigenvalue by (1 - self weight)
    scaled = lam[1:9] / (1.0 - _self_weight(B))
    expect = -np.repeat(np.arange(1, 5) ** 2, 2).astype(float)
    np.testing.assert_allclose(scaled, expect, rtol=0.03)
    # uniform density 1 / (2 pi) once the self term is removed
    assert abs(np.mean(_psi_without_self(B)) * 2 * math.pi - 1.0) < 0.01
    assert not B.den.at_boundary and not B.op_sweep.at_boundary


@pytest.mark.slow
def test_sphere_density_spectrum_dimension():
    x = W.sphere_uniform(3000, 2)
    B = M.build(x, 48, d=2, c=1.0)
    assert abs(np.mean(_psi_without_self(B)) / GOLD["uniform_sphere_density"]["psi"] - 1.0) < 0.01
    lam = M.leading_eigenpairs(B.lhat_csr(), B.op.S, 8).evals[1:]
    # clusters of size 3 (l = 1) and 5 (l = 2): the largest gap sits after the third eigenvalue
    gaps = np.diff(lam)
    assert int(np.argmin(gaps)) == 2
    ratio = np.mean(lam[3:8]) / np.mean(lam[0:3])   # -6 / -2
    assert abs(ratio - 3.0) < 0.25
    # dimension estimate 2 max chi' on the full pattern (Fig. 3)
    R = M.dense_all_pairs(W.sphere_uniform(1500, 2), 32, d=2, c=1.0)
    chip = np.diff(np.log(R["chi_den"])) / (M.DXI * math.log(2.0))
    assert abs(2 * chip.max() - 2.0) < 0.05


@pytest.mark.slow
def test_vmf_density_closed_form():
    kappa = 2.0
    x = W.sphere_vmf(4000, kappa, 2)
    B = M.build(x, 48, d=2, c=1.0)
    z = x[:, 2].astype(np.float64)
    exact = kappa * np.exp(kappa * z) / (4 * math.pi * math.sinh(kappa))
    est = _psi_without_self(B)
    # log psi = kappa z + log(kappa / (4 pi sinh kappa)): fit slope and intercept in z
    A = np.stack([z, np.ones_like(z)], axis=1)
    slope, icpt = np.linalg.lstsq(A, np.log(est), rcond=None)[0]
    assert abs(slope - kappa) < 0.1
    assert abs(icpt - math.log(kappa / (4 * math.pi * math.sinh(kappa)))) < 0.06
    assert np.corrcoef(np.log(est), np.log(exact))[0, 1] > 0.9


@pytest.mark.slow
def test_gaussian4d_spectrum_and_solve():
    g = GOLD["gaussian4d_eigenvalues"]
    x = W.gaussian(4000, 4, scales=g["variances"], seed=7)
    B = M.build(x, 48, d=4, c=1.0)
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, 6)
    lam = e.evals[1:5]
    # two pairs whose ratio is (1/sqrt2) / (1/sqrt3) = sqrt(3/2)
    assert abs(lam[1] - lam[0]) < 0.05 * abs(lam[0]) and abs(lam[3] - lam[2]) < 0.1 * abs(lam[2])
    assert abs(np.mean(lam[2:4]) / np.mean(lam[0:2]) - math.sqrt(1.5)) < 0.04
    s = GOLD["gaussian4d_solution"]
    gv = x.astype(np.float64) @ np.array(s["g_coeffs"])
    fv = x.astype(np.float64) @ np.array(s["f_coeffs"])
    f = M.spectral_solve(e, B.op.S, gv)
    err = np.sum((f - fv) ** 2) / np.sum(fv ** 2)   # Eq. (normalised error)
    assert err < 0.35
    # an eigenvector right-hand side is inverted exactly: g = phi_j  =>  f = phi_j / lambda_j
    f1 = M.spectral_solve(e, B.op.S, e.phi[:, 2])
    np.testing.assert_allclose(f1, e.phi[:, 2] / e.evals[2], rtol=1e-8, atol=1e-10)


def test_operator_centre_worked_example():
    # Three points on a line at 0, 1, 3 (squared distances 1, 9, 4 for the pairs (0,1), (0,2),
    # (1,2)), b = (1, 2, 4), P = (1, 1, 2), every pair stored in both directions plus the diagonal.
    # By hand: sum_E' d2 / (b_i b_j) = 2 (1/2 + 9/4 + 4/8) = 6.5 and
    # sum_E' d2 / (4 P_i P_j) = 2 (1/4 + 9/8 + 4/8) = 3.75, so 4 log2(3.75 / 6.5) = -3.174...
    # rounds to -3 and xi_c = -0.75.
    x = np.array([[0.0], [1.0], [3.0]], dtype=np.float32)
    p = M.full_pattern(x)
    b = np.array([1.0, 2.0, 4.0])
    P = np.array([1.0, 1.0, 2.0])
    assert M.operator_centre(p, b, P) == -0.75
    # doubling the coordinates quadruples d2 and doubles b: the density argument is unchanged,
    # the operator argument grows 4x, so the centre moves by log2(4) = 2 to 1.25
    assert M.operator_centre(M.full_pattern(2 * x), 2 * b, P) == 1.25
    # rounding to the nearest quarter (not down): a ratio of 2^0.45 gives 4 * 0.45 = 1.8 -> 2 -> 0.5
    P2 = np.full(3, 0.5 * 2.0 ** -0.225)
    b2 = np.full(3, 1.0)
    assert M.operator_centre(p, b2, P2) == 0.5


def test_sphere_drift_reference_spectrum():
    # The continuum reference for the von Mises-Fisher example of Sec. 5.2 with c = 1: at
    # kappa = 0 the Galerkin solver must give the spherical Laplacian's -l(l+1) with
    # multiplicity 2l + 1; at kappa = 2 it must agree with an independent finite-volume
    # discretisation in the polar angle.
    from oracle import spectra as SP
    lam0 = SP.sphere_drift_spectrum(0.0, 1.0, 36)
    expect = -np.concatenate([[l * (l + 1)] * (2 * l + 1) for l in range(6)])
    np.testing.assert_allclose(lam0, expect, atol=1e-9)
    lam = SP.sphere_drift_spectrum(2.0, 1.0, 33)
    fv = SP.sphere_drift_spectrum_fd(2.0, 1.0, 33)
    assert lam[0] == pytest.approx(0.0, abs=1e-9)
    np.testing.assert_allclose(lam[1:], fv[1:], rtol=5e-6)
    # the drift lifts the l = 1 triplet into the m = +-1 pair and the m = 0 level
    assert abs(lam[1] - lam[2]) < 1e-9 and lam[3] < lam[2] - 0.1
    # c = 0 ignores the density (Delta alone); the spectrum depends on c kappa only
    np.testing.assert_allclose(SP.sphere_drift_spectrum(2.0, 0.0, 16), expect[:16], atol=1e-9)
    np.testing.assert_allclose(SP.sphere_drift_spectrum(1.0, 2.0, 16), lam[:16], rtol=1e-12, atol=1e-12)


def test_manufactured_5d_closed_form():
    # The manufactured solve of the 5-dimensional Gaussian workload: f = z_1 exp(-|z|^2 / 4) and,
    # for psi = N(0, I_5) and c = 1 (L = Delta - z . grad), g = L f = z_1 exp(-|z|^2/4)(0.75 |z|^2 - 4.5).
    # Checked against central differences of f at random points, independently of the derivation.
    rng = np.random.default_rng(0)
    z = rng.standard_normal((50, 5))
    f = lambda y: y[..., 0] * np.exp(-(y * y).sum(-1) / 4)
    h = 1e-3
    lap = np.zeros(50)
    grad = np.zeros((50, 5))
    for a in range(5):
        e = np.zeros(5)
        e[a] = h
        lap += (f(z + e) - 2 * f(z) + f(z - e)) / h ** 2
        grad[:, a] = (f(z + e) - f(z - e)) / (2 * h)
    Lf = lap - (z * grad).sum(1)
    r2 = (z * z).sum(1)
    g = z[:, 0] * np.exp(-r2 / 4) * (0.75 * r2 - 4.5)
    np.testing.assert_allclose(Lf, g, atol=1e-5)
    # f has zero mean under psi (odd in z_1), as the solvability condition of Eq. (Kolmogorov problem) needs
    zz = rng.standard_normal((200000, 5))
    assert abs(np.mean(f(zz))) < 5e-3


@pytest.mark.slow
def test_gaussian4d_solve_error_falls_as_n_doubles():
    # Sec. 5.1.2 reports the normalised error of the manufactured solve falling as n grows. With
    # k = 48 and the kernel's self weight divided out of the spectrum (it scales every eigenvalue
    # by 1 - w, so the solve by 1 / (1 - w)), the error falls at each doubling of n.
    g = GOLD["gaussian4d_eigenvalues"]
    s = GOLD["gaussian4d_solution"]
    errs = []
    for n in (2000, 4000, 8000):
        x = W.gaussian(n, 4, scales=g["variances"], seed=7)
        B = M.build(x, 48, d=4, c=1.0)
        e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, 6)
        gv = x.astype(np.float64) @ np.array(s["g_coeffs"])
        fv = x.astype(np.float64) @ np.array(s["f_coeffs"])
        f = M.spectral_solve(e, B.op.S, gv) * (1.0 - _self_weight(B))
        errs.append(np.sum((f - fv) ** 2) / np.sum(fv ** 2))   # Eq. (normalised error)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05
