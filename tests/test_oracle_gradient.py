"""Pins of the oracle's gradient representation (Sec. 3.2), CPU only.

* With every eigenpair of a small operator kept, the truncated sums are complete,
  and the spectral formula must equal the Carre du Champ expression
  (L(uv) - u L v - v L u) / 2 of the same matrix L (Lemma, product rule) for any
  u and v: a dropped 1/2, a wrong sign on an eigenvalue, a wrong weight in the
  inner product or a transposed index in C-hat all break the equality.
* A closed form: on the unit circle the gradients of the coordinates are tangential,
  grad x1 . grad x1 = sin^2 theta, grad x1 . grad x2 = -sin theta cos theta.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import method as M
from paper_2104_15124_gb300 import workloads as W


def _dense_L(B):
    Lh = B.lhat_csr().toarray()
    S = B.op.S
    return Lh * (1.0 / S)[:, None] * S[None, :]     # L = S^-1 L-hat S


def test_full_basis_equals_carre_du_champ():
    x = W.gaussian(160, 2, seed=11)
    B = M.build(x, 40, d=2, c=1.0)
    n = x.shape[0]
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, n - 1)
    L = _dense_L(B)
    rng = np.random.default_rng(3)
    for _ in range(3):
        u, v = rng.standard_normal(n), rng.standard_normal(n)
        got = M.gradient_dot(e, B.op.S, u, v)
        want = M.carre_du_champ(L, u, v)
        assert np.abs(got - want).max() <= 1e-7 * np.abs(want).max()
    # the coordinate choice v = x_s gives du/dx_s (Eq. gradient of u) through the same identity
    u = np.sin(x[:, 0].astype(np.float64)) * x[:, 1]
    for s in range(2):
        vs = x[:, s].astype(np.float64)
        np.testing.assert_allclose(M.gradient_dot(e, B.op.S, u, vs), M.carre_du_champ(L, u, vs),
                                   rtol=0, atol=1e-7 * np.abs(M.carre_du_champ(L, u, vs)).max())


def test_triple_products_expand_products():
    # C-hat_ljk are the S-coefficients of phi_j * phi_k: with the full basis the expansion is exact
    x = W.gaussian(90, 2, seed=12)
    B = M.build(x, 30, d=2, c=1.0)
    n = x.shape[0]
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, n - 1)
    C = M.triple_products(e, B.op.S)
    for j, k in ((0, 0), (1, 2), (5, 7)):
        np.testing.assert_allclose(e.phi @ C[:, j, k], e.phi[:, j] * e.phi[:, k], rtol=0, atol=1e-8)
    assert np.allclose(C, np.swapaxes(C, 1, 2)) and np.allclose(C, np.swapaxes(C, 0, 1))


def test_tangential_gradients_on_the_circle():
    # On the unit circle (Laplace-Beltrami, c = 0) the Riemannian gradient is tangential:
    # grad x1 . grad x1 = sin^2 theta and grad x1 . grad x2 = -sin theta cos theta.  x1, x2 are
    # j = 1 eigenfunctions and their products lie in the j = 0, 2 modes, so eight eigenpairs
    # represent them; the kernel's diagonal scales every eigenvalue, hence the estimate, by
    # (1 - self weight), which is removed as in the spectrum check.
    x = W.circle(2000, 1)
    B = M.build(x, 32, d=1, c=0.0)
    p = B.pattern
    sw = float(np.mean(B.op.Kt[p.row == p.col] / B.op.D))
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, 8)
    th = np.arctan2(x[:, 1], x[:, 0]).astype(np.float64)
    x1, x2 = x[:, 0].astype(np.float64), x[:, 1].astype(np.float64)
    g11 = M.gradient_dot(e, B.op.S, x1, x1) / (1 - sw)
    g12 = M.gradient_dot(e, B.op.S, x1, x2) / (1 - sw)
    assert np.abs(g11 - np.sin(th) ** 2).max() < 0.05
    assert np.abs(g12 + np.sin(th) * np.cos(th)).max() < 0.05
