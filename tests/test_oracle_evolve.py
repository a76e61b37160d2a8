"""Pins of the oracle's particle evolution (Sec. 6; CPU only).

The paper's own validation case fixes the answer: standard Gaussian samples in R^2,
u = 0, sigma = I, g(x) = (x - x-bar) . r with r = (1, 0).  Then f = -x . r solves
L_{1,psi} f = g exactly (the generator of the Ornstein-Uhlenbeck process, L f = Laplacian f
- x . grad f), so the effective velocity -grad f is r at every sample and one step moves
every sample by dt r on top of its diffusion.  With g = 0 the step is pure diffusion,
x + sqrt(dt) sigma W.
"""
import numpy as np
import pytest

from oracle import evolve as E


def _gauss(n, seed):
    return np.random.default_rng(seed).standard_normal((n, 2)).astype(np.float32)


@pytest.fixture(scope="module")
def validation_step():
    x = _gauss(4000, 5)
    r = np.array([1.0, 0.0])
    g = x.astype(np.float64) @ r
    W = np.random.default_rng(6).standard_normal(x.shape)
    return x, r, W, E.evolve_step(x, 0.01, np.eye(2), W, g, k=128, ell=8, d=2.0)


def test_effective_velocity_is_r(validation_step):
    x, r, W, st = validation_step
    v = -st.grad_f
    bulk = np.linalg.norm(x, axis=1) < 1.5           # away from the thinly sampled tails
    # the kernel discretisation of the unbounded Gaussian leaves a few per cent of bias
    assert np.allclose(v[bulk].mean(axis=0), r, atol=0.12)
    assert np.sqrt(np.mean(np.sum((v[bulk] - r) ** 2, axis=1))) < 0.2
    # the solution itself is -x . r up to its (S-weighted) mean
    f_exact = -(x.astype(np.float64) @ r)
    f_exact -= f_exact.mean()
    assert np.corrcoef(st.f, f_exact)[0, 1] > 0.98


def test_step_translates_by_dt_r_and_diffuses(validation_step):
    x, r, W, st = validation_step
    dt = 0.01
    diffusion = x.astype(np.float64) + np.sqrt(dt) * W
    shift = (st.x_next - diffusion) / dt             # the drift part of the update
    assert np.allclose(shift, -st.grad_f, rtol=0, atol=1e-12)
    assert np.allclose(shift.mean(axis=0), r, atol=0.15)


def test_no_source_is_pure_diffusion():
    x = _gauss(800, 7)
    W = np.random.default_rng(8).standard_normal(x.shape)
    sigma = np.array([[0.5, 0.1], [0.0, 0.3]])
    st = E.evolve_step(x, 0.04, sigma, W, np.zeros(x.shape[0]), k=24, ell=8, d=2.0)
    assert np.allclose(st.grad_f, 0.0, atol=1e-12)
    assert np.allclose(st.x_next, x.astype(np.float64) + 0.2 * (W @ sigma.T), rtol=0, atol=1e-12)


def test_source_is_centred():
    x = _gauss(600, 9)
    g = 3.0 + x[:, 1].astype(np.float64)             # a constant part has no effect (R14)
    a = E.gradient_of_solution(x, g, 24, 8, 2.0)
    b = E.gradient_of_solution(x, g - 3.0, 24, 8, 2.0)
    assert abs(a[2].mean()) < 1e-12
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-9)
