"""One step of the particle evolution of Sec. 6 (vb_evolve_step) against the FP64
oracle's step (oracle/evolve.py), through the C ABI.

The paper's validation case: standard Gaussian samples in R^2, u = 0, sigma = I and
g = (x - x-bar) . r with r = (1, 0), where f = -x . r solves L_{1,psi} f = g exactly and
the effective velocity -grad f is r.  Bars: the solution f within 1e-2 of the oracle's
(the spectral-solve bar of the eigen-solver tests), grad f within 2e-2, the moved samples
within dt times that error, and the bulk velocity close to r as in the oracle's own pin.
With g = 0 the step is pure diffusion, x + sqrt(dt) sigma W, to FP32 rounding.
"""
import numpy as np
import pytest
import torch

from oracle import evolve as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import native
    native.compile_library()
    vb.lib()
    return vb


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to("cuda")


def test_validation_step_matches_oracle(vb):
    x = np.random.default_rng(5).standard_normal((4000, 2)).astype(np.float32)
    r = np.array([1.0, 0.0])
    g = x.astype(np.float64) @ r
    W = np.random.default_rng(6).standard_normal(x.shape)
    dt = 0.01
    ref = E.evolve_step(x, dt, np.eye(2), W, g, k=128, ell=8, d=2.0)
    st = vb.evolve_step(_t(x), dt, _t(np.eye(2)), _t(W), _t(g), k=128, ell=8, d=2.0)
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    assert st.converged
    f = st.f.cpu().numpy().astype(np.float64)
    grad = st.grad_f.cpu().numpy().astype(np.float64)
    xn = st.x_next.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(f - ref.f) <= 1e-2 * np.linalg.norm(ref.f)
    assert np.linalg.norm(grad - ref.grad_f) <= 2e-2 * np.linalg.norm(ref.grad_f)
    assert np.abs(xn - ref.x_next).max() <= dt * 0.05 * np.abs(ref.grad_f).max() + 1e-6 * np.abs(ref.x_next).max()
    # the paper's check: the effective velocity -grad f is r in the bulk of the samples
    v = -grad
    bulk = np.linalg.norm(x, axis=1) < 1.5
    assert np.allclose(v[bulk].mean(axis=0), r, atol=0.12)


def test_no_source_is_pure_diffusion(vb):
    x = np.random.default_rng(7).standard_normal((800, 2)).astype(np.float32)
    W = np.random.default_rng(8).standard_normal(x.shape)
    sigma = np.array([[0.5, 0.1], [0.0, 0.3]])
    st = vb.evolve_step(_t(x), 0.04, _t(sigma), _t(W), _t(np.zeros(800)), k=24, ell=8, d=2.0)
    torch.cuda.synchronize()
    assert float(st.grad_f.abs().max()) == 0.0
    want = x.astype(np.float64) + 0.2 * (W.astype(np.float32).astype(np.float64) @ sigma.astype(np.float32).astype(np.float64).T)
    np.testing.assert_allclose(st.x_next.cpu().numpy(), want, rtol=2e-7, atol=2e-7)


def test_prescribed_velocity_adds_dt_u(vb):
    # with a prescribed velocity u the drift is u - grad f: two steps on the same samples and
    # draws differ by exactly dt u (to FP32 rounding)
    x = np.random.default_rng(9).standard_normal((1500, 2)).astype(np.float32)
    W = np.random.default_rng(10).standard_normal(x.shape)
    g = x[:, 1].astype(np.float64)
    u = np.tile(np.array([[0.3, -0.2]], dtype=np.float32), (1500, 1))
    a = vb.evolve_step(_t(x), 0.01, _t(np.eye(2)), _t(W), _t(g), k=32, ell=8, d=2.0)
    b = vb.evolve_step(_t(x), 0.01, _t(np.eye(2)), _t(W), _t(g), k=32, ell=8, d=2.0, u=_t(u))
    torch.cuda.synchronize()
    assert torch.equal(a.grad_f, b.grad_f)
    diff = (b.x_next - a.x_next).cpu().numpy()
    np.testing.assert_allclose(diff, 0.01 * u, rtol=0, atol=1e-6)
