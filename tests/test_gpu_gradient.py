"""Parity of vb_gradient (gradient representation of Sec. 3.2) with the FP64 oracle.

The oracle forms the triple products C-hat_ljk and sums the truncated series
literally; the GPU path reaches the same finite sums by projections and expansions
(O(ell n) per coordinate).  Both sides take the same eigenpairs (those vb_solve
wrote, upcast to FP64 for the oracle), so the comparison isolates the gradient
arithmetic: FP32 products with FP64 sums across 1024-sample chunks, compared
element by element within 2e-4 of the largest derivative (a few FP32 rounding
steps amplified by at most max|lambda| / |lambda_1| in the lambda-weighted terms).
The circle case also checks the closed form: tangential gradients of the
coordinates, grad x1 . grad x1 = sin^2 theta and grad x1 . grad x2 = -sin theta
cos theta, both scaled by (1 - self weight) = -lambda_1.
"""
import numpy as np
import pytest
import torch

from oracle import method as M
from paper_2104_15124_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import native
    native.compile_library()
    vb.lib()
    return vb


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _run(vb, x, k, d, c, ell, u):
    out = vb.build(_t(x), k, d=d, c=c)
    e = vb.solve(out.graph, out.val, out.S, ell)
    grad = vb.gradient(e.evals, e.phi, out.S, _t(u.astype(np.float32)), _t(x))
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    ev = M.Eigen(evals=e.evals.cpu().numpy(), phi_hat=None, phi=e.phi.cpu().numpy().astype(np.float64).T)
    S = out.S.cpu().numpy()
    u64 = u.astype(np.float32).astype(np.float64)
    ref = np.stack([M.gradient_dot(ev, S, u64, x[:, s].astype(np.float64)) for s in range(x.shape[1])], axis=1)
    return grad.cpu().numpy().astype(np.float64), ref, ev


def _assert_close(got, ref):
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 2e-4 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_gradient_on_the_circle(vb):
    x = W.circle(2000, 1)
    th = np.arctan2(x[:, 1], x[:, 0]).astype(np.float64)
    got, ref, ev = _run(vb, x, 32, 1, 0.0, 8, x[:, 0])
    _assert_close(got, ref)
    # closed form: the kernel's diagonal scales the spectrum (lambda_1 = -(1 - self weight) for
    # the j = 1 modes, -1 on the unit circle) and the gradient estimate alike
    scale = -ev.evals[1]
    assert np.abs(got[:, 0] / scale - np.sin(th) ** 2).max() < 0.05
    assert np.abs(got[:, 1] / scale + np.sin(th) * np.cos(th)).max() < 0.05


@pytest.mark.parametrize("ell", [16, 31])
def test_gradient_on_the_sphere(vb, ell):
    x = W.sphere_vmf(6000, 2.0, 5)
    u = np.sin(2.0 * x[:, 0]) + x[:, 1] * x[:, 2]
    got, ref, _ = _run(vb, x, 32, 2, 1.0, ell, u)
    _assert_close(got, ref)


def test_gradient_wide_input(vb):
    # m = 100 coordinates: every batch of the per-sample expansions and a ragged last tile
    g = W.gauss_embedded(2500, 5, 100, 1e-3, 8)
    x = g.x
    u = np.tanh(g.z[:, 0]) * g.z[:, 1]
    got, ref, _ = _run(vb, x, 32, 5, 1.0, 20, u)
    _assert_close(got, ref)
