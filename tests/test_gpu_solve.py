"""Parity of vb_solve (eigenpairs of L and the spectral solve of Sec. 3.1) with
the FP64 oracle.

The build runs with the oracle's tuned bandwidths pinned, so both sides
factor the same operator up to the 1e-5 entry tolerance; relative weight
perturbations of size eta move the eigenvalues of this graph-Laplacian form by
at most about eta relative, so the bar for the leading eigenvalues is 1e-4
relative (|lambda_0| <= 1e-4 |lambda_1|).  Eigenvectors are checked through
their S-orthonormality and the solve through the oracle's spectral solution.
"""
import math

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


def _check(vb, x, w, ell, g):
    ref = M.build(x, w.k, d=w.d, c=w.c, beta=w.beta)
    out = vb.build(_t(x), w.k, d=w.d, c=w.c, beta=w.beta, eps2_den=ref.den.eps2, eps2_op=ref.op.eps2)
    e = vb.solve(out.graph, out.val, out.S, ell, rhs=_t(g.astype(np.float32)))
    torch.cuda.synchronize()
    assert e.converged, f"not converged after {e.iters} iterations"
    r = M.leading_eigenpairs(ref.lhat_csr(), ref.op.S, ell)
    lam = e.evals.cpu().numpy()
    assert abs(lam[0]) <= 1e-4 * abs(r.evals[1])
    np.testing.assert_allclose(lam[1:], r.evals[1:], rtol=1e-4)
    n = x.shape[0]
    phi = e.phi.cpu().numpy().astype(np.float64)
    S = out.S.cpu().numpy()
    G = (phi * S ** 2) @ phi.T / n        # <phi_i, phi_j>_S
    assert np.abs(G - np.eye(ell + 1)).max() < 1e-4
    f_ref = M.spectral_solve(r, ref.op.S, g)
    f = e.f.cpu().numpy()
    assert np.linalg.norm(f - f_ref) <= 1e-2 * np.linalg.norm(f_ref)
    return e


def test_circle_16_eigenpairs_and_solve(vb):
    w = W.CIRCLE_2K
    x = w.sample()
    th = np.arctan2(x[:, 1], x[:, 0]).astype(np.float64)
    e = _check(vb, x, w, 16, np.cos(th) + 0.3 * np.sin(3 * th))
    # paired eigenvalues, ratios close to j^2 (the self-loop weight scales all of them alike)
    lam = e.evals.cpu().numpy()[1:]
    assert abs(np.mean(lam[2:4]) / np.mean(lam[0:2]) - 4.0) < 0.15


def test_sphere_32_eigenpairs(vb):
    w = W.Workload("sphere_8k", 8000, 3, 32, 2, 1.0, seed=12)
    x = w.sample()
    z = x[:, 2].astype(np.float64)
    _check(vb, x, w, 32, z + 0.5 * (3 * z * z - 1))
