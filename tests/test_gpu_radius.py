"""The paper's delta_tol pattern on the GPU (vb_radius_pattern, vb_radius_sweep; Algorithm 1
and Sec. 4) against the oracle's brute force (oracle/radius.py).

Bars: row offsets, columns and canonical squared distances bit-exact (the test t < tau is
taken in FP64 on both sides with the same operation order); the per-grid-point sweep sums
within 1e-5 relative and the same grid point selected.  Cases: constant and variable
bandwidths, two tolerances, ragged sizes (not a multiple of the 64-point tile), m = 1..5,
and the bandwidth b of the kNN method as rho.
"""
import numpy as np
import pytest
import torch

from oracle import knn as OK
from oracle import method as M
from oracle import radius as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import native
    native.compile_library()
    vb.lib()
    return vb


def _t(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else a.astype(dtype))
    return torch.from_numpy(a).to("cuda")


def _compare(vb, x, rho, eps2, delta):
    ref = R.radius_pattern(x, rho, eps2, delta)
    got = vb.radius_pattern(_t(x, np.float32), _t(rho, np.float64), eps2, delta)
    assert got.nnz == ref.nnz
    assert np.array_equal(got.row_ptr.cpu().numpy(), ref.row_ptr)
    assert np.array_equal(got.col.cpu().numpy(), ref.col.astype(np.int32))
    assert np.array_equal(got.d2.cpu().numpy(), ref.d2)
    return ref


@pytest.mark.parametrize("n,m,const,delta", [(1500, 3, True, 1e-2), (3001, 2, False, 1e-2), (1000, 5, False, 1e-3),
                                             (777, 1, False, 1e-2), (2048, 4, False, 0.5)])
def test_pattern_bit_exact(vb, n, m, const, delta):
    rng = np.random.default_rng(n + m)
    x = rng.uniform(-1.0, 1.0, (n, m)).astype(np.float32)
    rho = np.ones(n) if const else rng.uniform(0.5, 2.0, n)
    eps2 = 0.02 * (1500 / n) ** (2.0 / m)
    ref = _compare(vb, x, rho, eps2, delta)
    assert ref.nnz >= n   # the diagonal at least


def test_pattern_with_the_method_bandwidth(vb):
    # rho = b, the bandwidth of Sec. 2.1 from the exact kNN, at the density sweep's eps
    from paper_2104_15124_gb300 import workloads as W
    x = W.sphere_vmf(4000, 2.0, 3)
    nbr, d2 = OK.knn(x, 32)
    b = M.bandwidth(d2, 32)
    _compare(vb, x, b, 2.0 ** -6, 1e-2)


def test_sweep_per_grid_point(vb):
    x = np.random.default_rng(4).uniform(-1.0, 1.0, (1500, 2)).astype(np.float32)
    rho = np.random.default_rng(5).uniform(0.5, 2.0, 1500) * 0.05
    xi = M.xi_grid()
    ref = R.radius_sweep(x, rho, 1.0, xi, 1e-2)
    chi, eps2, dim = vb.radius_sweep(_t(x), _t(rho), 1.0, 1e-2)
    chi = chi.cpu().numpy()
    np.testing.assert_allclose(chi, ref, rtol=1e-5)
    chip = np.diff(np.log(ref)) / (M.DXI * np.log(2.0))
    g = int(np.argmax(chip))
    assert eps2.item() == 2.0 ** xi[g]
    assert abs(dim.item() - 2 * chip[g]) < 1e-9


def test_capacity_too_small_is_reported(vb):
    x = np.random.default_rng(6).uniform(-1.0, 1.0, (500, 2)).astype(np.float32)
    rho = np.ones(500)
    n = x.shape[0]
    L = vb.lib()
    import ctypes
    xt, rt = _t(x), _t(rho)
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    d2 = torch.empty(n, dtype=torch.float64, device="cuda")
    nnz = torch.empty(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(L.vb_radius_workspace(n, 2), dtype=torch.uint8, device="cuda")
    vb.report_reset()
    rc = L.vb_radius_pattern(ctypes.c_void_p(vb._ctx(xt.device)), ctypes.c_void_p(xt.data_ptr()), n, 2,
                             ctypes.c_void_p(rt.data_ptr()), 0.05, 1e-2, ctypes.c_void_p(rp.data_ptr()),
                             ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(d2.data_ptr()), n,
                             ctypes.c_void_p(nnz.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel())
    assert rc == 0
    assert vb.report()["error"] == -3
    assert int(nnz.item()) > n
    vb.report_reset()
