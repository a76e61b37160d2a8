"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: neighbour lists, neighbour distances, bandwidths and the CSR pattern
bit-exact; sweep sums chi, density psi, q, D, S and L-hat entries within
1e-5 relative (an absolute floor of 1e-25 of the largest entry covers FP32
underflow of kernel values below 2^-126); the selected grid points, hence the
tuned bandwidths, identical; L-hat bitwise symmetric.
"""
import numpy as np
import pytest
import torch

from oracle import knn as OK
from oracle import method as M
from paper_2104_15124_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def vb():
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import native
    native.compile_library()
    vb.lib()
    return vb


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _close(gpu, ref, rtol=RTOL, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    atol = 1e-25 * np.abs(ref).max()
    err = np.abs(gpu - ref) - (rtol * np.abs(ref) + atol)
    assert err.max() <= 0, f"{what}: worst relative error {np.max(np.abs(gpu - ref) / (np.abs(ref) + atol)):.3e}"


def _eps_equal(gpu, ref):
    # the same grid point selected: 2^xi agrees up to the last bit of the exp2 rounding
    assert abs(gpu - ref) <= 4e-16 * ref, (gpu, ref)


def _knn_case(vb, x, k, prune=True, margin=16):
    nbr, d2 = vb.knn(_t(x), k, margin=margin, prune=prune)
    torch.cuda.synchronize()
    rep = vb.raise_on_device_error()
    ref_nbr, ref_d2 = OK.knn(x, k)
    assert np.array_equal(nbr.cpu().numpy(), ref_nbr)
    assert np.array_equal(d2.cpu().numpy(), ref_d2)
    return rep


@pytest.mark.parametrize("n,m,k", [(150, 3, 10), (200, 2, 199), (1000, 5, 20), (777, 17, 33), (130, 1, 5),
                                   (65, 4, 64), (4099, 3, 48), (3000, 100, 40)])
@pytest.mark.parametrize("prune", [True, False])
def test_knn_exact_random(vb, n, m, k, prune):
    x = np.random.default_rng(n * 7 + m).standard_normal((n, m)).astype(np.float32)
    _knn_case(vb, x, k, prune)


def test_knn_ties_and_duplicates_use_fallback(vb):
    g = np.stack(np.meshgrid(np.arange(30), np.arange(30), indexing="ij"), -1).reshape(-1, 2).astype(np.float32)
    x = np.concatenate([g, g[:40], g[:40]])          # lattice ties plus triplicated points
    _knn_case(vb, x, 12)                      # exact whatever mix of certified and fallback rows
    # without a margin the certificate cannot separate the k-th candidate: rows go to the exact fallback
    vb.report_reset()
    rep = _knn_case(vb, x, 12, margin=0)
    assert rep["knn_fallback_rows"] > 100
    rep = _knn_case(vb, np.random.default_rng(9).standard_normal((5000, 3)).astype(np.float32), 40, margin=0)


def test_knn_circle_2k_and_vmf_50k(vb):
    _knn_case(vb, W.CIRCLE_2K.sample(), 32)
    _knn_case(vb, W.VMF_50K.sample(), 64)


@pytest.mark.parametrize("prune", [True, False])
def test_knn_two_level_scan_70k(vb, prune):
    # 70,000 points are 1,094 tiles, 18 super-tiles of 64 tiles: more than the one-level scan
    # takes, so query tiles bound super-tiles first (pruned) or gather them all (unpruned)
    x = np.random.default_rng(70).uniform(-1.0, 1.0, (70000, 3)).astype(np.float32)
    _knn_case(vb, x, 24, prune)


@pytest.mark.parametrize("m", [2, 3, 4])
def test_knn_hilbert_and_morton_orders(vb, m):
    # the tile order (Hilbert curve by default at 2 <= m <= 4, or Morton) changes which tiles are
    # visited, never the lists; the Hilbert tiles visit fewer candidate pairs on a uniform cloud
    x = np.random.default_rng(40 + m).uniform(-1.0, 1.0, (30000, m)).astype(np.float32)
    ref_nbr, ref_d2 = OK.knn(x, 24)
    pairs = {}
    for curve in ("auto", "morton"):
        for tc in (None, "bf16"):
            vb.report_reset()
            nbr, d2 = vb.knn(_t(x), 24, margin=8, curve=curve, tensor_cores=tc)
            torch.cuda.synchronize()
            rep = vb.raise_on_device_error()
            assert np.array_equal(nbr.cpu().numpy(), ref_nbr), (curve, tc)
            assert np.array_equal(d2.cpu().numpy(), ref_d2), (curve, tc)
            pairs[curve, tc] = rep["knn_candidates"]
    assert pairs["auto", None] < pairs["morton", None], pairs


def test_knn_torus_1m_sampled_rows(vb):
    x = W.TORUS_1M.sample()
    nbr, d2 = vb.knn(_t(x), 64)
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    rows = np.sort(np.random.default_rng(0).choice(x.shape[0], 1500, replace=False))
    nbr_h, d2_h = nbr.cpu().numpy(), d2.cpu().numpy()
    ref_nbr, ref_d2 = OK.knn_rows(x, 64, rows)
    assert np.array_equal(nbr_h[rows], ref_nbr)
    assert np.array_equal(d2_h[rows], ref_d2)
    # every list is sorted by (d2, index) and excludes the point itself
    assert np.all(np.diff(d2_h, axis=1) >= 0)
    assert not np.any(nbr_h == np.arange(x.shape[0])[:, None])


@pytest.fixture(scope="module")
def circle(vb):
    w = W.CIRCLE_2K
    x = w.sample()
    ref = M.build(x, w.k, d=w.d, c=w.c, beta=w.beta)
    out = vb.build(_t(x), w.k, d=w.d, c=w.c, beta=w.beta)
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    return w, x, ref, out


def test_pattern_and_bandwidth_exact(vb, circle):
    w, x, ref, out = circle
    nnz = out.graph.nnz
    p = ref.pattern
    assert nnz == p.nnz
    assert np.array_equal(out.graph.row_ptr.cpu().numpy(), p.row_ptr)
    assert np.array_equal(out.graph.col[:nnz].cpu().numpy(), p.col.astype(np.int32))
    assert np.array_equal(out.graph.ed2[:nnz].cpu().numpy(), p.d2.astype(np.float32))
    assert np.array_equal(out.b.cpu().numpy(), ref.b)


def test_sweeps_density_operator(vb, circle):
    w, x, ref, out = circle
    _close(out.chi_den.cpu().numpy(), ref.den.chi, what="chi density")
    _eps_equal(out.eps2_den.item(), ref.den.eps2)
    assert abs(out.dim_den.item() - ref.den.dim_est) < 1e-4
    _close(out.psi.cpu().numpy(), ref.psi, what="psi")
    _close(out.P.cpu().numpy(), ref.P, what="P")
    assert out.xi_c.item() == ref.xi_c
    _close(out.chi_op.cpu().numpy(), ref.op_sweep.chi, what="chi operator")
    _eps_equal(out.eps2_op.item(), ref.op_sweep.eps2)


def test_lhat_values_and_symmetry(vb, circle):
    w, x, ref, out = circle
    nnz = out.graph.nnz
    val = out.val[:nnz].cpu().numpy()
    _close(val, ref.op.Lhat, what="L-hat")
    for name in ("q", "D", "S"):
        _close(getattr(out, name).cpu().numpy(), getattr(ref.op, name), what=name)
    p = ref.pattern
    # bitwise symmetry: entry (i, j) equals entry (j, i)
    key = p.row * p.n + p.col
    tkey = p.col * p.n + p.row
    pos = np.searchsorted(key, tkey)
    assert np.array_equal(val, val[pos])


def test_vmf_50k_full_build(vb):
    w = W.VMF_50K
    x = w.sample()
    ref = M.build(x, w.k, d=w.d, c=w.c, beta=w.beta)
    out = vb.build(_t(x), w.k, d=w.d, c=w.c, beta=w.beta)
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    assert np.array_equal(out.nbr.cpu().numpy(), ref.nbr)
    nnz = out.graph.nnz
    assert nnz == ref.pattern.nnz
    assert np.array_equal(out.graph.col[:nnz].cpu().numpy(), ref.pattern.col.astype(np.int32))
    _eps_equal(out.eps2_den.item(), ref.den.eps2)
    _eps_equal(out.eps2_op.item(), ref.op_sweep.eps2)
    _close(out.psi.cpu().numpy(), ref.psi, what="psi")
    _close(out.val[:nnz].cpu().numpy(), ref.op.Lhat, what="L-hat")
    _close(out.S.cpu().numpy(), ref.op.S, what="S")


def test_build_equals_stepwise_and_is_deterministic(vb, circle):
    w, x, ref, out = circle
    xt = _t(x)
    nbr, d2 = vb.knn(xt, w.k)
    g = vb.graph(nbr, d2)
    b = vb.bandwidth(d2)
    e_den, chi_den, _ = vb.epsilon_tune(g, b, 1.0)
    psi, P = vb.density(g, b, e_den, w.d, w.beta)
    xc = vb.operator_centre(g, b, P)
    e_op, chi_op, _ = vb.epsilon_tune(g, P, 4.0, xc, warn_bit=2)
    val, q, D, S = vb.kernel_csr(g, psi, P, e_op, w.c, w.beta, w.d)
    again = vb.build(xt, w.k, d=w.d, c=w.c, beta=w.beta)
    torch.cuda.synchronize()
    nnz = out.graph.nnz
    for a, b_ in ((val[:nnz], out.val[:nnz]), (chi_den, out.chi_den), (chi_op, out.chi_op), (psi, out.psi),
                  (S, out.S), (again.val[:nnz], out.val[:nnz]), (again.chi_op, out.chi_op)):
        assert torch.equal(a, b_)


def test_spmv_plain_and_laplacian(vb, circle):
    w, x, ref, out = circle
    n = x.shape[0]
    nnz = out.graph.nnz
    val = out.val[:nnz].cpu().numpy()
    A = ref.lhat_csr()
    rng = np.random.default_rng(1)
    xr = rng.standard_normal(n).astype(np.float32)
    y = vb.spmv(out.graph, out.val, _t(xr)).cpu().numpy()
    y64 = A @ xr.astype(np.float64)
    bound = abs(A) @ np.abs(xr.astype(np.float64))
    assert np.all(np.abs(y - y64) <= 2e-5 * bound + 1e-30)
    # y = alpha A x + beta y
    y0 = rng.standard_normal(n).astype(np.float32)
    y2 = vb.spmv(out.graph, out.val, _t(xr), alpha=0.5, beta=2.0, y=_t(y0)).cpu().numpy()
    assert np.all(np.abs(y2 - (0.5 * y64 + 2.0 * y0)) <= 2e-5 * (0.5 * bound + 2 * np.abs(y0)) + 1e-30)
    # difference form against the oracle: y64 = L-hat_64 x in FP64 from the oracle's L-hat and S.
    # The GPU evaluates sum_j v_ij (x_j - x_i s_j / s_i) with its own v = L-hat (1 + eta) and
    # s = S (1 + sigma), so its error is bounded by |eta| times the oracle's term magnitudes
    # sum_j |L-hat_ij S_j (z_j - z_i)| plus |sigma_j - sigma_i| times sum_j |L-hat_ij| |x_i| S_j / S_i;
    # both relative errors are held to the 1e-5 bar of the entries (2e-5 for the difference of
    # two S errors), plus the FP32 rounding of the row sum.
    Lr, Sr = ref.op.Lhat, ref.op.S
    rows, cols = ref.pattern.row, ref.pattern.col
    off = rows != cols
    ro, co = rows[off], cols[off]
    th = np.arctan2(x[:, 1], x[:, 0]).astype(np.float64)
    vg, Sg = val.astype(np.float64), out.S.cpu().numpy()
    for xs in (Sr.astype(np.float32), (Sr * np.cos(2 * th)).astype(np.float32), xr):
        ys = vb.spmv(out.graph, out.val, _t(xs), S=out.S, laplacian=True).cpu().numpy()
        x64 = xs.astype(np.float64)
        z = x64 / Sr
        terms = Lr[off] * Sr[co] * (z[co] - z[ro])
        ys64 = np.bincount(ro, weights=terms, minlength=n)
        tb = np.bincount(ro, weights=np.abs(terms), minlength=n)
        sb = np.bincount(ro, weights=np.abs(Lr[off]) * np.abs(x64[ro]) * Sr[co] / Sr[ro], minlength=n)
        assert np.all(np.abs(ys - ys64) <= 1e-5 * tb + 2e-5 * sb + 1e-6 * np.abs(ys64) + 1e-30)
        # against the GPU's own L-hat and S the difference form is exact up to FP32 term rounding
        zg = x64 / Sg
        tg = vg[off] * Sg[co] * (zg[co] - zg[ro])
        yg = np.bincount(ro, weights=tg, minlength=n)
        assert np.all(np.abs(ys - yg) <= 1e-5 * np.bincount(ro, weights=np.abs(tg), minlength=n) + 1e-30)


def test_device_errors_are_reported(vb):
    x = np.random.default_rng(3).standard_normal((300, 3)).astype(np.float32)
    with pytest.raises(vb.VbError):
        vb.knn(_t(x), 300)
    bad = x.copy()
    bad[17, 1] = np.nan
    vb.report_reset()
    vb.knn(_t(bad), 8)
    assert vb.report()["error"] == -4
    dup = np.repeat(x[:50], 6, axis=0)          # six copies of every point: b = 0 with k_bw = 5
    vb.report_reset()
    nbr, d2 = vb.knn(_t(dup), 5)
    vb.bandwidth(d2)
    assert vb.report()["error"] == -4
    vb.report_reset()
