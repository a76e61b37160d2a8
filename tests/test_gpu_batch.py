"""Batched build (vb_build_batch) against the FP64 oracle, cloud by cloud.

Several point clouds of uneven size go through one call; each cloud's slice
of the output must equal what the oracle computes for that cloud alone:
neighbour lists and the CSR pattern bit-exact (after removing the cloud's row
offset), the same grid points selected by both sweeps, and psi, S and L-hat
within the 1e-5 relative bar of the single-cloud parity tests.  A CUDA-graph
replay of the batched build must reproduce the eager build bit for bit, and
a one-cloud batch must equal vb_build.
"""
import numpy as np
import pytest
import torch

from oracle import method as M
from paper_2104_15124_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5
K, D, C, BETA = 32, 2.0, 1.0, -0.25


@pytest.fixture(scope="module")
def vb():
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import native
    native.compile_library()
    vb.lib()
    return vb


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _close(gpu, ref, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    atol = 1e-25 * np.abs(ref).max()
    err = np.abs(gpu - ref) - (RTOL * np.abs(ref) + atol)
    assert err.max() <= 0, f"{what}: worst relative error {np.max(np.abs(gpu - ref) / (np.abs(ref) + atol)):.3e}"


def _eps_equal(gpu, ref):
    assert abs(gpu - ref) <= 4e-16 * ref, (gpu, ref)


@pytest.fixture(scope="module")
def batch(vb):
    bt = W.ellipsoids(n_clouds=5, n_lo=700, n_hi=3000, seed=7)
    ptr = bt.cloud_ptr
    n = int(ptr[-1])
    builder = vb.Builder(n, 3, K, D, C, BETA, cloud_ptr=ptr)
    out = builder(_t(bt.x))
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    return bt, builder, out


def test_batched_build_matches_oracle_per_cloud(vb, batch):
    bt, builder, out = batch
    ptr = bt.cloud_ptr
    nbr = out.nbr.cpu().numpy()
    rp = out.graph.row_ptr.cpu().numpy()
    col = out.graph.col.cpu().numpy()
    val = out.val.cpu().numpy()
    for b in range(len(ptr) - 1):
        lo, hi = int(ptr[b]), int(ptr[b + 1])
        ref = M.build(bt.x[lo:hi], K, d=D, c=C, beta=BETA)
        assert np.array_equal(nbr[lo:hi] - lo, ref.nbr), f"cloud {b}: neighbour lists"
        e0, e1 = int(rp[lo]), int(rp[hi])
        assert np.array_equal(rp[lo:hi + 1] - e0, ref.pattern.row_ptr), f"cloud {b}: row_ptr"
        assert np.array_equal(col[e0:e1] - lo, ref.pattern.col.astype(np.int32)), f"cloud {b}: columns"
        _eps_equal(out.eps2_den[b].item(), ref.den.eps2)
        _close(out.chi_den[b].cpu().numpy(), ref.den.chi, what=f"cloud {b}: chi density")
        _close(out.psi[lo:hi].cpu().numpy(), ref.psi, what=f"cloud {b}: psi")
        assert out.xi_c[b].item() == ref.xi_c
        _eps_equal(out.eps2_op[b].item(), ref.op_sweep.eps2)
        _close(out.S[lo:hi].cpu().numpy(), ref.op.S, what=f"cloud {b}: S")
        _close(val[e0:e1], ref.op.Lhat, what=f"cloud {b}: L-hat")
    assert out.graph.nnz == int(rp[-1])


def test_graph_replay_is_bitwise_identical(vb, batch):
    bt, builder, out = batch
    x = _t(bt.x)
    builder(x)
    torch.cuda.synchronize()
    eager = {f: getattr(out, f).clone() for f in ("nbr", "val", "eps2_den", "eps2_op", "S")}
    eager_col = out.graph.col.clone()
    for f in ("val", "S"):
        getattr(out, f).zero_()
    g = builder.graph(x)
    for f in ("val", "S"):
        getattr(out, f).zero_()
    g.replay()
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    nnz = out.graph.nnz   # entries past nnz are never written (the caller's buffer keeps what it held)
    for f, v in eager.items():
        got = getattr(out, f)
        assert torch.equal(got[:nnz] if f == "val" else got, v[:nnz] if f == "val" else v), f
    assert torch.equal(out.graph.col[:nnz], eager_col[:nnz])


def test_single_cloud_batch_equals_build(vb):
    w = W.CIRCLE_2K
    x = _t(w.sample())
    one = vb.Builder(w.n, w.m, w.k, w.d, w.c, w.beta, cloud_ptr=[0, w.n])(x)
    ref = vb.build(x, w.k, d=w.d, c=w.c, beta=w.beta)
    torch.cuda.synchronize()
    for f in ("nbr", "nbr_d2", "b", "psi", "P", "S", "val"):
        assert torch.equal(getattr(one, f), getattr(ref, f)), f
    for f in ("eps2_den", "eps2_op", "xi_c"):
        assert torch.equal(getattr(one, f), getattr(ref, f)), f


def test_invalid_cloud_ptr_is_rejected(vb):
    x = _t(np.random.default_rng(1).standard_normal((200, 3)).astype(np.float32))
    with pytest.raises(ValueError):
        vb.Builder(200, 3, 10, 2.0, 1.0, cloud_ptr=[0, 5, 200])   # a cloud smaller than k + 1
    b = vb.Builder(200, 3, 10, 2.0, 1.0, cloud_ptr=[0, 100, 200])
    b._cp_host[1] = 3                                              # the C entry point checks it too
    with pytest.raises(vb.VbError):
        b(x)


def test_batch_with_a_large_cloud_starting_mid_tile(vb):
    # the second cloud starts inside tile 46 and spans 1,094 tiles: its queries run the two-level
    # (super-tile) scan over a tile range that is not aligned to super-tiles
    from oracle import knn as OK
    rng = np.random.default_rng(46)
    x = np.concatenate([rng.standard_normal((3000, 3)), 3.0 + rng.uniform(-1.0, 1.0, (70000, 3))]).astype(np.float32)
    ptr = [0, 3000, 73000]
    out = vb.Builder(73000, 3, K, D, C, BETA, cloud_ptr=ptr)(_t(x))
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    nbr = out.nbr.cpu().numpy()
    for b in range(2):
        lo, hi = ptr[b], ptr[b + 1]
        ref_nbr, _ = OK.knn(x[lo:hi], K)
        assert np.array_equal(nbr[lo:hi] - lo, ref_nbr), f"cloud {b}: neighbour lists"


def test_autotune_picks_a_shape_and_keeps_results(vb, batch):
    bt, builder, out = batch
    x = _t(bt.x)
    builder(x)
    torch.cuda.synchronize()
    before = (out.nbr.clone(), out.val.clone(), out.eps2_op.clone())
    shape = builder.autotune(x)
    assert shape["margin"] in (2, 4, 8, 16, 32) and shape["seed_tiles"] in (1, 2, 3)
    assert shape["knn_ms"] > 0
    again = builder.autotune(x)                      # cached: no timing the second time
    assert again["knn_ms"] == 0 and again["margin"] == shape["margin"]
    builder(x)
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    assert torch.equal(out.nbr, before[0])
    assert torch.equal(out.eps2_op, before[2])
    assert torch.equal(out.val, before[1])
