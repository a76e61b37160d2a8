"""vb_spmv_laplacian_noalloc: the difference-form SpMV for callers that cannot
allocate device memory (for example a solver loop being recorded into a CUDA
graph, where cudaMalloc is not allowed).  Its scratch is a static device array
inside libvb, so it takes no workspace.  Called through the C ABI, it must give
the same result as vb_spmv in Laplacian mode, call after call, and agree with
L-hat x evaluated in FP64 from the oracle's L-hat and S."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_spmv_matches_workspace_spmv_twice():
    import paper_2104_15124_gb300 as vb
    from oracle import method as M
    from paper_2104_15124_gb300 import native
    from paper_2104_15124_gb300 import workloads as W
    native.compile_library()
    L = vb.lib()
    x = W.circle(3000, 5)
    out = vb.build(torch.from_numpy(x).cuda(), 24, d=1, c=0.0)
    ref_op = M.build(x, 24, d=1, c=0.0)
    rows, cols = ref_op.pattern.row, ref_op.pattern.col
    off = rows != cols
    ro, co = rows[off], cols[off]
    Lr, Sr = ref_op.op.Lhat[off], ref_op.op.S
    g = out.graph
    gc = g.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(0)
    for _ in range(2):
        v = torch.from_numpy(rng.standard_normal(g.n).astype(np.float32)).cuda()
        y0 = torch.from_numpy(rng.standard_normal(g.n).astype(np.float32)).cuda()
        ref = vb.spmv(g, out.val, v, S=out.S, laplacian=True, alpha=0.7, beta=0.3, y=y0.clone())
        y = y0.clone()
        rc = L.vb_spmv_laplacian_noalloc(stream, ctypes.byref(gc), ctypes.c_void_p(out.val.data_ptr()),
                                         ctypes.c_void_p(out.S.data_ptr()), 0.7, ctypes.c_void_p(v.data_ptr()),
                                         0.3, ctypes.c_void_p(y.data_ptr()))
        assert rc == 0
        torch.cuda.synchronize()
        err = (y - ref).abs().max().item()
        assert err <= 1e-5 * ref.abs().max().item()
        # FP64 L-hat x from the oracle, with the error terms of its entries (1e-5) and of S
        # (2e-5 on a difference of two S errors), as in the parity test of vb_spmv
        v64 = v.cpu().numpy().astype(np.float64)
        z = v64 / Sr
        terms = Lr * Sr[co] * (z[co] - z[ro])
        y64 = 0.7 * np.bincount(ro, weights=terms, minlength=g.n) + 0.3 * y0.cpu().numpy().astype(np.float64)
        tb = np.bincount(ro, weights=np.abs(terms), minlength=g.n)
        sb = np.bincount(ro, weights=np.abs(Lr) * np.abs(v64[ro]) * Sr[co] / Sr[ro], minlength=g.n)
        bound = 0.7 * (1e-5 * tb + 2e-5 * sb) + 1e-6 * np.abs(y64) + 1e-30
        assert np.all(np.abs(y.cpu().numpy() - y64) <= bound)
    # a graph beyond the static scratch is refused before anything is launched
    big = vb.GraphC(vb.VB_NOALLOC_MAX_N + 1, gc.row_ptr, gc.col, gc.ed2)
    rc = L.vb_spmv_laplacian_noalloc(stream, ctypes.byref(big), ctypes.c_void_p(out.val.data_ptr()),
                                     ctypes.c_void_p(out.S.data_ptr()), 1.0, ctypes.c_void_p(v.data_ptr()), 0.0,
                                     ctypes.c_void_p(y.data_ptr()))
    assert rc == -9
