"""The tensor-core tile primitive (tcgen05.mma, BF16 operands, FP32 accumulation in
tensor memory) against an FP64 product of the same BF16-rounded operands."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _bf16(a):
    return torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("K,N", [(16, 128), (48, 64), (112, 128), (128, 32)])
def test_tc_dot_tile_matches_fp64(K, N):
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import native
    native.compile_library()
    rng = np.random.default_rng(K + N)
    a = rng.standard_normal((128, K)).astype(np.float32)
    b = rng.standard_normal((N, K)).astype(np.float32)
    d = vb.tc_dot_tile(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    vb.raise_on_device_error()
    ref = _bf16(a) @ _bf16(b).T
    # products of BF16 values are exact in FP32; only the FP32 sums round
    bound = 4 * K * 2.0 ** -24 * (np.abs(_bf16(a)) @ np.abs(_bf16(b)).T)
    assert np.all(np.abs(d - ref) <= bound + 1e-30)


def _knn_ref(x, k):
    from oracle import knn as OK
    return OK.knn(x, k)


@pytest.mark.parametrize("variant", ["staged", "pipelined"])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("with_radius", [False, True])
@pytest.mark.parametrize("name,n,k,m", [("vmf", 20000, 32, 3), ("torus", 9000, 64, 4), ("gauss100", 3000, 32, 100)])
def test_tensor_core_knn_is_exact(name, n, k, m, prec, with_radius, variant):
    """The search with 16-bit tensor-core distance tiles returns the exact FP64 neighbour
    lists (FP64 rescoring, certificate with the tiles' error bound), with and without a
    radius guess, and settles most query tiles without the FP32 search; both kernels
    (staged, and the pipelined one fed by bulk copies)."""
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import workloads as W
    x = {"vmf": lambda: W.sphere_vmf(n, 2.0, 21), "torus": lambda: W.torus4(n, 0.01, 22),
         "gauss100": lambda: W.gauss_embedded(n, 5, 100, 1e-3, 23).x}[name]()
    ref_nbr, ref_d2 = _knn_ref(x, k)
    xt = torch.from_numpy(x).cuda()
    kw = {}
    if with_radius:
        kw = dict(radius=torch.from_numpy(np.sqrt(ref_d2[:, k - 1]).astype(np.float32)).cuda(), inflate=1.3)
    vb.report_reset()
    nbr, d2 = vb.knn(xt, k, tensor_cores=prec, tc_variant=variant, **kw)
    torch.cuda.synchronize()
    rep = vb.raise_on_device_error()
    assert np.array_equal(nbr.cpu().numpy(), ref_nbr)
    assert np.array_equal(d2.cpu().numpy(), ref_d2)
    tiles = (n + 63) // 64
    # the pipelined kernel centres its operands on the cloud, so BF16's band is too wide for most
    # rows there (still exact: they are redone by the FP32 search); only FP16 must settle its tiles
    limit = {("fp16", "staged"): 0.05, ("fp16", "pipelined"): 0.05, ("bf16", "staged"): 0.5,
             ("bf16", "pipelined"): 1.0}[(prec, variant)]
    assert rep["knn_retry_tiles"] <= limit * tiles, (rep["knn_retry_tiles"], tiles)


def test_tensor_core_knn_ragged_and_small():
    """Sizes that leave a half-empty query tile, a lone tile and k close to n."""
    import paper_2104_15124_gb300 as vb
    from oracle import knn as OK
    rng = np.random.default_rng(5)
    for n, m, k in ((65, 3, 40), (130, 4, 16), (1000, 20, 48), (300, 7, 64)):
        x = rng.standard_normal((n, m)).astype(np.float32)
        ref_nbr, ref_d2 = OK.knn(x, k)
        for prec in ("fp16", "bf16"):
            for variant in ("staged", "pipelined"):
                nbr, d2 = vb.knn(torch.from_numpy(x).cuda(), k, tensor_cores=prec, tc_variant=variant)
                torch.cuda.synchronize()
                vb.raise_on_device_error()
                assert np.array_equal(nbr.cpu().numpy(), ref_nbr), (n, m, k, prec, variant)
                assert np.array_equal(d2.cpu().numpy(), ref_d2), (n, m, k, prec, variant)


@pytest.mark.parametrize("prec,u,dabs", [("bf16", 2.0 ** -8, 0.0), ("fp16", 2.0 ** -11, 1e-6)])
@pytest.mark.parametrize("name,m", [("vmf", 3), ("torus", 4)])
def test_split_operand_tile_distances(name, m, prec, u, dabs):
    """At m <= 4 the staged kernel writes every operand coordinate as hi + lo, two 16-bit
    numbers, and the four products fill the K = 16 of one MMA step: the tile distances it
    keeps (diagnostic output, full heap keys) lie within the error bound E_D(d) of the FP64
    distances with the unit roundoff u^2 (+ 2^-23 for the FP32 centring), taking |q - c| at
    most the diagonal of the cloud's box.  Unsplit 16-bit operands (unit roundoff u) give
    errors of several per cent of the k-th distance on these clouds; split ones stay far
    below 1e-3 of it."""
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import workloads as W
    n, k = 9000, 64
    x = W.sphere_vmf(n, 2.0, 31) if name == "vmf" else W.torus4(n, 0.01, 32)
    xt = torch.from_numpy(x).cuda()
    nbr, nd2, idx, d16 = vb.knn(xt, k, tensor_cores=prec, tc_variant="staged", debug=True, heap_keys="full")
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    ref_nbr, ref_d2 = _knn_ref(x, k)
    assert np.array_equal(nbr.cpu().numpy(), ref_nbr)
    idx, d16 = idx.cpu().numpy(), d16.cpu().numpy().astype(np.float64)
    rows, cols = np.nonzero(idx >= 0)
    x64 = x.astype(np.float64)
    d = ((x64[rows] - x64[idx[rows, cols]]) ** 2).sum(1)
    dt = d16[rows, cols]
    D = ref_d2[rows, k - 1]
    diag = float(np.linalg.norm(x64.max(0) - x64.min(0)))
    us = u * u + 2.0 ** -23
    Z = 1.01 * (2.0 * diag + np.sqrt(D))
    delta = 1.01 * us * Z + dabs
    E = 1.01 * (2.0 * np.sqrt(d) * delta + delta ** 2 + 2 * (16 + 4) * 2.0 ** -24 * Z ** 2)
    assert np.all(np.abs(dt - d) <= E)
    assert np.max(np.abs(dt - d) / D) < 1e-3


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_short_radius_tiles_are_searched_again_in_the_launch(prec):
    """Radius-first 16-bit search with a radius far below the k-th neighbour distance: every
    128-point query tile has a row short of k points, is searched again at twice the radius by
    the same CTA, and whatever is still short goes to the FP32 search; the lists stay exact."""
    import paper_2104_15124_gb300 as vb
    from paper_2104_15124_gb300 import workloads as W
    n, k = 12000, 32
    x = W.torus4(n, 0.01, 41)
    ref_nbr, ref_d2 = _knn_ref(x, k)
    rk = np.sqrt(ref_d2[:, k - 1]).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    qtiles, tiles = (n + 127) // 128, (n + 63) // 64
    # inside 0.85 r_k no row holds k points, so every query tile is searched again: at 1.7 r_k
    # every row is settled; at 0.6 r_k none is, and every tile goes on to the FP32 search
    for scale, retried in ((0.85, 0), (0.3, tiles)):
        vb.report_reset()
        nbr, d2 = vb.knn(xt, k, margin=8, radius=torch.from_numpy(scale * rk).cuda(), inflate=1.0,
                         tensor_cores=prec, tc_variant="staged")
        torch.cuda.synchronize()
        rep = vb.raise_on_device_error()
        assert np.array_equal(nbr.cpu().numpy(), ref_nbr), scale
        assert np.array_equal(d2.cpu().numpy(), ref_d2), scale
        assert rep["knn_redo_tiles"] == qtiles, (scale, rep["knn_redo_tiles"])
        # (the FP32 pass over handed-back tiles counts the few it hands on in turn)
        assert rep["knn_retry_tiles"] >= retried and (retried or rep["knn_retry_tiles"] == 0), \
            (scale, rep["knn_retry_tiles"])
