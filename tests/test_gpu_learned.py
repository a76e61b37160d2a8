"""The learned radius (step a7) and the radius-first kNN search it feeds.

* The network's gradient (our forward/backward kernels, BF16 weights, FP32
  arithmetic) matches the FP64 oracle's chain rule at the same weights.
* Training with our Adam kernel fits log r_k of a torus sample.
* The radius-first search is exact whatever the radius: learned, exact,
  too small (every tile retried by the exact search) or too large (the
  heaps' own running threshold takes over).
"""
import math

import numpy as np
import pytest
import torch

from oracle import knn as OK
from oracle import mlp as OM
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


def test_mlp_gradient_matches_fp64_oracle(vb):
    x = W.torus4(4096, 0.01, 31)
    y = np.random.default_rng(2).standard_normal(4096).astype(np.float32) * 0.3 - 2.0
    net = vb.Mlp(4, seed=7)
    mean, scale = x.mean(0), x.std(0)
    net.set_standardisation(mean, scale, -2.0, 0.3)
    g, loss = net.gradient(_t(x), _t(y))
    theta = net.bf16_weights().cpu().numpy().astype(np.float64)
    Xs = (x.astype(np.float64) - mean.astype(np.float32)) / scale.astype(np.float32)
    Ys = (y.astype(np.float64) + 2.0) / 0.3
    ref_loss, ref_g = OM.loss_and_grad(theta, Xs, Ys)
    assert abs(loss.item() - ref_loss) <= 1e-4 * ref_loss
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - ref_g) <= 2e-3 * np.linalg.norm(ref_g)
    # predictions: our BF16 forward against the FP64 forward at the same weights
    pred = net.predict(_t(x)).cpu().numpy()
    np.testing.assert_allclose(pred, -2.0 + 0.3 * OM.forward(theta, Xs), rtol=0, atol=1e-4)


def test_tensor_core_inference_matches_fp32_forward(vb):
    # the tcgen05 forward of the radius-first search (BF16 activations) against the FP32 forward
    # and the FP64 oracle at the same BF16 weights: the hidden activations' BF16 rounding (2^-9
    # relative) bounds the difference; ragged n (not a multiple of the 128-row step)
    x = W.sphere_vmf(3001, 2.0, 41)
    net = vb.Mlp(3, seed=11)
    mean, scale = x.mean(0), x.std(0)
    net.set_standardisation(mean, scale, -3.0, 0.5)
    p32 = net.predict(_t(x)).cpu().numpy().astype(np.float64)
    ptc = net.predict(_t(x), tensor_cores=True).cpu().numpy().astype(np.float64)
    theta = net.bf16_weights().cpu().numpy().astype(np.float64)
    Xs = (x.astype(np.float64) - mean.astype(np.float32)) / scale.astype(np.float32)
    ref = -3.0 + 0.5 * OM.forward(theta, Xs)
    spread = np.abs(ref - ref.mean()).max() + 1e-3
    assert np.abs(ptc - ref).max() <= 2e-2 * spread + 2e-3
    assert np.abs(ptc - p32).max() <= 2e-2 * spread + 2e-3
    assert np.all(np.isfinite(ptc))


def test_training_fits_log_radius(vb):
    # von Mises-Fisher on S^2 (kappa = 2): the density, hence r_k, varies about 7-fold from pole to pole
    x = W.sphere_vmf(20000, 2.0, 103)
    k = 64
    nbr, d2 = vb.knn(_t(x), k)
    logr = 0.5 * torch.log(d2[:, k - 1]).float()
    net = vb.train_radius_model(_t(x), logr, epochs=25, batch=2048, lr=3e-3, seed=103)
    pred = net.predict(_t(x))
    resid = (pred - logr).float()
    # the fit explains most of the spread of log r_k around its mean
    assert resid.pow(2).mean().item() < 0.6 * (logr - logr.mean()).pow(2).mean().item() + 1e-4


@pytest.mark.parametrize("mode", ["exact", "small", "large"])
def test_radius_search_exact_for_any_radius(vb, mode):
    w = W.VMF_50K
    x = w.sample(20000)
    k = 32
    ref_nbr, ref_d2 = OK.knn(x, k)
    rk = np.sqrt(ref_d2[:, k - 1]).astype(np.float32)
    if mode == "exact":
        radius, infl = rk, 1.0001
    elif mode == "small":
        radius, infl = np.full_like(rk, 0.3 * float(np.median(rk))), 1.0
    else:
        radius, infl = np.full_like(rk, 3.0 * float(rk.max())), 1.0
    vb.report_reset()
    nbr, d2 = vb.knn(_t(x), k, radius=_t(radius), inflate=infl)
    torch.cuda.synchronize()
    rep = vb.raise_on_device_error()
    assert np.array_equal(nbr.cpu().numpy(), ref_nbr)
    assert np.array_equal(d2.cpu().numpy(), ref_d2)
    ntiles = (x.shape[0] + 63) // 64
    if mode == "small":
        # nobody finds k points inside: every tile is searched again at twice the radius, and the
        # tiles still short after that are redone exactly
        assert rep["knn_redo_tiles"] == ntiles
        assert rep["knn_retry_tiles"] <= ntiles
    else:
        assert rep["knn_retry_tiles"] == 0        # a loose radius only loosens the initial pruning
        assert rep["knn_redo_tiles"] == 0


@pytest.mark.parametrize("scale", [0.5, 1.0, 1.5])
def test_radius_search_exact_in_a_cloud_smaller_than_the_heap(vb, scale):
    # 20 points, k + margin = 24 slots: every candidate would fit in the heap, but the radius
    # still excludes those beyond it, so a row is settled by its certificate against the radius
    # (or redone by the exact search), never by counting the cloud
    x = np.random.default_rng(11).standard_normal((20, 3)).astype(np.float32)
    k = 8
    ref_nbr, ref_d2 = OK.knn(x, k)
    radius = (scale * np.sqrt(ref_d2[:, k - 1])).astype(np.float32)
    nbr, d2 = vb.knn(_t(x), k, radius=_t(radius), inflate=1.0)
    torch.cuda.synchronize()
    vb.raise_on_device_error()
    assert np.array_equal(nbr.cpu().numpy(), ref_nbr)
    assert np.array_equal(d2.cpu().numpy(), ref_d2)


def test_learned_radius_search_exact_and_prunes(vb):
    k = 64
    xt_train = _t(W.torus4(100000, 0.01, 103))
    nbr, d2 = vb.knn(xt_train, k)
    net = vb.train_radius_model(xt_train, 0.5 * torch.log(d2[:, k - 1]).float(), epochs=20, batch=4096, seed=103)
    n = 200000
    x = W.torus4(n, 0.01, 3)
    shift = math.log(100000 / n) / 2.0        # r_k scales like n^(-1/d), d = 2
    vb.report_reset()
    nbr_l, d2_l = vb.knn(_t(x), k, mlp=net, log_shift=shift, inflate=1.5)
    torch.cuda.synchronize()
    rep_l = vb.raise_on_device_error()
    vb.report_reset()
    nbr_p, d2_p = vb.knn(_t(x), k)
    torch.cuda.synchronize()
    rep_p = vb.raise_on_device_error()
    assert torch.equal(nbr_l, nbr_p) and torch.equal(d2_l, d2_p)
    rows = np.sort(np.random.default_rng(5).choice(n, 800, replace=False))
    ref_nbr, ref_d2 = OK.knn_rows(x, k, rows)
    assert np.array_equal(nbr_l.cpu().numpy()[rows], ref_nbr)
    # the learned radius settles most tiles and evaluates fewer candidates than the exact heap search
    assert rep_l["knn_retry_tiles"] < 0.05 * ((n + 63) // 64)
    assert rep_l["knn_candidates"] < rep_p["knn_candidates"]


def test_standardisation_is_computed_on_the_device(vb):
    x = W.torus4(5000, 0.01, 44)
    y = (np.random.default_rng(3).standard_normal(5000) * 0.2 - 3.0).astype(np.float32)
    net = vb.Mlp(4, seed=5)
    net.fit_standardisation(_t(x), _t(y))
    x64 = x.astype(np.float64)
    np.testing.assert_allclose(list(net.c.in_mean)[:4], x64.mean(0), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(list(net.c.in_scale)[:4], x64.std(0, ddof=1), rtol=1e-6)
    assert abs(net.c.out_mean - y.astype(np.float64).mean()) < 1e-6
    assert abs(net.c.out_scale - y.astype(np.float64).std(ddof=1)) < 1e-6


@pytest.mark.parametrize("name", ["vmf_s2_50k", "torus_r4_1m"])
def test_learned_radius_against_a_constant_radius(vb, name, record_property):
    # The ablation of the learned part: the same radius-first search with one global radius for
    # every point (the training targets' mean inflated by 3 standard deviations) and with the
    # network's radius (inflated by 3 standard deviations of its residual).  Both are exact, like
    # the plain search.  What the network gains is its prediction: on the von Mises-Fisher sphere
    # r_k varies with the density and the network explains most of that spread; on the uniform
    # torus there is nothing to learn and it predicts a constant.  The candidate pairs each search
    # evaluates are recorded.
    w = W.WORKLOADS[name]
    x = _t(w.sample())
    n_train = 100000
    kp = max(1, int(round(w.k * n_train / w.n)))
    xtr = _t(W.Workload(w.name, n_train, w.m, w.k, w.d, w.c, w.beta, w.margin, 103).sample())
    _, d2tr = vb.knn(xtr, kp)
    target = 0.5 * torch.log(d2tr[:, kp - 1]).float()
    net = vb.train_radius_model(xtr, target, epochs=20, batch=4096, seed=103)
    resid = (target - net.predict(xtr)).float()
    tstd, rstd = float(target.std()), float(resid.std())
    counts = {}
    vb.report_reset()
    ref_nbr, ref_d2 = vb.knn(x, w.k)
    counts["plain"] = vb.report()["knn_candidates"]
    const = torch.full((w.n,), math.exp(float(target.mean()) + 3 * tstd), dtype=torch.float32, device="cuda")
    vb.report_reset()
    nbr_c, d2_c = vb.knn(x, w.k, radius=const, inflate=1.0)
    counts["constant"] = vb.report()["knn_candidates"]
    vb.report_reset()
    nbr_m, d2_m = vb.knn(x, w.k, mlp=net, log_shift=float(resid.mean()), inflate=math.exp(3 * rstd))
    counts["learned"] = vb.report()["knn_candidates"]
    for a, b in ((nbr_c, ref_nbr), (nbr_m, ref_nbr), (d2_c, ref_d2), (d2_m, ref_d2)):
        assert torch.equal(a, b)
    record_property("candidate_pairs", counts)
    record_property("target_std", tstd)
    record_property("residual_std", rstd)
    if name.startswith("vmf"):
        assert rstd < 0.6 * tstd          # the density variation is learned
    else:
        assert rstd <= 1.02 * tstd        # nothing to learn on the uniform torus
