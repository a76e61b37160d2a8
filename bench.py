#!/usr/bin/env python
"""Benchmark of the variable-bandwidth kernel build (kNN + VB kernel -> L-hat CSR).

One step = one complete build (exact kNN, symmetric pattern, bandwidth,
density sweep, density, operator sweep, normalisations, L-hat CSR) of a
synthetic workload whose coordinates are already resident in HBM, replayed
from a CUDA graph recorded once per form.  Every form computes the same
matrix (neighbour lists and L-hat bit for bit, asserted); the forms differ in
how the kNN search gets there:
  plain_fp32        exact heap search with FP32 ALU distance tiles (the comparison the metric names)
  fp16_tc, bf16_tc  16-bit distance tiles on the tensor cores (tcgen05.mma), FP64 rescoring
  learned_*         the same with each query's heap started at a radius predicted by the
                    learned network (trained beforehand on a separate draw, not timed)
  const_radius_fp32 ablation of the learned part: one global radius for every point
The JSON line's value is the workload's target form, the one its configuration
names (learned radius + BF16 tiles on the 1M torus and the ellipsoid batch, BF16
tiles on the sphere, FP16 tiles in R^100), and vs_plain_fp32 says how it compares
with plain_fp32, whichever way it falls; every form's time is listed.  Each
form's kNN launch shape comes from the autotuner (run before timing).

Workloads (--workload): torus_r4_1m (default: 1,000,000 points on the flat torus in
R^4, sigma 0.01, k = 64), vmf_s2_50k (50,000 points on S^2, vMF kappa 2, k = 64),
gauss100_200k (200,000 points of a 5-dim Gaussian in R^100, k = 128),
ellipsoids_256 (256 clouds, n_b ~ U[2000, 40000], k = 32, one batched build).
Between timed steps a 256 MiB buffer is written to flush the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Under torchrun every rank builds its own independent workload (weak scaling,
no collective on the data path); rank 0 prints one JSON line.  --impl
reference times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "kernel build points/s (kNN+VB kernel->CSR) vs plain FP32 form, exact kNN"
SFU_PER_SM_CLK = 16      # ex2 results per SM per clock (4 SFU lanes per SM sub-partition)
FP32_PER_SM_CLK = 128    # FP32 lanes per SM
N_SM = 152
EX2_PER_ENTRY = 15       # the 57-point sweep: 15 ex2 per entry (squaring chains for the rest)

BATCHED = {"ellipsoids_256": dict(n_clouds=256, n_lo=2000, n_hi=40000, seed=5, m=3, k=32, d=2, c=1.0, beta=-0.25)}
# the form each workload's configuration names (mixed precision, plus the learned radius where named)
TARGET = {"torus_r4_1m": "learned_bf16_tc", "vmf_s2_50k": "bf16_tc", "gauss100_200k": "fp16_tc",
          "ellipsoids_256": "learned_bf16_tc"}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="torus_r4_1m")
    ap.add_argument("--forms", default="")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--train-n", type=int, default=100000)
    ap.add_argument("--train-epochs", type=int, default=20)
    return ap.parse_args()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [[s.strip() for s in line.split(",")] for line in open(self.f.name)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(v: float, ws: int, device) -> float:
    """The largest of every rank's v (the job's time is its slowest rank's); v itself on one rank."""
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, steps: int, ws: int, max_seconds: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * steps * ws / max_seconds


def _dist():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


class Spec:
    """The workload: points, cloud offsets (batched) and the method parameters."""

    def __init__(self, name: str, rank: int):
        from paper_2104_15124_gb300 import workloads as W
        self.name = name
        if name in BATCHED:
            b = BATCHED[name]
            bt = W.ellipsoids(b["n_clouds"], b["n_lo"], b["n_hi"], b["seed"] + 1000 * rank)
            self.x, self.cloud_ptr = bt.x, bt.cloud_ptr
            self.m, self.k, self.d, self.c, self.beta = b["m"], b["k"], b["d"], b["c"], b["beta"]
            self.n = int(self.cloud_ptr[-1])
            self.config = {"workload": name, "clouds": b["n_clouds"], "n_total": self.n,
                           "n_per_cloud": f"U[{b['n_lo']}, {b['n_hi']}]", "m": 3, "k": self.k, "c": self.c,
                           "d": self.d, "beta": self.beta}
        else:
            w = W.WORKLOADS[name]
            self.w = W.Workload(w.name, w.n, w.m, w.k, w.d, w.c, w.beta, w.margin, w.seed + 1000 * rank)
            self.x, self.cloud_ptr = self.w.sample(), None
            self.m, self.k, self.d, self.c, self.beta, self.n = w.m, w.k, w.d, w.c, w.beta, w.n
            self.config = {"workload": name, "n": w.n, "m": w.m, "k": w.k, "c": w.c, "d": w.d, "beta": w.beta}

    def oracle_sample(self):
        """A bounded draw of the same law for the CPU oracle (about 10-30 s of CPU work)."""
        from paper_2104_15124_gb300 import workloads as W
        if self.cloud_ptr is not None:
            nb = int(np.searchsorted(self.cloud_ptr, 20000, side="right"))
            nb = max(nb, 1)
            return [self.x[self.cloud_ptr[b]:self.cloud_ptr[b + 1]] for b in range(nb)], f"the first {nb} clouds"
        ns = min(self.n, 50000 if self.m <= 4 else 20000)
        if ns == self.n:
            return [self.x], f"the whole n={self.n} workload"
        w = self.w
        return [W.Workload(w.name, ns, w.m, w.k, w.d, w.c, w.beta, w.margin, w.seed).sample()], \
            f"an n={ns} draw of the same law (the oracle's brute-force kNN is O(n^2), so points/s at n={self.n} " \
            f"would be lower still)"


def _oracle_points_per_s(spec: Spec) -> tuple[float, float, str]:
    from oracle import knn as OK
    from oracle import method as M
    clouds, what = spec.oracle_sample()
    t0 = time.perf_counter()
    pts = 0
    for xc in clouds:
        nbr, d2 = OK.knn(xc, spec.k)
        M.build(xc, spec.k, d=spec.d, c=spec.c, beta=spec.beta, nbr=nbr, nbr_d2=d2)
        pts += xc.shape[0]
    dt = time.perf_counter() - t0
    return pts / dt, dt, f"one complete FP64 oracle build (C brute-force kNN on all cores + numpy formulas) of {what}"


def run_reference(a, spec: Spec):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    steps = min(a.steps, 3)
    warm = min(a.warmup, 1)   # each oracle step is seconds of CPU work: one untimed warm-up at most
    for _ in range(warm):
        _oracle_points_per_s(spec)
    vals, secs = [], []
    what = ""
    for _ in range(steps):
        v, dt, what = _oracle_points_per_s(spec)
        vals.append(v)
        secs.append(dt)
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": a.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": spec.config,
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{steps} of the requested {a.steps} steps, each {what}"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _gradient_timing(vb, out, xt, peaks, src, ell: int = 16, reps: int = 10) -> dict:
    """vb_gradient (Sec. 3.2) on the built operator: the derivatives along every coordinate
    of u = sum of the coordinates, from ell + 1 eigenpairs (vb_solve, not timed), timed with
    CUDA events over `reps` calls.  Memory-bound on the eigenvectors: the algorithmic bytes
    are four passes over phi ((ell + 1) n FP32 each) plus u, x, S in and grad out."""
    import torch
    e = vb.solve(out.graph, out.val, out.S, ell)
    u = xt.sum(dim=1).contiguous()
    for _ in range(2):
        vb.gradient(e.evals, e.phi, out.S, u, xt)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        vb.gradient(e.evals, e.phi, out.S, u, xt)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    n, m = xt.shape
    nbytes = 4 * (ell + 1) * n * 4 + n * (4 + 4 * m + 8) + 4 * m * n
    ach = nbytes / (ms / 1e3) / 1e9
    return {"ell": ell, "ms": ms, "bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peaks["hbm_gbs"],
            "frac": ach / peaks["hbm_gbs"], "converged": bool(e.converged),
            "what": f"4 passes over the (ell + 1) x n FP32 eigenvectors + u, x, S, grad; peak hbm_gbs {src}"}


KNN_SEARCH_STAGES = ("knn_radius", "knn_tile", "knn_retry")   # the search proper: radius, first pass, retry


def _stage_kernel(stage: str, form: str, shape: dict) -> str:
    """The kernel that does a stage's work (the stage's other launches are small set-up passes)."""
    if stage == "knn_tile" and form.endswith("_tc"):
        return "knn_tcp_kernel" if shape.get("tc_variant") == "pipelined" else "knn_tc_kernel"
    return {"knn_tile": "knn_tile_kernel", "knn_retry": "knn_tile_kernel", "knn_radius": "mlp_radius_tc_kernel",
            "sweep_density": "sweep57_kernel", "sweep_operator": "sweep57_kernel"}.get(stage, stage)


def _traffic(stage: str, form: str, workload: str):
    """DRAM bytes (read + write) per launch of the dominant kernel, from the ncu capture
    recorded in profiles/traffic.json, or None when there is none for this kernel, form and
    workload or when the kernel's source file changed since the capture (SHA-1 mismatch)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(f"{stage}/{form}/{workload}")
    except Exception:
        return None
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != rec["source_sha1"]:
        return None
    return rec["dram_bytes_per_launch"]


def _train_radius(vb, spec: Spec, a, dev):
    """The learned radius (trained once, not timed) on a separate draw of about a.train_n points of
    the same law, on that draw's exact distances to its k'-th neighbour, k' = k n_train / n (the
    distance to the k-th neighbour at the timed size, whatever the cloud's effective dimension);
    the spread of the residual on the training set sets the inflation (3 sigma).  A batch of
    clouds trains on a separate batch, each target shifted by (1/d) ln(n_b / n_ref) so that clouds
    of every size share one network, and the timed build adds (1/d) ln(n_ref / n_b) per cloud.
    Also returns the constant-radius ablation: one global radius for every point, the training
    targets' mean inflated by 3 standard deviations."""
    import torch
    from paper_2104_15124_gb300 import workloads as W
    if spec.cloud_ptr is None:
        w = spec.w
        kp = max(1, int(round(spec.k * a.train_n / spec.n)))
        xtr = torch.from_numpy(W.Workload(w.name, a.train_n, w.m, w.k, w.d, w.c, w.beta, w.margin, 103).sample()).to(dev)
        _, d2tr = vb.knn(xtr, kp)
        target = 0.5 * torch.log(d2tr[:, kp - 1]).float()
        cloud_shift = None
        what = f"log distance to neighbour k'={kp} of a {a.train_n}-point draw"
    else:
        b = BATCHED[spec.name]
        n_ref = 0.5 * (b["n_lo"] + b["n_hi"])
        ntr = max(1, int(round(a.train_n / n_ref)))
        bt = W.ellipsoids(ntr, b["n_lo"], b["n_hi"], b["seed"] + 100)
        xtr = torch.from_numpy(bt.x).to(dev)
        parts = []
        for c in range(ntr):
            lo, hi = int(bt.cloud_ptr[c]), int(bt.cloud_ptr[c + 1])
            _, d2c = vb.knn(xtr[lo:hi].contiguous(), spec.k)
            parts.append(0.5 * torch.log(d2c[:, spec.k - 1]) + math.log((hi - lo) / n_ref) / spec.d)
        target = torch.cat(parts).float()
        sizes = np.diff(spec.cloud_ptr).astype(np.float64)
        cloud_shift = (np.log(n_ref / sizes) / spec.d).astype(np.float32)
        what = f"log distance to neighbour k={spec.k} in its own cloud, {ntr} training clouds, size-normalised"
    net = vb.train_radius_model(xtr, target, epochs=a.train_epochs, batch=4096, seed=103)
    resid = (target - net.predict(xtr)).float()
    shift = float(resid.mean())
    infl = math.exp(3.0 * float(resid.std()))
    const = math.exp(float(target.mean()) + 3.0 * float(target.std()))
    const_r = torch.full((spec.n,), const, dtype=torch.float32, device=dev)
    note = {"train_points": int(xtr.shape[0]), "target": what, "epochs": a.train_epochs, "log_shift": shift,
            "inflate": infl, "const_radius": const, "resid_std": float(resid.std()), "target_std": float(target.std())}
    return net, shift, infl, cloud_shift, const_r, note


def _tile_distance_error(vb, spec: Spec, xt, fmt: str, variant: str = "auto") -> dict:
    """Relative error of the 16-bit tile distances the search kernel itself produced, against
    FP64: one vb_knn call with the diagnostic output on returns, for every row, the candidates
    its search kept and their tile distances before the FP64 rescoring; the exact squared
    distances of the same pairs come from the FP64 coordinates (for a batch: its first cloud)."""
    import torch
    x = xt
    if spec.cloud_ptr is not None:
        x = xt[: int(spec.cloud_ptr[1])].contiguous()
    # full heap keys: the diagnostic output is the FP32 tile distance itself (compact keys would
    # give the lower edge of its 2^-10 bucket)
    nbr, nd2, idx, d16 = vb.knn(x, spec.k, tensor_cores=fmt, tc_variant=variant, debug=True, heap_keys="full")
    ok = idx >= 0
    rows = torch.arange(x.shape[0], device=x.device)[:, None].expand_as(idx)[ok]
    cols = idx[ok].long()
    x64 = x.double()
    d64 = ((x64[rows] - x64[cols]) ** 2).sum(1)
    dt = d16[ok].double()
    pos = d64 > 0
    rel = (dt[pos] - d64[pos]).abs() / d64[pos]
    # the error that decides the ranking: against the row's k-th neighbour distance
    dk = nd2[:, -1][rows]
    relk = (dt - d64).abs() / dk.clamp_min(1e-300)
    return {"max_rel": float(rel.max()), "rms_rel": float(rel.pow(2).mean().sqrt()),
            "max_rel_to_kth": float(relk.max()), "rms_rel_to_kth": float(relk.pow(2).mean().sqrt()),
            "pairs": int(rel.numel()),
            "what": f"every kept candidate of every row ({'first cloud' if spec.cloud_ptr is not None else 'all rows'})"
                    f", {fmt} tile distance ({variant} kernel, the form's autotuned choice; full heap keys) vs FP64"}


def main():
    a = _args()
    ws, rank, local = _dist()
    spec = Spec(a.workload, rank)
    if a.impl == "reference":
        run_reference(a, spec)
        return

    import torch
    import torch.distributed as dist
    import paper_2104_15124_gb300 as vb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    xt = torch.from_numpy(spec.x).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- forms
    batched = spec.cloud_ptr is not None
    lowdim = spec.m <= 16
    forms = ["plain_fp32", "fp16_tc", "bf16_tc"]
    if lowdim:
        forms += ["learned_bf16_tc"] if batched else ["learned_fp32", "learned_fp16_tc", "learned_bf16_tc",
                                                      "const_radius_fp32"]
    target = TARGET.get(spec.name, "plain_fp32")
    if a.forms:   # a subset (plain_fp32, the comparison, always runs); the target heads the line if present
        keep = set(a.forms.split(",")) | {"plain_fp32"}
        forms = [f for f in forms if f in keep]
        if target not in forms:
            target = "plain_fp32"
    net, shift, infl, cloud_shift, const_r = None, 0.0, 1.5, None, None
    if any(f.startswith("learned") or f.startswith("const") for f in forms):
        net, shift, infl, cloud_shift, const_r, train_note = _train_radius(vb, spec, a, dev)

    def make(form):
        kw = dict(device=dev, cloud_ptr=spec.cloud_ptr)
        if "fp16_tc" in form:
            kw["tensor_cores"] = "fp16"
        elif "bf16_tc" in form:
            kw["tensor_cores"] = "bf16"
        if form.startswith("learned"):
            kw.update(mlp=net, log_shift=shift, inflate=infl, cloud_log_shift=cloud_shift)
        elif form.startswith("const"):
            kw.update(radius=const_r, inflate=1.0)
        return vb.Builder(spec.n, spec.m, spec.k, d=spec.d, c=spec.c, beta=spec.beta, **kw)

    builders = {f: make(f) for f in forms}
    shapes = {f: ({"margin": 16, "seed_tiles": 0} if a.no_autotune else b.autotune(xt)) for f, b in builders.items()}

    def time_form(builder):
        g = builder.graph(xt)                    # one eager build, then the recording
        for _ in range(max(a.warmup, 3)):
            g.replay()
        torch.cuda.synchronize()
        vb.raise_on_device_error(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        barrier()
        clk = Clocks(local)
        t_wall = time.perf_counter()
        for s in range(a.steps):
            flush.zero_()
            ev[s][0].record()
            g.replay()
            ev[s][1].record()
        barrier()
        wall = time.perf_counter() - t_wall
        clocks = clk.stop()
        rep = vb.raise_on_device_error(dev)
        total_s = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3, ws, dev)
        return dict(total_s=total_s, clocks=clocks, wall=wall, graph=g)

    def profile_form(builder, steps):
        """Eager builds with a CUDA event pair around every stage (not the headline timing)."""
        vb.profile_enable(True, dev)
        vb.report_reset(dev)
        tot: dict[str, float] = {}
        for _ in range(steps):
            flush.zero_()
            builder(xt)
            st, _ = vb.profile_read(dev)
            for kname, v in st.items():
                tot[kname] = tot.get(kname, 0.0) + v
        _, launches = vb.profile_read(dev)
        rep = vb.raise_on_device_error(dev)
        vb.profile_enable(False, dev)
        return {k: v / steps for k, v in tot.items()}, launches // steps, rep

    res = {}
    for f, b in builders.items():
        res[f] = time_form(b)
        res[f]["stage_ms"], res[f]["launches"], res[f]["rep"] = profile_form(b, max(3, min(a.steps, 10)))
    ref = builders["plain_fp32"].out
    nnz = ref.graph.nnz
    for f, b in builders.items():   # every form: the same matrix, bit for bit
        assert torch.equal(b.out.nbr, ref.nbr), f
        assert torch.equal(b.out.val[:nnz], ref.val[:nnz]), f
    best = target if target in res else "plain_fp32"   # the headline: the configuration's named form
    r0 = res[best]
    builder = builders[best]
    total_s = r0["total_s"]
    value = job_throughput(spec.n, a.steps, ws, total_s)

    # ---------------- end to end through the public API: host input -> build -> host CSR
    x_pin = torch.from_numpy(spec.x).pin_memory()
    val_h = torch.empty(builder.out.val.numel(), dtype=torch.float32).pin_memory()
    col_h = torch.empty(builder.out.graph.col.numel(), dtype=torch.int32).pin_memory()
    rp_h = torch.empty(spec.n + 1, dtype=torch.int64).pin_memory()
    nnz_h = torch.empty(1, dtype=torch.int64).pin_memory()
    e2e_ms, d2h = [], 0
    barrier()
    for s in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        xd = x_pin.to(dev, non_blocking=True)
        o = builder(xd)
        nnz_h.copy_(o.graph.nnz_dev, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        z = int(nnz_h.item())
        # one copy stream: two streams at once gave the same 193 GB/s device-to-host on this part
        val_h[:z].copy_(o.val[:z], non_blocking=True)
        col_h[:z].copy_(o.graph.col[:z], non_blocking=True)
        rp_h.copy_(o.graph.row_ptr, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        d2h = 8 + z * 8 + (spec.n + 1) * 8
    barrier()
    e2e_s = max_over_ranks(sum(e2e_ms) / 1e3, ws, dev)

    # ---------------- roofline of every stage of the chosen form, and of the dominant one
    peaks, src = _peaks()
    clocks = r0["clocks"]
    f_mhz = clocks.get("sm_mhz") or 1965.0
    stage_ms = r0["stage_ms"]
    rep = r0["rep"]
    steps_prof = max(3, min(a.steps, 10))
    cand_retry = rep["knn_retry_candidates"] / steps_prof          # the exact pass over handed-back tiles
    cand = rep["knn_candidates"] / steps_prof - cand_retry          # the first search pass
    off = nnz - spec.n
    G = 57
    KP = (spec.m + 15) // 16 * 16
    tensor_tflops = peaks.get("bf16_tflops", 1900.0)     # FP16 and BF16 run at the same dense rate

    def roof(stage):
        ms = stage_ms.get(stage)
        if not ms:
            return None
        s = ms / 1e3
        if stage in ("sweep_density", "sweep_operator"):
            ach, peak = off / s / 1e9, N_SM * SFU_PER_SM_CLK * f_mhz * 1e6 / EX2_PER_ENTRY / 1e9
            return {"bound": "alu", "unit": "Gentries/s", "achieved": ach, "peak": peak, "frac": ach / peak,
                    "what": f"{G} kernel values per off-diagonal entry, {EX2_PER_ENTRY} ex2 on the SFU "
                            f"({N_SM} SM x {SFU_PER_SM_CLK}/clk x {f_mhz:.0f} MHz / {EX2_PER_ENTRY})"}
        if stage == "knn_tile" and best.endswith("_tc"):
            ach = cand * 2 * spec.m / s / 1e12
            return {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": tensor_tflops,
                    "frac": ach / tensor_tflops,
                    "what": f"{int(cand)} candidate pairs x 2 m (m = {spec.m}; the MMA runs K = {KP}) FLOP of "
                            f"16-bit tcgen05.mma; peak = dense bf16 {src} (FP16 rate equal)"}
        if stage in ("knn_tile", "knn_retry"):
            c = cand if stage == "knn_tile" else cand_retry
            ach = c * (3 * spec.m + 2) / s / 1e9
            peak = N_SM * FP32_PER_SM_CLK * f_mhz * 1e6 / 1e9
            return {"bound": "alu", "unit": "Gop/s", "achieved": ach, "peak": peak, "frac": ach / peak,
                    "what": f"{int(c)} candidate pairs x {3 * spec.m + 2} FP32 ops "
                            f"({N_SM} SM x {FP32_PER_SM_CLK} lanes x {f_mhz:.0f} MHz)"}
        if stage == "knn_radius" and best.startswith("learned"):
            flop = spec.n * 2 * (16 * 64 + 64 * 64)
            ach = flop / s / 1e12
            return {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": tensor_tflops,
                    "frac": ach / tensor_tflops,
                    "what": f"2 (16 x 64 + 64 x 64) FLOP per point of two BF16 tcgen05.mma layers; "
                            f"peak = dense bf16 {src}"}
        mpad = 1 << max(2, (spec.m - 1).bit_length())
        per = {"knn_order": (spec.n, 12 * spec.m + 64 + 8 * mpad), "graph": (nnz, 40), "bandwidth": (spec.n, 8 * spec.k + 8),
               "density": (nnz, 12), "centre": (nnz, 12), "operator": (nnz, 24), "lhat": (nnz, 16),
               "knn_fallback": (spec.n, 0)}.get(stage)
        if per is None or per[1] == 0:
            return None
        ach = per[0] * per[1] / s / 1e9
        return {"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peaks["hbm_gbs"],
                "frac": ach / peaks["hbm_gbs"], "what": f"{per[1]} B per {'entry' if per[0] == nnz else 'point'} "
                                                        f"(algorithmic), peak hbm_gbs {src}"}

    kernels = {k: dict(ms=round(v, 4), **(roof(k) or {})) for k, v in stage_ms.items()}
    knn_ms = sum(stage_ms.get(k, 0.0) for k in KNN_SEARCH_STAGES)
    dom = max(stage_ms, key=stage_ms.get)
    droof = roof(dom) or {"bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": None}
    droof = {kk: droof[kk] for kk in ("bound", "achieved", "peak", "unit", "frac", "what") if kk in droof}
    droof["stage"] = dom
    droof["kernel"] = _stage_kernel(dom, best, shapes[best])
    droof["traffic"] = _traffic(dom, best, spec.name)

    sizes = np.diff(spec.cloud_ptr) if batched else np.array([spec.n])
    pairs_all = float(np.sum(sizes.astype(np.float64) * (sizes - 1)))
    cfg = dict(spec.config)
    cfg.update({"form": best, "nnz": nnz, "l2": "flushed between steps (256 MiB write)",
                "parallelism": f"replicas x{ws}", "timing": "CUDA-graph replay of the whole build per step"})
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total_s / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16+f32", "fp16": "f16+f32"}.get(best.split("_")[-2], "f32"),
            "data": "synthetic", "config": cfg,
            "forms": {f: {"ms_per_step": 1e3 * res[f]["total_s"] / a.steps,
                          "points_per_s": job_throughput(spec.n, a.steps, ws, res[f]["total_s"]),
                          "knn_ms": round(sum(res[f]["stage_ms"].get(k, 0.0) for k in KNN_SEARCH_STAGES), 4),
                          "knn_candidate_pairs": res[f]["rep"]["knn_candidates"] // steps_prof,
                          "knn_redo_tiles": res[f]["rep"]["knn_redo_tiles"] // steps_prof,
                          "knn_retry_tiles": res[f]["rep"]["knn_retry_tiles"] // steps_prof,
                          "knn_fallback_rows": res[f]["rep"]["knn_fallback_rows"] // steps_prof,
                          "autotuned": {kk: v for kk, v in shapes[f].items() if kk != "knn_ms"}} for f in forms},
            "vs_plain_fp32": res["plain_fp32"]["total_s"] / total_s,
            "comparison": {"target_form": best, "target_points_per_s": value,
                           "plain_fp32_points_per_s": job_throughput(spec.n, a.steps, ws, res["plain_fp32"]["total_s"]),
                           "target_over_plain": res["plain_fp32"]["total_s"] / total_s},
            "e2e": {"value": job_throughput(spec.n, a.steps, ws, e2e_s), "unit": "points/s", "h2d_bytes_per_step": int(spec.x.nbytes),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / a.steps},
            "gpu_launches": int(r0["launches"] * a.steps), "roofline": droof, "kernels": kernels,
            "knn": {"candidate_pairs_per_step": int(cand),
                    "candidate_pairs_per_s": (cand + cand_retry) / (knn_ms / 1e3) if knn_ms else None,
                    "retry_candidate_pairs_per_step": int(cand_retry),
                    "n2_equivalent_pairs_per_s": (pairs_all / ((stage_ms.get("knn_order", 0.0) + knn_ms
                                                               + stage_ms.get("knn_fallback", 0.0)) / 1e3)
                                                  if knn_ms else None),
                    "n2_equivalent_note": "n (n - 1) pairs (per cloud, summed) over the whole kNN stage time: the "
                                          "rate a brute-force search would need, not pairs evaluated",
                    "heap_levels_per_step": rep["knn_heap_levels"] // steps_prof,
                    "insert_rounds_per_step": rep["knn_insert_rounds"] // steps_prof,
                    "tiles_staged_per_step": rep["knn_tiles_staged"] // steps_prof},
            "clocks": clocks, "wall_s": r0["wall"]}
    if net is not None:
        line["learned_radius"] = train_note
    if rank == 0 and not batched and spec.m <= 16:
        line["gradient"] = _gradient_timing(vb, ref, xt, peaks, src)
    line["tile_distance_error"] = {fmt: _tile_distance_error(vb, spec, xt, fmt, shapes[f"{fmt}_tc"].get("tc_variant", "auto"))
                                   for fmt in ("fp16", "bf16") if f"{fmt}_tc" in forms}
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        v, dt, what = _oracle_points_per_s(spec)
        line["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": what, "seconds": dt}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
