#!/usr/bin/env python
"""Benchmark of the variable-bandwidth kernel build (kNN + VB kernel -> L-hat CSR).

One step = one complete build (vb_build: exact kNN, symmetric pattern,
bandwidth, density sweep, density, operator sweep, normalisations, L-hat CSR)
of one synthetic point cloud whose coordinates are already resident in HBM.
The default workload is 50,000 points on S^2 from a von Mises-Fisher law
(kappa = 2 about +z), k = 64, c = 1, d = 2, beta = -1/4, plain FP32 distances
with exact kNN.  Between timed steps a 256 MiB buffer is written to flush the
129 MB L2 (the workload's working set fits in L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank builds its own independent cloud (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  --impl reference
times the FP64 CPU oracle on the host cores instead (rank 0 only).
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


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vmf_s2_50k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-n", type=int, default=20000)
    ap.add_argument("--train-epochs", type=int, default=20)
    return ap.parse_args()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
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
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_baseline(w, x) -> dict:
    """The FP64 oracle as it stands, on the host cores, over the whole workload once."""
    from oracle import knn as OK
    from oracle import method as M
    t0 = time.perf_counter()
    nbr, d2 = OK.knn(x, w.k)
    t1 = time.perf_counter()
    M.build(x, w.k, d=w.d, c=w.c, beta=w.beta, nbr=nbr, nbr_d2=d2)
    t2 = time.perf_counter()
    return {"value": x.shape[0] / (t2 - t0), "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one complete FP64 oracle build of the n={x.shape[0]} workload "
                      f"(C brute-force kNN {t1 - t0:.2f} s on all cores, numpy formulas {t2 - t1:.2f} s)",
            "seconds": t2 - t0}


def run_reference(a, w, x):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import knn as OK
    from oracle import method as M
    steps = min(a.steps, 3)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        nbr, d2 = OK.knn(x, w.k)
        M.build(x, w.k, d=w.d, c=w.c, beta=w.beta, nbr=nbr, nbr_d2=d2)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    v = x.shape[0] / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": a.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "m": w.m, "k": w.k, "c": w.c, "d": w.d, "beta": w.beta},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{steps} of the requested {a.steps} steps, each one complete FP64 oracle "
                                       f"build of the n={x.shape[0]} workload"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    from paper_2104_15124_gb300 import workloads as W
    w = W.WORKLOADS[a.workload]
    ws, rank, local = _dist()
    if a.impl == "reference":
        run_reference(a, w, w.sample())
        return

    import torch
    import torch.distributed as dist
    import paper_2104_15124_gb300 as vb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    # weak scaling: every rank builds its own cloud of the same law (seed offset by rank)
    wl = W.Workload(w.name, w.n, w.m, w.k, w.d, w.c, w.beta, w.margin, w.seed + 1000 * rank)
    x = wl.sample()
    xt = torch.from_numpy(x).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # The learned radius: trained once (not timed) on a separate draw of the same law, on the
    # method's own exact k-th neighbour distances (the model is weights, like any network's).
    wt = W.Workload(w.name, a.train_n, w.m, w.k, w.d, w.c, w.beta, w.margin, 103)
    xtr = torch.from_numpy(wt.sample()).to(dev)
    _, d2tr = vb.knn(xtr, w.k)
    net = vb.train_radius_model(xtr, 0.5 * torch.log(d2tr[:, w.k - 1]).float(), epochs=a.train_epochs,
                                batch=4096, seed=103)
    shift = math.log(a.train_n / w.n) / w.d    # r_k scales like n^(-1/d)
    forms = {
        "learned": vb.Builder(w.n, w.m, w.k, d=w.d, c=w.c, beta=w.beta, margin=4, device=dev, mlp=net,
                              log_shift=shift, inflate=1.5),
        "plain_fp32": vb.Builder(w.n, w.m, w.k, d=w.d, c=w.c, beta=w.beta, margin=4, device=dev),
    }

    def time_form(builder):
        for _ in range(max(a.warmup, 3)):
            builder(xt)
        torch.cuda.synchronize()
        vb.raise_on_device_error(dev)
        vb.profile_enable(True, dev)
        vb.report_reset(dev)
        stage_tot: dict[str, float] = {}
        step_ms = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        barrier()
        clk = Clocks(local)
        t_wall = time.perf_counter()
        for s in range(a.steps):
            flush.zero_()
            ev[s][0].record()
            builder(xt)
            ev[s][1].record()
            st, _ = vb.profile_read(dev)          # synchronises the stream
            for kname, v in st.items():
                stage_tot[kname] = stage_tot.get(kname, 0.0) + v
            step_ms.append(ev[s][0].elapsed_time(ev[s][1]))
        barrier()
        wall = time.perf_counter() - t_wall
        clocks = clk.stop()
        _, launches = vb.profile_read(dev)
        rep = vb.raise_on_device_error(dev)
        vb.profile_enable(False, dev)
        total_s = sum(step_ms) / 1e3
        if ws > 1:
            t = torch.tensor([total_s], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_s = float(t.item())
        return dict(total_s=total_s, stage_ms={k: v / a.steps for k, v in stage_tot.items()}, launches=launches,
                    rep=rep, clocks=clocks, wall=wall)

    res = {name: time_form(b) for name, b in forms.items()}
    primary = "learned"
    builder = forms[primary]
    r0 = res[primary]
    total_s, stage_tot, launches, rep, clocks, wall = (r0["total_s"], None, r0["launches"], r0["rep"], r0["clocks"],
                                                       r0["wall"])
    value = w.n * a.steps * ws / total_s
    nnz = builder.out.graph.nnz
    # the plain FP32 form computes the same matrix: neighbour lists and L-hat bit for bit
    assert torch.equal(forms["plain_fp32"].out.nbr, builder.out.nbr)
    assert torch.equal(forms["plain_fp32"].out.val[:nnz], builder.out.val[:nnz])

    # ---------------- end to end through the public API: host input -> build -> host CSR
    x_pin = torch.from_numpy(x).pin_memory()
    val_h = torch.empty(builder.out.val.numel(), dtype=torch.float32).pin_memory()
    col_h = torch.empty(builder.out.graph.col.numel(), dtype=torch.int32).pin_memory()
    rp_h = torch.empty(w.n + 1, dtype=torch.int64).pin_memory()
    nnz_h = torch.empty(1, dtype=torch.int64).pin_memory()
    e2e_ms = []
    d2h = 0
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
        val_h[:z].copy_(o.val[:z], non_blocking=True)
        col_h[:z].copy_(o.graph.col[:z], non_blocking=True)
        rp_h.copy_(o.graph.row_ptr, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        d2h = 8 + z * 8 + (w.n + 1) * 8
    barrier()
    e2e_s = sum(e2e_ms) / 1e3
    if ws > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # ---------------- roofline of the dominant kernel
    peaks, src = _peaks()
    f_mhz = clocks.get("sm_mhz") or 1965.0
    stage_ms = r0["stage_ms"]
    dom = max(stage_ms, key=stage_ms.get)
    off = nnz - w.n
    G = builder.out.chi_den.numel()
    cand = rep["knn_candidates"] / a.steps
    if dom in ("sweep_density", "sweep_operator"):
        achieved = G * off / (stage_ms[dom] / 1e3) / 1e9
        peak = N_SM * SFU_PER_SM_CLK * f_mhz * 1e6 / 1e9
        roof = {"bound": "alu", "unit": "Gexp/s", "what": f"{dom}: {G} ex2 per off-diagonal entry on the SFU",
                "peak_source": f"{N_SM} SM x {SFU_PER_SM_CLK} ex2/clk x {f_mhz:.0f} MHz (sampled)"}
    elif dom == "knn_tile":
        ops = cand * (3 * w.m + 2)
        achieved = ops / (stage_ms[dom] / 1e3) / 1e9
        peak = N_SM * FP32_PER_SM_CLK * f_mhz * 1e6 / 1e9
        roof = {"bound": "alu", "unit": "Gop/s", "what": f"knn_tile: {int(cand)} candidate pairs x {3 * w.m + 2} FP32 ops",
                "peak_source": f"{N_SM} SM x {FP32_PER_SM_CLK} FP32 lanes x {f_mhz:.0f} MHz (sampled)"}
    else:
        per_nnz = {"lhat": 16, "operator": 24, "density": 12, "centre": 12, "graph": 40}.get(dom, 8)
        achieved = per_nnz * nnz / (stage_ms[dom] / 1e3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "unit": "GB/s", "what": f"{dom}: {per_nnz} B per stored entry",
                "peak_source": f"hbm_gbs of {src}"}
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak, "traffic": None})

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total_s / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "m": w.m, "k": w.k, "c": w.c, "d": w.d, "beta": w.beta,
                       "form": "learned radius-first search (MLP 3->64->64->1, BF16 weights) + FP32 ALU distances "
                               "+ FP64 rescoring, exact kNN", "radius_train": f"{a.train_n} points, seed 103, "
                       f"{a.train_epochs} epochs", "nnz": nnz, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"replicas x{ws}"},
            "plain_fp32": {"value": w.n * a.steps * ws / res["plain_fp32"]["total_s"], "unit": "points/s",
                           "ms_per_step": 1e3 * res["plain_fp32"]["total_s"] / a.steps,
                           "stages_ms": {k: round(v, 4) for k, v in res["plain_fp32"]["stage_ms"].items()},
                           "knn_candidate_pairs_per_step": res["plain_fp32"]["rep"]["knn_candidates"] // a.steps,
                           "note": "exact heap search (margin 4), same output bit for bit"},
            "e2e": {"value": w.n * a.steps * ws / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(x.nbytes),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / a.steps},
            "gpu_launches": int(launches), "roofline": roof,
            "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "knn": {"candidate_pairs_per_step": int(cand),
                    "candidate_pairs_per_s": cand / (stage_ms["knn_tile"] / 1e3) if "knn_tile" in stage_ms else None,
                    "fallback_rows_per_step": rep["knn_fallback_rows"] // a.steps,
                    "retry_tiles_per_step": rep["knn_retry_tiles"] // a.steps},
            "clocks": clocks, "wall_s": wall}
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(w, x)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
