"""Python binding of libvb (the C ABI in include/vb.h): argument marshalling only.

Every step of the variable-bandwidth kernel build runs in the CUDA kernels of
libvb.so; this module allocates the caller-side device buffers with PyTorch,
passes their pointers and the current CUDA stream, and turns status codes into
exceptions.  There is no CPU fallback: without the compiled library every call
raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvb.so")

VB_PREC_FP32, VB_PREC_BF16, VB_PREC_FP16 = 0, 1, 2
VB_PRUNE_NONE, VB_PRUNE_EXACT, VB_PRUNE_LEARNED = 0, 1, 2
VB_TC_AUTO, VB_TC_STAGED, VB_TC_PIPELINED = 0, 1, 2
VB_KEYS_COMPACT, VB_KEYS_FULL = 0, 1
VB_SPMV_PLAIN, VB_SPMV_LAPLACIAN = 0, 1
XI_LO, XI_HI, DXI = -10.0, 4.0, 0.25
VB_NOALLOC_MAX_N = 1 << 20   # rows vb_spmv_laplacian_noalloc accepts (its static scratch size)

_STATUS = {0: "VB_OK", -1: "VB_ERR_ARG", -2: "VB_ERR_CUDA", -3: "VB_ERR_WORKSPACE", -4: "VB_ERR_DEGENERATE",
           -5: "VB_ERR_EPS_BOUNDARY", -6: "VB_ERR_NOT_CONVERGED", -7: "VB_ERR_TIMEOUT", -8: "VB_ERR_BOUNDS",
           -9: "VB_ERR_UNSUPPORTED"}


class VbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_STATUS.get(code, code)}")


# ----------------------------------------------------------------------------- ctypes mirrors of vb.h
c_p = ctypes.c_void_p
c_i32, c_i64, c_f32, c_f64, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_size_t


class KnnParams(ctypes.Structure):
    _fields_ = [("k", c_i32), ("margin", c_i32), ("precision", c_i32), ("prune", c_i32), ("radius", c_p),
                ("mlp", c_p), ("radius_inflate", c_f32), ("radius_log_shift", c_f32), ("cloud_log_shift", c_p),
                ("seed_tiles", c_i32), ("tc_variant", c_i32), ("heap_keys", c_i32), ("dbg_d2", c_p), ("dbg_idx", c_p),
                ("curve", c_i32)]


class GraphC(ctypes.Structure):
    _fields_ = [("n", c_i64), ("row_ptr", c_p), ("col", c_p), ("ed2", c_p)]


class OpParams(ctypes.Structure):
    _fields_ = [("c", c_f64), ("beta", c_f64), ("d", c_f64)]


class BuildParams(ctypes.Structure):
    _fields_ = [("knn", KnnParams), ("k_bw", c_i32), ("op", OpParams), ("xi_lo", c_f64), ("xi_hi", c_f64),
                ("dxi", c_f64), ("pin_eps", c_i32)]


class BuildOut(ctypes.Structure):
    _fields_ = [(f, c_p) for f in ("nbr", "nbr_d2", "b", "row_ptr", "col", "ed2")] + [("cap", c_i64)] + \
               [(f, c_p) for f in ("nnz", "eps2_den", "chi_den", "dim_den", "psi", "P", "xi_c", "eps2_op", "chi_op",
                                   "dim_op", "val", "q", "D", "S")]


class SolveParams(ctypes.Structure):
    _fields_ = [("ell", c_i32), ("block", c_i32), ("degree", c_i32), ("max_iter", c_i32), ("tol", c_f64),
                ("seed", ctypes.c_uint64)]


class EvolveParams(ctypes.Structure):
    _fields_ = [("build", BuildParams), ("solve", SolveParams), ("dt", c_f64)]


class MlpC(ctypes.Structure):
    _fields_ = [("in_dim", c_i32), ("master", c_p), ("weights", c_p), ("adam_m", c_p), ("adam_v", c_p),
                ("in_mean", c_f32 * 16), ("in_scale", c_f32 * 16), ("out_mean", c_f32), ("out_scale", c_f32),
                ("step", c_i64)]


class Report(ctypes.Structure):
    _fields_ = [("error", c_i32), ("warnings", c_i32), ("knn_fallback_rows", c_i64), ("knn_candidates", c_i64),
                ("union_big_rows", c_i64), ("knn_heap_levels", c_i64), ("knn_tiles_staged", c_i64),
                ("knn_insert_rounds", c_i64), ("knn_retry_tiles", c_i64), ("knn_rows_short", c_i64),
                ("knn_rows_long_run", c_i64), ("knn_rows_uncertified", c_i64), ("knn_retry_candidates", c_i64),
                ("knn_redo_tiles", c_i64)]


_SIGS = {
    "vb_status_string": (ctypes.c_char_p, [c_i32]),
    "vb_create": (c_i32, [ctypes.POINTER(c_p), c_i32, c_p]),
    "vb_destroy": (c_i32, [c_p]),
    "vb_set_stream": (c_i32, [c_p, c_p]),
    "vb_report_read": (c_i32, [c_p, ctypes.POINTER(Report)]),
    "vb_report_reset": (c_i32, [c_p]),
    "vb_profile_enable": (c_i32, [c_p, c_i32]),
    "vb_profile_read": (c_i32, [c_p, ctypes.POINTER(c_f32), ctypes.POINTER(c_i64)]),
    "vb_knn_workspace": (c_sz, [c_i64, c_i32, ctypes.POINTER(KnnParams)]),
    "vb_knn": (c_i32, [c_p, c_p, c_i64, c_i32, ctypes.POINTER(KnnParams), c_p, c_p, c_p, c_sz]),
    "vb_knn_autotune": (c_i32, [c_p, c_p, c_i64, c_i32, c_p, c_i32, ctypes.POINTER(KnnParams), c_p, c_p, c_p,
                                c_sz, ctypes.POINTER(KnnParams), ctypes.POINTER(c_f32)]),
    "vb_graph_workspace": (c_sz, [c_i64, c_i32]),
    "vb_graph_build": (c_i32, [c_p, c_i64, c_i32, c_p, c_p, c_p, c_p, c_p, c_i64, c_p, c_p, c_sz]),
    "vb_bandwidth": (c_i32, [c_p, c_i64, c_i32, c_i32, c_p, c_p]),
    "vb_epsilon_tune_workspace": (c_sz, [c_i64]),
    "vb_epsilon_tune": (c_i32, [c_p, ctypes.POINTER(GraphC), c_p, c_f64, c_p, c_f64, c_f64, c_f64, c_i32, c_p, c_p,
                                c_p, c_p, c_sz]),
    "vb_density_workspace": (c_sz, [c_i64]),
    "vb_density": (c_i32, [c_p, ctypes.POINTER(GraphC), c_p, c_p, c_f64, c_f64, c_p, c_p, c_p, c_sz]),
    "vb_operator_centre_workspace": (c_sz, [c_i64]),
    "vb_operator_centre": (c_i32, [c_p, ctypes.POINTER(GraphC), c_p, c_p, c_p, c_p, c_sz]),
    "vb_kernel_csr_workspace": (c_sz, [c_i64]),
    "vb_kernel_csr": (c_i32, [c_p, ctypes.POINTER(GraphC), c_p, c_p, ctypes.POINTER(OpParams), c_p, c_p, c_p, c_p,
                              c_p, c_p, c_sz]),
    "vb_spmv_workspace": (c_sz, [c_i64]),
    "vb_spmv": (c_i32, [c_p, ctypes.POINTER(GraphC), c_p, c_p, c_i32, c_f32, c_p, c_f32, c_p, c_p, c_sz]),
    "vb_spmv_laplacian_noalloc": (c_i32, [c_p, ctypes.POINTER(GraphC), c_p, c_p, c_f32, c_p, c_f32, c_p]),
    "vb_solve_workspace": (c_sz, [c_i64, c_i64, ctypes.POINTER(SolveParams)]),
    "vb_gradient_workspace": (c_sz, [c_i64, c_i32, c_i32]),
    "vb_gradient": (c_i32, [c_p, c_i64, c_i32, c_p, c_p, c_p, c_p, c_p, c_i32, c_p, c_p, c_sz]),
    "vb_solve": (c_i32, [c_p, ctypes.POINTER(GraphC), c_i64, c_p, c_p, ctypes.POINTER(SolveParams), c_p, c_p, c_p,
                         c_p, ctypes.POINTER(c_i32), c_p, c_sz]),
    "vb_mlp_param_count": (c_i64, [c_i32]),
    "vb_mlp_init": (c_i32, [c_p, ctypes.POINTER(MlpC), ctypes.c_uint64]),
    "vb_mlp_standardise": (c_i32, [c_p, ctypes.POINTER(MlpC), c_p, c_i32, c_p, c_i64, c_p, c_sz]),
    "vb_mlp_workspace": (c_sz, [c_i32, c_i64]),
    "vb_mlp_train_epoch": (c_i32, [c_p, ctypes.POINTER(MlpC), c_p, c_i32, c_p, c_i64, c_i32, c_f32, ctypes.c_uint64,
                                   c_p, c_p, c_sz]),
    "vb_mlp_gradient": (c_i32, [c_p, ctypes.POINTER(MlpC), c_p, c_i32, c_p, c_i64, c_p, c_p, c_p, c_sz]),
    "vb_mlp_predict": (c_i32, [c_p, ctypes.POINTER(MlpC), c_p, c_i32, c_i64, c_p]),
    "vb_mlp_predict_tc": (c_i32, [c_p, ctypes.POINTER(MlpC), c_p, c_i32, c_i64, c_p]),
    "vb_tc_dot_tile": (c_i32, [c_p, c_p, c_p, c_i32, c_i32, c_p]),
    "vb_build_workspace": (c_sz, [c_i64, c_i32, ctypes.POINTER(BuildParams)]),
    "vb_build": (c_i32, [c_p, c_p, c_i64, c_i32, ctypes.POINTER(BuildParams), ctypes.POINTER(BuildOut), c_p, c_sz]),
    "vb_radius_workspace": (c_sz, [c_i64, c_i32]),
    "vb_radius_pattern": (c_i32, [c_p, c_p, c_i64, c_i32, c_p, c_f64, c_f64, c_p, c_p, c_p, c_i64, c_p, c_p, c_sz]),
    "vb_radius_sweep": (c_i32, [c_p, c_p, c_i64, c_i32, c_p, c_f64, c_f64, c_f64, c_f64, c_f64, c_p, c_p, c_p, c_p,
                                c_sz]),
    "vb_evolve_workspace": (c_sz, [c_i64, c_i32, ctypes.POINTER(EvolveParams)]),
    "vb_evolve_step": (c_i32, [c_p, c_p, c_i64, c_i32, ctypes.POINTER(EvolveParams), c_p, c_p, c_p, c_p,
                               ctypes.POINTER(BuildOut), c_p, c_p, c_p, c_p, c_sz]),
    "vb_build_batch_workspace": (c_sz, [c_i64, c_i32, c_i32, ctypes.POINTER(BuildParams)]),
    "vb_build_batch": (c_i32, [c_p, c_p, c_i64, c_i32, ctypes.POINTER(c_i64), c_p, c_i32, ctypes.POINTER(BuildParams),
                               ctypes.POINTER(BuildOut), c_p, c_sz]),
}
EXPORTED = tuple(_SIGS)

_lock = threading.Lock()
_lib = None
_ctxs: dict[int, int] = {}


def lib():
    """The loaded libvb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libvb.so is not built ({LIB_PATH}); run paper_2104_15124_gb300.native.compile_library()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(code: int, where: str) -> None:
    if code != 0:
        raise VbError(code, where)


def _ctx(device: torch.device) -> int:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    with _lock:
        h = _ctxs.get(idx)
    if h is None:
        out = c_p()
        _check(lib().vb_create(ctypes.byref(out), idx, c_p(torch.cuda.current_stream(idx).cuda_stream)), "vb_create")
        with _lock:
            _ctxs[idx] = out.value
        h = out.value
    _check(lib().vb_set_stream(c_p(h), c_p(torch.cuda.current_stream(idx).cuda_stream)), "vb_set_stream")
    return h


def _p(t: torch.Tensor | None) -> c_p:
    if t is None:
        return c_p(0)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return c_p(t.data_ptr())


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def report(device=None) -> dict:
    """Synchronises the current stream and returns the device report."""
    dev = torch.device("cuda", device if isinstance(device, int) else torch.cuda.current_device()) \
        if not isinstance(device, torch.device) else device
    r = Report()
    _check(lib().vb_report_read(c_p(_ctx(dev)), ctypes.byref(r)), "vb_report_read")
    return {name: getattr(r, name) for name, _ in Report._fields_}


def report_reset(device=None) -> None:
    dev = torch.device("cuda", device if isinstance(device, int) else torch.cuda.current_device()) \
        if not isinstance(device, torch.device) else device
    _check(lib().vb_report_reset(c_p(_ctx(dev))), "vb_report_reset")


def raise_on_device_error(device=None) -> dict:
    r = report(device)
    if r["error"] != 0:
        raise VbError(r["error"], "device report")
    return r


STAGES = ("knn_order", "knn_tile", "knn_fallback", "graph", "bandwidth", "sweep_density", "density", "centre",
          "sweep_operator", "operator", "lhat", "knn_radius", "knn_retry")


def profile_enable(on: bool = True, device=None) -> None:
    """Bracket every stage with CUDA events on the stream and count launches (measurement hook)."""
    dev = torch.device("cuda", device if isinstance(device, int) else torch.cuda.current_device()) \
        if not isinstance(device, torch.device) else device
    _check(lib().vb_profile_enable(c_p(_ctx(dev)), 1 if on else 0), "vb_profile_enable")


def profile_read(device=None) -> tuple[dict, int]:
    """(stage -> ms of its latest run, kernel launches enqueued since enabling); synchronises."""
    dev = torch.device("cuda", device if isinstance(device, int) else torch.cuda.current_device()) \
        if not isinstance(device, torch.device) else device
    ms = (c_f32 * len(STAGES))()
    n = c_i64()
    _check(lib().vb_profile_read(c_p(_ctx(dev)), ms, ctypes.byref(n)), "vb_profile_read")
    return {s: ms[i] for i, s in enumerate(STAGES) if ms[i] >= 0}, int(n.value)


# ----------------------------------------------------------------------------- graph handle
@dataclasses.dataclass
class Graph:
    """The symmetric CSR pattern: row_ptr [n+1] int64, col [cap] int32, ed2 [cap] fp32, nnz [1] int64 (device)."""
    n: int
    row_ptr: torch.Tensor
    col: torch.Tensor
    ed2: torch.Tensor
    nnz_dev: torch.Tensor

    def c(self) -> GraphC:
        return GraphC(self.n, _p(self.row_ptr), _p(self.col), _p(self.ed2))

    @property
    def nnz(self) -> int:
        return int(self.nnz_dev.item())


# ----------------------------------------------------------------------------- the calls
def knn(x: torch.Tensor, k: int, margin: int = 16, prune: bool = True, radius: torch.Tensor | None = None,
        inflate: float = 0.0, mlp=None, log_shift: float = 0.0, tensor_cores: str | None = None,
        tc_variant: str = "auto", seed_tiles: int = 0, heap_keys: str = "compact", debug: bool = False,
        curve: str = "auto"):
    """Exact kNN (vb_knn): returns (nbr int32 [n, k], nbr_d2 fp64 [n, k]).  With `radius` (per-point
    guess of the k-th neighbour distance) or a learned `mlp`, the radius-first search runs;
    tensor_cores = "fp16" or "bf16" computes its distance tiles on the tensor cores, with the
    kernel tc_variant = "auto", "staged" or "pipelined" (VB_TC_*); seed_tiles and heap_keys
    ("compact" or "full") and curve ("auto": Hilbert order at 2 <= m <= 4, or "morton") as in
    vb_knn_params.  debug=True (16-bit tiles) also returns the
    candidates each row kept and their 16-bit tile distances before rescoring:
    (nbr, nbr_d2, dbg_idx int32 [n, k + margin], dbg_d2 fp32 [n, k + margin])."""
    n, m = x.shape
    dev = x.device
    mode = VB_PRUNE_LEARNED if (radius is not None or mlp is not None) else (VB_PRUNE_EXACT if prune else VB_PRUNE_NONE)
    prec = {None: VB_PREC_FP32, "bf16": VB_PREC_BF16, "fp16": VB_PREC_FP16}[tensor_cores]
    p = KnnParams(k, margin, prec, mode, _p(radius),
                  c_p(0) if mlp is None else c_p(mlp.handle()), inflate, log_shift)
    p.tc_variant = {"auto": VB_TC_AUTO, "staged": VB_TC_STAGED, "pipelined": VB_TC_PIPELINED}[tc_variant]
    p.seed_tiles = seed_tiles
    p.heap_keys = {"compact": VB_KEYS_COMPACT, "full": VB_KEYS_FULL}[heap_keys]
    p.curve = {"auto": 0, "morton": 1}[curve]
    nbr = torch.empty((n, k), dtype=torch.int32, device=dev)
    d2 = torch.empty((n, k), dtype=torch.float64, device=dev)
    if debug:
        dbg_idx = torch.full((n, k + margin), -1, dtype=torch.int32, device=dev)
        dbg_d2 = torch.full((n, k + margin), float("nan"), dtype=torch.float32, device=dev)
        p.dbg_idx, p.dbg_d2 = _p(dbg_idx), _p(dbg_d2)
    ws = _ws(lib().vb_knn_workspace(n, m, ctypes.byref(p)), dev)
    _check(lib().vb_knn(c_p(_ctx(dev)), _p(x), n, m, ctypes.byref(p), _p(nbr), _p(d2), _p(ws), ws.numel()), "vb_knn")
    if debug:
        return nbr, d2, dbg_idx, dbg_d2
    return nbr, d2


def graph(nbr: torch.Tensor, nbr_d2: torch.Tensor) -> Graph:
    """Symmetric pattern diag U kNN U kNN^T (vb_graph_build)."""
    n, k = nbr.shape
    dev = nbr.device
    cap = n * (2 * k + 1)
    g = Graph(n, torch.empty(n + 1, dtype=torch.int64, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
              torch.empty(cap, dtype=torch.float32, device=dev), torch.empty(1, dtype=torch.int64, device=dev))
    ws = _ws(lib().vb_graph_workspace(n, k), dev)
    _check(lib().vb_graph_build(c_p(_ctx(dev)), n, k, _p(nbr), _p(nbr_d2), _p(g.row_ptr), _p(g.col), _p(g.ed2), cap,
                                _p(g.nnz_dev), _p(ws), ws.numel()), "vb_graph_build")
    return g


def bandwidth(nbr_d2: torch.Tensor, k_bw: int | None = None) -> torch.Tensor:
    n, k = nbr_d2.shape
    b = torch.empty(n, dtype=torch.float64, device=nbr_d2.device)
    _check(lib().vb_bandwidth(c_p(_ctx(nbr_d2.device)), n, k, k if k_bw is None else k_bw, _p(nbr_d2), _p(b)),
           "vb_bandwidth")
    return b


def epsilon_tune(g: Graph, rho: torch.Tensor, scale: float, xi_c: torch.Tensor | None = None,
                 grid=(XI_LO, XI_HI, DXI), warn_bit: int = 1):
    """One fused sweep over the grid (vb_epsilon_tune): returns (eps2 [1], chi [G], dim_est [1]) on the device."""
    dev = rho.device
    G = int(round((grid[1] - grid[0]) / grid[2])) + 1
    eps2 = torch.empty(1, dtype=torch.float64, device=dev)
    chi = torch.empty(G, dtype=torch.float64, device=dev)
    dim = torch.empty(1, dtype=torch.float64, device=dev)
    ws = _ws(lib().vb_epsilon_tune_workspace(g.n), dev)
    gc = g.c()
    _check(lib().vb_epsilon_tune(c_p(_ctx(dev)), ctypes.byref(gc), _p(rho), scale, _p(xi_c), grid[0], grid[1],
                                 grid[2], warn_bit, _p(eps2), _p(chi), _p(dim), _p(ws), ws.numel()), "vb_epsilon_tune")
    return eps2, chi, dim


def density(g: Graph, b: torch.Tensor, eps2: torch.Tensor, d: float, beta: float):
    dev = b.device
    psi = torch.empty(g.n, dtype=torch.float64, device=dev)
    P = torch.empty(g.n, dtype=torch.float64, device=dev)
    ws = _ws(lib().vb_density_workspace(g.n), dev)
    gc = g.c()
    _check(lib().vb_density(c_p(_ctx(dev)), ctypes.byref(gc), _p(b), _p(eps2), d, beta, _p(psi), _p(P), _p(ws),
                            ws.numel()), "vb_density")
    return psi, P


def operator_centre(g: Graph, b: torch.Tensor, P: torch.Tensor) -> torch.Tensor:
    dev = b.device
    xi_c = torch.empty(1, dtype=torch.float64, device=dev)
    ws = _ws(lib().vb_operator_centre_workspace(g.n), dev)
    gc = g.c()
    _check(lib().vb_operator_centre(c_p(_ctx(dev)), ctypes.byref(gc), _p(b), _p(P), _p(xi_c), _p(ws), ws.numel()),
           "vb_operator_centre")
    return xi_c


def kernel_csr(g: Graph, psi: torch.Tensor, P: torch.Tensor, eps2_op: torch.Tensor, c: float, beta: float, d: float):
    """K_{eps,beta}, normalisations and the CSR values of L-hat (vb_kernel_csr): returns (val, q, D, S)."""
    dev = psi.device
    val = torch.empty(g.col.numel(), dtype=torch.float32, device=dev)
    q, D, S = (torch.empty(g.n, dtype=torch.float64, device=dev) for _ in range(3))
    ws = _ws(lib().vb_kernel_csr_workspace(g.n), dev)
    gc = g.c()
    op = OpParams(c, beta, d)
    _check(lib().vb_kernel_csr(c_p(_ctx(dev)), ctypes.byref(gc), _p(psi), _p(P), ctypes.byref(op), _p(eps2_op),
                               _p(val), _p(q), _p(D), _p(S), _p(ws), ws.numel()), "vb_kernel_csr")
    return val, q, D, S


def tc_dot_tile(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Diagnostic tensor-core tile: a [128, K] @ b [N, K]^T with BF16 operands, FP32 result (vb_tc_dot_tile)."""
    K = a.shape[1]
    N = b.shape[0]
    d = torch.empty((128, N), dtype=torch.float32, device=a.device)
    _check(lib().vb_tc_dot_tile(c_p(_ctx(a.device)), _p(a), _p(b), K, N, _p(d)), "vb_tc_dot_tile")
    return d


def spmv(g: Graph, val: torch.Tensor, x: torch.Tensor, S: torch.Tensor | None = None, laplacian: bool = False,
         alpha: float = 1.0, beta: float = 0.0, y: torch.Tensor | None = None) -> torch.Tensor:
    """y = alpha A x + beta y (vb_spmv); laplacian=True applies L-hat in difference form with S."""
    dev = x.device
    if y is None:
        y = torch.zeros(g.n, dtype=torch.float32, device=dev)
    ws = _ws(lib().vb_spmv_workspace(g.n), dev) if laplacian else None
    gc = g.c()
    _check(lib().vb_spmv(c_p(_ctx(dev)), ctypes.byref(gc), _p(val), _p(S), VB_SPMV_LAPLACIAN if laplacian else
                         VB_SPMV_PLAIN, alpha, _p(x), beta, _p(y), _p(ws), 0 if ws is None else ws.numel()), "vb_spmv")
    return y


class Mlp:
    """The learned-radius network (vb_mlp): device parameters held in torch tensors, plus the
    host-side standardisation constants.  `handle()` is the address of the C struct."""

    def __init__(self, in_dim: int, device=None, seed: int = 1):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        P = int(lib().vb_mlp_param_count(in_dim))
        self.master = torch.empty(P, dtype=torch.float32, device=dev)
        self.weights = torch.empty(P, dtype=torch.int16, device=dev)   # BF16 bit patterns
        self.adam_m = torch.empty(P, dtype=torch.float32, device=dev)
        self.adam_v = torch.empty(P, dtype=torch.float32, device=dev)
        self.c = MlpC(in_dim, _p(self.master), _p(self.weights), _p(self.adam_m), _p(self.adam_v))
        for r in range(16):
            self.c.in_scale[r] = 1.0
        self.c.out_scale = 1.0
        _check(lib().vb_mlp_init(c_p(_ctx(dev)), ctypes.byref(self.c), seed), "vb_mlp_init")

    @property
    def param_count(self) -> int:
        return self.master.numel()

    def handle(self) -> int:
        return ctypes.addressof(self.c)

    def fit_standardisation(self, x: torch.Tensor, y: torch.Tensor) -> None:
        """Standardisation constants from the training data (vb_mlp_standardise)."""
        n, ld = x.shape
        ws = _ws(8 * 2 * 17, self.device)
        _check(lib().vb_mlp_standardise(c_p(_ctx(self.device)), ctypes.byref(self.c), _p(x), ld, _p(y), n, _p(ws),
                                        ws.numel()), "vb_mlp_standardise")

    def set_standardisation(self, in_mean, in_scale, out_mean: float, out_scale: float) -> None:
        for r in range(self.c.in_dim):
            self.c.in_mean[r] = float(in_mean[r])
            self.c.in_scale[r] = float(in_scale[r])
        self.c.out_mean = float(out_mean)
        self.c.out_scale = float(out_scale)

    def bf16_weights(self) -> torch.Tensor:
        """FP32 values of the BF16 weights the forward passes use."""
        return (self.weights.to(torch.int32) << 16).view(torch.float32)

    def train_epoch(self, x: torch.Tensor, y: torch.Tensor, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
        n, ld = x.shape
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        ws = _ws(lib().vb_mlp_workspace(self.c.in_dim, batch), self.device)
        _check(lib().vb_mlp_train_epoch(c_p(_ctx(self.device)), ctypes.byref(self.c), _p(x), ld, _p(y), n, batch, lr,
                                        seed, _p(loss), _p(ws), ws.numel()), "vb_mlp_train_epoch")
        return loss

    def gradient(self, x: torch.Tensor, y: torch.Tensor):
        n, ld = x.shape
        grad = torch.empty(self.param_count, dtype=torch.float32, device=self.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        ws = _ws(lib().vb_mlp_workspace(self.c.in_dim, n), self.device)
        _check(lib().vb_mlp_gradient(c_p(_ctx(self.device)), ctypes.byref(self.c), _p(x), ld, _p(y), n, _p(grad),
                                     _p(loss), _p(ws), ws.numel()), "vb_mlp_gradient")
        return grad, loss

    def predict(self, x: torch.Tensor, tensor_cores: bool = False) -> torch.Tensor:
        """Predicted log radius per row (vb_mlp_predict; vb_mlp_predict_tc, the tensor-core form the
        radius-first search uses, with tensor_cores=True)."""
        n, ld = x.shape
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        f = lib().vb_mlp_predict_tc if tensor_cores else lib().vb_mlp_predict
        _check(f(c_p(_ctx(self.device)), ctypes.byref(self.c), _p(x), ld, n, _p(y)), "vb_mlp_predict")
        return y


def train_radius_model(x: torch.Tensor, logr: torch.Tensor, epochs: int = 30, batch: int = 4096, lr: float = 3e-3,
                       seed: int = 103) -> Mlp:
    """Fits the learned-radius network to (x, log r_k) pairs on the GPU (vb_mlp_train_epoch)."""
    n, m = x.shape
    net = Mlp(min(m, 16), x.device, seed)
    net.fit_standardisation(x, logr)
    for ep in range(epochs):
        net.train_epoch(x, logr, batch=batch, lr=lr, seed=seed * 1000 + ep)
    return net


@dataclasses.dataclass
class Eigen:
    evals: torch.Tensor        # [ell + 1] FP64, descending (lambda_0 ~ 0 first)
    phi: torch.Tensor          # [ell + 1, n] FP32, <phi_i, phi_j>_S = delta_ij
    f: torch.Tensor | None     # [n] FP32 spectral solution of L f = g, when g was given
    iters: int
    converged: bool


def solve(g: Graph, val: torch.Tensor, S: torch.Tensor, ell: int, rhs: torch.Tensor | None = None,
          block: int = 0, degree: int = 0, max_iter: int = 0, tol: float = 0.0, seed: int = 1) -> Eigen:
    """Leading eigenpairs of L and, with rhs, the spectral solve of L f = g (vb_solve)."""
    dev = val.device
    p = SolveParams(ell, block, degree, max_iter, tol, seed)
    evals = torch.empty(ell + 1, dtype=torch.float64, device=dev)
    phi = torch.empty((ell + 1, g.n), dtype=torch.float32, device=dev)
    f = torch.empty(g.n, dtype=torch.float32, device=dev) if rhs is not None else None
    it = c_i32()
    ws = _ws(lib().vb_solve_workspace(g.n, val.numel(), ctypes.byref(p)), dev)
    gc = g.c()
    rc = lib().vb_solve(c_p(_ctx(dev)), ctypes.byref(gc), val.numel(), _p(val), _p(S), ctypes.byref(p), _p(evals),
                        _p(phi), _p(rhs), _p(f), ctypes.byref(it), _p(ws), ws.numel())
    if rc not in (0, -6):
        _check(rc, "vb_solve")
    return Eigen(evals, phi, f, int(it.value), rc == 0)


def gradient(evals: torch.Tensor, phi: torch.Tensor, S: torch.Tensor, u: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Derivatives of u along every coordinate from the eigenpairs of L (vb_gradient):
    returns grad [n, m] FP32 with grad[i, s] = du/dx_s at sample i."""
    n, m = x.shape
    ell = phi.shape[0] - 1
    grad = torch.empty((n, m), dtype=torch.float32, device=x.device)
    ws = _ws(lib().vb_gradient_workspace(n, ell, m), x.device)
    _check(lib().vb_gradient(c_p(_ctx(x.device)), n, ell, _p(evals), _p(phi), _p(S), _p(u), _p(x), m, _p(grad),
                             _p(ws), ws.numel()), "vb_gradient")
    return grad


@dataclasses.dataclass
class Build:
    nbr: torch.Tensor
    nbr_d2: torch.Tensor
    b: torch.Tensor
    graph: Graph
    eps2_den: torch.Tensor
    chi_den: torch.Tensor
    dim_den: torch.Tensor
    psi: torch.Tensor
    P: torch.Tensor
    xi_c: torch.Tensor
    eps2_op: torch.Tensor
    chi_op: torch.Tensor
    dim_op: torch.Tensor
    val: torch.Tensor
    q: torch.Tensor
    D: torch.Tensor
    S: torch.Tensor


class Builder:
    """Holds the output and workspace buffers of vb_build for one problem size, so
    repeated builds (and timing loops) allocate nothing.

    With cloud_ptr (B + 1 offsets of the rows of each point cloud) it runs the
    batched build vb_build_batch: every per-cloud scalar output then holds B
    values (chi: B x G) and the CSR is block-diagonal.  cloud_log_shift (B floats)
    adds a per-cloud term to a learned radius.  `radius` (n floats on the device,
    original order) runs the radius-first search with a given guess of every
    point's k-th neighbour distance instead of a learned one.  graph() records one
    build in a CUDA graph for replay."""

    def __init__(self, n: int, m: int, k: int, d: float, c: float, beta: float = -0.25, margin: int = 16,
                 k_bw: int | None = None, prune: bool = True, device=None, grid=(XI_LO, XI_HI, DXI),
                 mlp: "Mlp | None" = None, log_shift: float = 0.0, inflate: float = 0.0,
                 tensor_cores: str | None = None, cloud_ptr=None, cloud_log_shift=None,
                 radius: torch.Tensor | None = None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.n, self.m, self.k, self.device = n, m, k, dev
        self.mlp = mlp   # kept alive: the C parameters point at it
        self.radius = radius
        G = int(round((grid[1] - grid[0]) / grid[2])) + 1
        self.batched = cloud_ptr is not None
        if self.batched:
            cp = np.asarray(cloud_ptr, dtype=np.int64)
            if cp.ndim != 1 or len(cp) < 2 or cp[0] != 0 or cp[-1] != n or np.any(np.diff(cp) < k + 1):
                raise ValueError("cloud_ptr must rise from 0 to n with at least k + 1 points per cloud")
            self.B = len(cp) - 1
            self._cp_host = (c_i64 * len(cp))(*cp.tolist())
            self.cloud_ptr = torch.from_numpy(cp).to(dev)
        else:
            self.B = 1
        B = self.B
        self._shift = None
        if cloud_log_shift is not None:
            self._shift = torch.as_tensor(np.asarray(cloud_log_shift, dtype=np.float32)).to(dev).contiguous()
            if self._shift.numel() != B:
                raise ValueError("cloud_log_shift needs one value per cloud")
        if radius is not None and (radius.shape != (n,) or radius.dtype != torch.float32):
            raise ValueError("radius must be float32 [n] (a guess of every point's k-th neighbour distance)")
        mode = VB_PRUNE_LEARNED if (mlp is not None or radius is not None) else \
            (VB_PRUNE_EXACT if prune else VB_PRUNE_NONE)
        prec = {None: VB_PREC_FP32, "bf16": VB_PREC_BF16, "fp16": VB_PREC_FP16}[tensor_cores]
        self.params = BuildParams(KnnParams(k, margin, prec, mode, _p(radius),
                                            c_p(0) if mlp is None else c_p(mlp.handle()), inflate, log_shift,
                                            _p(self._shift)),
                                  0 if k_bw is None else k_bw, OpParams(c, beta, d), grid[0], grid[1], grid[2], 0)
        cap = n * (2 * k + 1)
        f64 = lambda s: torch.empty(s, dtype=torch.float64, device=dev)
        g = Graph(n, torch.empty(n + 1, dtype=torch.int64, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
                  torch.empty(cap, dtype=torch.float32, device=dev), torch.empty(1, dtype=torch.int64, device=dev))
        chi = (B, G) if self.batched else G
        self.out = Build(nbr=torch.empty((n, k), dtype=torch.int32, device=dev), nbr_d2=f64((n, k)), b=f64(n), graph=g,
                         eps2_den=f64(B), chi_den=f64(chi), dim_den=f64(B), psi=f64(n), P=f64(n), xi_c=f64(B),
                         eps2_op=f64(B), chi_op=f64(chi), dim_op=f64(B),
                         val=torch.empty(cap, dtype=torch.float32, device=dev), q=f64(n), D=f64(n), S=f64(n))
        o = self.out
        self.cout = BuildOut(_p(o.nbr), _p(o.nbr_d2), _p(o.b), _p(g.row_ptr), _p(g.col), _p(g.ed2), cap, _p(g.nnz_dev),
                             _p(o.eps2_den), _p(o.chi_den), _p(o.dim_den), _p(o.psi), _p(o.P), _p(o.xi_c),
                             _p(o.eps2_op), _p(o.chi_op), _p(o.dim_op), _p(o.val), _p(o.q), _p(o.D), _p(o.S))
        if self.batched:
            nbytes = lib().vb_build_batch_workspace(n, m, B, ctypes.byref(self.params))
        else:
            nbytes = lib().vb_build_workspace(n, m, ctypes.byref(self.params))
        self.ws = _ws(nbytes, dev)

    def __call__(self, x: torch.Tensor, eps2_den=None, eps2_op=None) -> Build:
        """One build of x; eps2_den / eps2_op (a float, or B values) pin both bandwidths."""
        if x.shape != (self.n, self.m) or x.dtype != torch.float32:
            raise ValueError("x must be float32 [n, m] matching the builder")
        pin = eps2_den is not None or eps2_op is not None
        if pin:
            if eps2_den is None or eps2_op is None:
                raise ValueError("pin both eps2_den and eps2_op")
            for dst, v in ((self.out.eps2_den, eps2_den), (self.out.eps2_op, eps2_op)):
                if isinstance(v, (int, float)):
                    dst.fill_(float(v))
                else:
                    dst.copy_(torch.as_tensor(np.asarray(v, dtype=np.float64)).reshape(dst.shape))
        self.params.pin_eps = 1 if pin else 0
        h = c_p(_ctx(self.device))
        if self.batched:
            rc = lib().vb_build_batch(h, _p(x), self.n, self.m, self._cp_host, _p(self.cloud_ptr), self.B,
                                      ctypes.byref(self.params), ctypes.byref(self.cout), _p(self.ws), self.ws.numel())
            _check(rc, "vb_build_batch")
        else:
            _check(lib().vb_build(h, _p(x), self.n, self.m, ctypes.byref(self.params), ctypes.byref(self.cout),
                                  _p(self.ws), self.ws.numel()), "vb_build")
        return self.out

    def autotune(self, x: torch.Tensor) -> dict:
        """Chooses the kNN launch shape (heap margin, seed window) for this builder by
        timing the candidates on x (vb_knn_autotune; cached per shape key), and keeps it
        for every later build.  Synchronises; not for use inside a timed region."""
        best = KnnParams()
        ms = c_f32()
        cp = _p(self.cloud_ptr) if self.batched else c_p(0)
        _check(lib().vb_knn_autotune(c_p(_ctx(self.device)), _p(x), self.n, self.m, cp, self.B,
                                     ctypes.byref(self.params.knn),
                                     _p(self.out.nbr), _p(self.out.nbr_d2), _p(self.ws), self.ws.numel(),
                                     ctypes.byref(best), ctypes.byref(ms)), "vb_knn_autotune")
        self.params.knn.margin = best.margin
        self.params.knn.seed_tiles = best.seed_tiles
        self.params.knn.tc_variant = best.tc_variant
        out = {"margin": best.margin, "seed_tiles": best.seed_tiles, "knn_ms": ms.value}
        if self.params.knn.precision != VB_PREC_FP32:
            out["tc_variant"] = {VB_TC_STAGED: "staged", VB_TC_PIPELINED: "pipelined"}.get(best.tc_variant, "auto")
        return out

    def graph(self, x: torch.Tensor) -> "torch.cuda.CUDAGraph":
        """Records one build of x (bandwidths tuned, not pinned) in a CUDA graph;
        g.replay() then reruns every launch of the build on x's current contents
        into the same output buffers.  One eager build runs first (it creates the
        library context and sets the kernels' attributes outside the capture)."""
        self(x)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            self(x)
        return g


def build(x: torch.Tensor, k: int, d: float, c: float, beta: float = -0.25, margin: int = 16,
          k_bw: int | None = None, prune: bool = True, eps2_den: float | None = None,
          eps2_op: float | None = None) -> Build:
    """The whole build, kNN to L-hat (vb_build), on x's device and current stream."""
    n, m = x.shape
    return Builder(n, m, k, d, c, beta, margin, k_bw, prune, x.device)(x, eps2_den, eps2_op)


@dataclasses.dataclass
class EvolveStep:
    x_next: torch.Tensor   # [n, m] FP32 samples after the step
    grad_f: torch.Tensor   # [n, m] FP32 grad f at the samples before the step
    f: torch.Tensor        # [n] FP32 solution of L_{1,psi} f = g - mean(g)
    build: Build           # the operator of the step
    converged: bool


def evolve_step(x: torch.Tensor, dt: float, sigma: torch.Tensor, W: torch.Tensor, g: torch.Tensor, k: int,
                ell: int, d: float, u: torch.Tensor | None = None, beta: float = -0.25, margin: int = 16,
                max_iter: int = 0) -> EvolveStep:
    """One explicit step of the particle evolution of Sec. 6 (vb_evolve_step): the build of
    L_{1,psi} on x, the spectral solve of L f = g - mean(g) with ell eigenpairs, grad f, and
    x + dt (u - grad f) + sqrt(dt) sigma W.  x, W, u: [n, m] FP32; sigma: [m, m] FP32; g: [n] FP32."""
    n, m = x.shape
    dev = x.device
    b = Builder(n, m, k, d=d, c=1.0, beta=beta, margin=margin, device=dev)
    p = EvolveParams(b.params, SolveParams(ell, 0, 0, max_iter, 0.0, 1), dt)
    f = torch.empty(n, dtype=torch.float32, device=dev)
    grad = torch.empty((n, m), dtype=torch.float32, device=dev)
    x_next = torch.empty((n, m), dtype=torch.float32, device=dev)
    ws = _ws(lib().vb_evolve_workspace(n, m, ctypes.byref(p)), dev)
    rc = lib().vb_evolve_step(c_p(_ctx(dev)), _p(x), n, m, ctypes.byref(p), _p(u), _p(sigma), _p(W), _p(g),
                              ctypes.byref(b.cout), _p(f), _p(grad), _p(x_next), _p(ws), ws.numel())
    if rc not in (0, -6):
        _check(rc, "vb_evolve_step")
    return EvolveStep(x_next, grad, f, b.out, rc == 0)


@dataclasses.dataclass
class RadiusPattern:
    """The delta_tol pattern (vb_radius_pattern): CSR with rows sorted by column."""
    n: int
    row_ptr: torch.Tensor   # [n + 1] int64
    col: torch.Tensor       # [nnz] int32
    d2: torch.Tensor        # [nnz] FP64 canonical squared distances
    nnz: int


def radius_pattern(x: torch.Tensor, rho: torch.Tensor, eps2: float, delta_tol: float, cap: int = 0) -> RadiusPattern:
    """Algorithm 1's pattern: every (i, j) with exp(-d2 / (eps^2 rho_i rho_j)) > delta_tol, evaluated as
    d2 / (eps^2 (rho_i rho_j)) < -log(delta_tol) (vb_radius_pattern).  cap: entries to allocate (0 = 32 per
    row to begin with); a pattern larger than cap is computed again with room for all of it."""
    n, m = x.shape
    dev = x.device
    cap = cap or 32 * n
    ws = _ws(lib().vb_radius_workspace(n, m), dev)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = torch.empty(1, dtype=torch.int64, device=dev)
    for _ in range(2):
        col = torch.empty(cap, dtype=torch.int32, device=dev)
        d2 = torch.empty(cap, dtype=torch.float64, device=dev)
        report_reset(dev)
        _check(lib().vb_radius_pattern(c_p(_ctx(dev)), _p(x), n, m, _p(rho), eps2, delta_tol, _p(row_ptr), _p(col),
                                       _p(d2), cap, _p(nnz), _p(ws), ws.numel()), "vb_radius_pattern")
        z = int(nnz.item())
        if z <= cap:
            raise_on_device_error(dev)
            return RadiusPattern(n, row_ptr, col[:z], d2[:z], z)
        cap = z
    raise VbError(-3, "vb_radius_pattern")


def radius_sweep(x: torch.Tensor, rho: torch.Tensor, scale: float, delta_tol: float, grid=(XI_LO, XI_HI, DXI)):
    """Eq. (bandwidth sensitivity) over the delta_tol pattern of every grid point (vb_radius_sweep):
    returns (chi [G], eps2 [1], dim_est [1]) on the device."""
    n, m = x.shape
    dev = x.device
    G = int(round((grid[1] - grid[0]) / grid[2])) + 1
    chi = torch.empty(G, dtype=torch.float64, device=dev)
    eps2 = torch.empty(1, dtype=torch.float64, device=dev)
    dim = torch.empty(1, dtype=torch.float64, device=dev)
    ws = _ws(lib().vb_radius_workspace(n, m), dev)
    _check(lib().vb_radius_sweep(c_p(_ctx(dev)), _p(x), n, m, _p(rho), scale, grid[0], grid[1], grid[2], delta_tol,
                                 _p(chi), _p(eps2), _p(dim), _p(ws), ws.numel()), "vb_radius_sweep")
    return chi, eps2, dim
