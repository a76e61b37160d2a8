"""Exact kNN for the oracle (TEST INFRASTRUCTURE ONLY; see oracle/__init__.py).

`knn` calls the plain C brute force in knn_bf.c (compiled by `build()` with
-ffp-contract=off, OpenMP over rows).  `knn_dense` is an independent numpy
brute force over the full distance matrix, used to pin the C code on small n.
`knn_large` returns the same lists at sizes where the brute force takes too
long: a library primitive (scipy's k-d tree, or FP64 matrix products and a
top-k) proposes candidates, the canonical distance ranks them, and rows whose
k-th distance is not certified against the candidates left out go to the brute
force.

Definition (Sec. 2.1, Eq. for b^2 and I(x, k)): the k nearest *other* samples,
ordered by the canonical FP64 squared distance, ties broken by smaller index.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_bf.c")
_LIB = os.path.join(_HERE, "_build", "libknn_bf.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile knn_bf.c into oracle/_build/libknn_bf.so (plain gcc, no contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_knn.restype = ctypes.c_int
            lib.oracle_knn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_knn_rows.restype = ctypes.c_int
            lib.oracle_knn_rows.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_pair_d2.restype = None
            lib.oracle_pair_d2.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_void_p]
            _lib = lib
    return _lib


def knn(x: np.ndarray, k: int, rows: tuple[int, int] | None = None):
    """Exact kNN of the FP32 points x [n, m] for rows [r0, r1) (all rows by default).
    Returns (nbr int32 [rows, k], nbr_d2 float64 [rows, k])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, m = x.shape
    r0, r1 = (0, n) if rows is None else rows
    nbr = np.empty((r1 - r0, k), dtype=np.int32)
    d2 = np.empty((r1 - r0, k), dtype=np.float64)
    rc = _load().oracle_knn(x.ctypes.data, n, m, k, r0, r1, nbr.ctypes.data, d2.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_knn: k={k} outside [1, n-1] for n={n}")
    return nbr, d2


def knn_rows(x: np.ndarray, k: int, rows: np.ndarray):
    """Exact kNN of the listed rows only (output row t is point rows[t])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n, m = x.shape
    nbr = np.empty((rows.shape[0], k), dtype=np.int32)
    d2 = np.empty((rows.shape[0], k), dtype=np.float64)
    rc = _load().oracle_knn_rows(x.ctypes.data, n, m, k, rows.ctypes.data, rows.shape[0], nbr.ctypes.data,
                                 d2.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_knn_rows: bad k or row index")
    return nbr, d2


def pair_d2(x: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Canonical FP64 squared distances of the pairs (a[t], b[t])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    out = np.empty(a.shape[0], dtype=np.float64)
    _load().oracle_pair_d2(x.ctypes.data, x.shape[1], a.ctypes.data, b.ctypes.data, a.shape[0], out.ctypes.data)
    return out


def dense_d2(x: np.ndarray) -> np.ndarray:
    """Full n x n matrix of canonical FP64 squared distances, in numpy: per
    coordinate an RN difference and square, summed in ascending coordinate order."""
    x64 = np.asarray(x, dtype=np.float32).astype(np.float64)
    acc = None
    for r in range(x64.shape[1]):
        dl = x64[:, None, r] - x64[None, :, r]
        s = dl * dl
        acc = s if acc is None else acc + s
    return acc


def knn_dense(x: np.ndarray, k: int):
    """Independent brute force for small n: lexicographic sort of every row of
    the dense distance matrix by (d2, j), self removed."""
    d2 = dense_d2(x)
    n = d2.shape[0]
    nbr = np.empty((n, k), dtype=np.int32)
    out = np.empty((n, k), dtype=np.float64)
    idx = np.arange(n)
    for i in range(n):
        mask = idx != i
        j = idx[mask]
        dj = d2[i, mask]
        order = np.lexsort((j, dj))[:k]
        nbr[i] = j[order]
        out[i] = dj[order]
    return nbr, out


def _certified_rows(x: np.ndarray, k: int, cand: np.ndarray, bound: np.ndarray):
    """Exact lists from candidate sets: the canonical FP64 distances of every row's
    candidates (cand [n, c], c > k, any order), sorted by (d2, j); a row is certified
    when its k-th canonical distance lies below `bound` (a lower bound on the canonical
    distance of every point outside its candidate set).  Rows that are not certified,
    or whose candidates include the point itself fewer or more than once, are
    recomputed by the brute force."""
    n = x.shape[0]
    rows = np.repeat(np.arange(n, dtype=np.int64), cand.shape[1])
    d2 = pair_d2(x, rows, cand.ravel().astype(np.int64)).reshape(cand.shape)
    own = cand == np.arange(n)[:, None]
    d2 = np.where(own, np.inf, d2)
    order = np.lexsort((cand, d2), axis=1)[:, :k]
    nbr = np.take_along_axis(cand, order, axis=1).astype(np.int32)
    out = np.take_along_axis(d2, order, axis=1)
    bad = (out[:, k - 1] >= bound) | (own.sum(axis=1) != 1)
    if bad.any():
        r = np.nonzero(bad)[0]
        nbr[r], out[r] = knn_rows(x, k, r)
    return nbr, out, int(bad.sum())


def knn_large(x: np.ndarray, k: int, margin: int = 16, block: int = 2048):
    """The same exact lists as knn() for large n, with library primitives choosing
    candidates and the canonical FP64 distance deciding:
      m <= 8: scipy's k-d tree (exact Euclidean k + margin + 1 nearest, self included);
      m > 8:  FP64 |x|^2 + |y|^2 - 2 x.y by matrix products over row blocks, then the
              k + margin + 1 smallest per row (torch.topk on the CPU).
    Every kept row's k-th canonical distance must lie below a lower bound on the
    canonical distance of every candidate left out (the (k + margin + 1)-th candidate's
    distance, less a bound on the candidate distance's rounding error); other rows go
    to the brute force.  Returns (nbr, nbr_d2, rows sent to the brute force)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, m = x.shape
    c = min(n, k + margin + 1)
    x64 = x.astype(np.float64)
    if m <= 8:
        from scipy.spatial import cKDTree
        dist, cand = cKDTree(x64).query(x64, c, workers=-1)
        # the tree's FP64 Euclidean distance is within a few ulps of the canonical one
        bound = (dist[:, -1] ** 2) * (1.0 - 1e-12)
        cand = cand[:, :-1] if c < n else cand
        return _certified_rows(x, k, cand.astype(np.int64), bound if c < n else np.full(n, np.inf))
    import torch
    X = torch.from_numpy(x64)
    XT = X.T.contiguous()
    sq = (X * X).sum(1)
    cand = np.empty((n, c), dtype=np.int64)
    bound = np.empty(n)
    # |y|^2 - 2 x.y ranks the candidates of row x like the squared distance; adding |x|^2
    # gives a value within (m + 2) 2^-52 (|x| + |y|)^2 of the exact squared distance, and
    # the canonical sum lies within m 2^-53 of that
    nrm = sq.sqrt()
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        D = torch.addmm(sq[None, :], X[r0:r1], XT, beta=1.0, alpha=-2.0)
        v, i = torch.topk(D, c, dim=1, largest=False, sorted=True)
        cand[r0:r1] = i.numpy()
        err = (m + 3) * 2.0 ** -52 * (nrm[r0:r1] + nrm.max()) ** 2
        bound[r0:r1] = (v[:, -1] + sq[r0:r1] - err).numpy() * (1.0 - 1e-12)
    if c == n:
        bound[:] = np.inf
    return _certified_rows(x, k, cand[:, :-1] if c < n else cand, bound)
