"""Seeded synthetic point clouds shaped like the workloads of Davis & Giannakis
(arXiv 2104.15124, Sec. 5): samples on the unit circle, on S^2 (uniform and
von Mises-Fisher), on a flat torus embedded in R^4, a low-dimensional Gaussian
embedded in R^100, batches of ellipsoids, and plain Gaussians in R^m.

This module only draws samples.  It holds none of the method's arithmetic and
is shared by the CUDA path's tests, the benchmark and the FP64 oracle's tests.
Every generator uses numpy's PCG64 in FP64 and returns FP32 row-major
coordinates (the canonical input layout), plus whatever generating
coordinates a closed-form check needs.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def circle(n: int, seed: int = 1) -> np.ndarray:
    """n points on the unit circle in R^2, angle uniform on [0, 2pi) (density 1/(2pi))."""
    th = 2.0 * np.pi * _rng(seed).random(n)
    return np.stack([np.cos(th), np.sin(th)], axis=1).astype(np.float32)


def sphere_uniform(n: int, seed: int = 2) -> np.ndarray:
    """n points uniform on S^2 in R^3 (density 1/(4pi), Sec. 5.2)."""
    g = _rng(seed).standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def sphere_vmf(n: int, kappa: float = 2.0, seed: int = 2) -> np.ndarray:
    """n points on S^2 from the von Mises-Fisher law with concentration kappa
    about +z (density proportional to exp(kappa z), Sec. 5.2).  The polar
    coordinate w = z is drawn by the exact inverse CDF, the azimuth uniformly."""
    r = _rng(seed)
    u = r.random(n)
    phi = 2.0 * np.pi * r.random(n)
    w = np.log(np.exp(-kappa) + u * (np.exp(kappa) - np.exp(-kappa))) / kappa
    w = np.clip(w, -1.0, 1.0)
    s = np.sqrt(1.0 - w * w)
    return np.stack([s * np.cos(phi), s * np.sin(phi), w], axis=1).astype(np.float32)


def torus4(n: int, sigma: float = 0.01, seed: int = 3) -> np.ndarray:
    """n points on the flat torus embedded in R^4 as (cos a, sin a, cos b, sin b),
    a, b uniform on [0, 2pi), plus isotropic Gaussian noise of std sigma."""
    r = _rng(seed)
    a = 2.0 * np.pi * r.random(n)
    b = 2.0 * np.pi * r.random(n)
    x = np.stack([np.cos(a), np.sin(a), np.cos(b), np.sin(b)], axis=1)
    if sigma > 0:
        x = x + sigma * r.standard_normal((n, 4))
    return x.astype(np.float32)


@dataclasses.dataclass
class Embedded:
    x: np.ndarray      # FP32 [n, m] ambient samples
    z: np.ndarray      # FP64 [n, d] generating coordinates
    A: np.ndarray      # FP64 [m, d] orthonormal embedding


def gauss_embedded(n: int, d: int = 5, m: int = 100, sigma: float = 1e-3, seed: int = 4) -> Embedded:
    """z ~ N(0, I_d) mapped into R^m by a seeded orthonormal m x d matrix A
    (QR of a Gaussian matrix with diag(R) > 0), plus N(0, sigma^2 I_m) noise."""
    r = _rng(seed)
    q, rr = np.linalg.qr(r.standard_normal((m, d)))
    q = q * np.sign(np.diag(rr))[None, :]
    z = r.standard_normal((n, d))
    x = z @ q.T + sigma * r.standard_normal((n, m))
    return Embedded(x=x.astype(np.float32), z=z, A=q)


def gaussian(n: int, m: int = 2, scales=None, seed: int = 6) -> np.ndarray:
    """n samples of N(0, diag(scales)) in R^m (Sec. 5.1 uses covariance I in R^2
    and diag(sqrt2, sqrt2, sqrt3, sqrt3) in R^4); `scales` are variances."""
    v = np.ones(m) if scales is None else np.asarray(scales, dtype=np.float64)
    return (_rng(seed).standard_normal((n, m)) * np.sqrt(v)[None, :]).astype(np.float32)


@dataclasses.dataclass
class Batch:
    x: np.ndarray          # FP32 [N, 3] all clouds, concatenated
    cloud_ptr: np.ndarray  # int64 [B+1] offsets of each cloud in x
    axes: np.ndarray       # FP64 [B, 3] semi-axes


def ellipsoids(n_clouds: int = 256, n_lo: int = 2000, n_hi: int = 40000, seed: int = 5) -> Batch:
    """A batch of point clouds on ellipsoids in R^3 with semi-axes U[0.5, 2],
    each with n_b ~ U[n_lo, n_hi] points sampled uniformly in the polar and
    azimuthal angles (so non-uniformly on the surface)."""
    r = _rng(seed)
    sizes = np.floor(r.uniform(n_lo, n_hi + 1, n_clouds)).astype(np.int64)
    axes = r.uniform(0.5, 2.0, (n_clouds, 3))
    xs = []
    for b in range(n_clouds):
        th = np.pi * r.random(sizes[b])
        ph = 2.0 * np.pi * r.random(sizes[b])
        a = axes[b]
        xs.append(np.stack([a[0] * np.sin(th) * np.cos(ph), a[1] * np.sin(th) * np.sin(ph),
                            a[2] * np.cos(th)], axis=1))
    ptr = np.zeros(n_clouds + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(sizes)
    return Batch(x=np.concatenate(xs).astype(np.float32), cloud_ptr=ptr, axes=axes)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named synthetic workload and the method parameters it is run with."""
    name: str
    n: int
    m: int
    k: int          # neighbours per point (also the bandwidth's k_nn)
    d: int          # intrinsic dimension used by the normalisations
    c: float        # Kolmogorov operator parameter
    beta: float = -0.25
    margin: int = 16
    seed: int = 1

    def sample(self, n: int | None = None) -> np.ndarray:
        n = self.n if n is None else n
        if self.name.startswith("circle"):
            return circle(n, self.seed)
        if self.name.startswith("vmf"):
            return sphere_vmf(n, 2.0, self.seed)
        if self.name.startswith("sphere"):
            return sphere_uniform(n, self.seed)
        if self.name.startswith("torus"):
            return torus4(n, 0.01, self.seed)
        if self.name.startswith("gauss100"):
            return gauss_embedded(n, 5, 100, 1e-3, self.seed).x
        if self.name.startswith("gauss"):
            return gaussian(n, self.m, None, self.seed)
        raise KeyError(self.name)


# The five workloads the hot path is measured and checked on.
CIRCLE_2K = Workload("circle_2k", 2000, 2, 32, 1, 0.0, seed=1)
VMF_50K = Workload("vmf_s2_50k", 50000, 3, 64, 2, 1.0, seed=2)
TORUS_1M = Workload("torus_r4_1m", 1000000, 4, 64, 2, 1.0, seed=3)
GAUSS100_200K = Workload("gauss100_200k", 200000, 100, 128, 5, 1.0, seed=4)
ELLIPSOIDS_5M = "ellipsoids_256"   # batched; see ellipsoids()

WORKLOADS = {w.name: w for w in (CIRCLE_2K, VMF_50K, TORUS_1M, GAUSS100_200K)}
