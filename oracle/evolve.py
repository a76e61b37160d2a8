"""Particle evolution of a time-dependent density in plain FP64 (TEST INFRASTRUCTURE
ONLY; see oracle/__init__.py).

Sec. 6, "Evolution of a time-dependent density": samples x_t of psi(.; t) follow the SDE
dX = (u - grad f) dt + sigma dW (Eq. (SDE)), where f solves the Kolmogorov problem
L_{1,psi} f = g with E_psi f = 0 (Eq. (advection-diffusion-Laplace)) on the current samples.
One explicit step (Eq. (discrete sample evolution)):

    x_{t+dt} = x_t + dt (u - grad f) + sqrt(dt) sigma W,   W ~ N(0, I).

Each step therefore runs the whole method of this package on the current samples:
  1. the operator of Sec. 2 with c = 1 (L_{1,psi}: alpha from c = 2 - 2 alpha + d beta + 2 beta);
  2. its leading eigenpairs and the spectral solve of Sec. 3.1 (the constant mode dropped,
     so E_psi f = 0 in the S-weighted sense);
  3. grad f at every sample by the gradient representation of Sec. 3.2 with v = x_s;
  4. the update above.  The Gaussian increments W are inputs (the caller draws them), so
     the step is a deterministic function of its arguments.

Readings of the paper this module takes:
  R14 g is centred on the samples, g - mean(g) (the paper's g = g' - g-bar with the sample
      mean for the expectation under psi(.; t)).
  R15 the kernel's diagonal scales the eigenvalues by (1 - self weight); the solve divides
      by them and the gradient multiplies by them, so grad f needs no correction.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import method as M


@dataclasses.dataclass
class Step:
    x_next: np.ndarray     # [n, m] samples after the step
    grad_f: np.ndarray     # [n, m] grad f at the samples (before the step)
    f: np.ndarray          # [n] the solution of L_{1,psi} f = g
    g: np.ndarray          # [n] the centred right-hand side (R14)


def gradient_of_solution(x: np.ndarray, g: np.ndarray, k: int, ell: int, d: float,
                         beta: float = -0.25) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Steps 1-3: f with L_{1,psi} f = g - mean(g) over ell eigenpairs, and grad f [n, m]."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, m = x.shape
    gc = np.asarray(g, dtype=np.float64) - float(np.mean(g))           # R14
    B = M.build(x, k, d=d, c=1.0, beta=beta)                          # L_{1,psi}
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, ell)
    f = M.spectral_solve(e, B.op.S, gc)
    xs = x.astype(np.float64)
    grad = np.stack([M.gradient_dot(e, B.op.S, f, xs[:, s]) for s in range(m)], axis=1)
    return f, grad, gc


def evolve_step(x: np.ndarray, dt: float, sigma: np.ndarray, W: np.ndarray, g: np.ndarray, k: int, ell: int,
                d: float, u: np.ndarray | None = None, beta: float = -0.25) -> Step:
    """Eq. (discrete sample evolution) for one step of length dt: u [n, m] the prescribed
    velocity at the samples (0 if None), sigma [m, m], W [n, m] standard normal draws,
    g [n] the source at the samples."""
    x64 = np.asarray(x, dtype=np.float64)
    f, grad, gc = gradient_of_solution(x, g, k, ell, d, beta)
    drift = -grad if u is None else np.asarray(u, dtype=np.float64) - grad
    x_next = x64 + dt * drift + np.sqrt(dt) * (np.asarray(W, dtype=np.float64) @ np.asarray(sigma, dtype=np.float64).T)
    return Step(x_next=x_next, grad_f=grad, f=f, g=gc)
