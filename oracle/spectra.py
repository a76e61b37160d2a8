"""Continuum reference spectra for the closed-form checks (TEST INFRASTRUCTURE ONLY;
see oracle/__init__.py).

The operator is the paper's Kolmogorov operator L_{psi,c} f = Delta f + c grad f . grad psi / psi
(Sec. 2, Eq. Kolmogorov).  On the unit sphere S^2 with the von Mises-Fisher density
psi ~ exp(kappa z) about +z (Sec. 5.2) the drift is c kappa grad z, and in the polar
coordinate z = cos(theta) with f = g(z) e^{i m phi} it separates into one weighted
Sturm-Liouville problem per azimuthal order m:

    (e^{c kappa z} (1 - z^2) g')' / e^{c kappa z} - m^2 g / (1 - z^2) = lambda g,

symmetric in the weight e^{c kappa z} (the psi^c weight under which Sec. 2 states that
L_{psi,c} is symmetric).  Every order m >= 1 appears twice (cos and sin of m phi).
With kappa = 0 it is the spherical Laplacian, lambda = -l(l+1) with multiplicity 2l + 1.

Two independent discretisations:
  sphere_drift_spectrum   Galerkin in the basis (1 - z^2)^{m/2} P_a(z) (Legendre P_a),
                          Gauss-Legendre quadrature of the weak form;
  sphere_drift_spectrum_fd second-order finite volumes in theta on the flux form
                          (w sin(theta) f')' / (w sin(theta)) - m^2 f / sin^2(theta),
                          w = e^{c kappa cos(theta)}.
The tests pin the Galerkin solver to -l(l+1) at kappa = 0 and to the finite-volume
solver at kappa = 2.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from numpy.polynomial import legendre as npleg


def _sector_galerkin(m: int, drift: float, nbasis: int, nquad: int) -> np.ndarray:
    """Eigenvalues of the order-m problem with drift coefficient `drift` = c kappa."""
    z, wq = npleg.leggauss(nquad)
    w = wq * np.exp(drift * z)
    one_m = 1.0 - z * z
    P = np.empty((nbasis, nquad))
    dP = np.empty((nbasis, nquad))
    for a in range(nbasis):
        e = np.zeros(a + 1)
        e[a] = 1.0
        P[a] = npleg.legval(z, e)
        dP[a] = npleg.legval(z, npleg.legder(e)) if a > 0 else 0.0
    if m == 0:
        # g = P_a: stiffness (1 - z^2) g_a' g_b', mass g_a g_b
        A = (dP * (w * one_m)) @ dP.T
        B = (P * w) @ P.T
    else:
        # g = (1 - z^2)^{m/2} P_a, g' = (1 - z^2)^{m/2 - 1} ((1 - z^2) P_a' - m z P_a):
        # (1 - z^2) g_a' g_b' and m^2 g_a g_b / (1 - z^2) both carry (1 - z^2)^{m-1}
        Q = one_m * dP - m * z * P
        A = (Q * (w * one_m ** (m - 1))) @ Q.T + m * m * ((P * (w * one_m ** (m - 1))) @ P.T)
        B = (P * (w * one_m ** m)) @ P.T
    lam = sla.eigh(-A, B, eigvals_only=True)
    return np.sort(lam)[::-1]


def sphere_drift_spectrum(kappa: float, c: float = 1.0, count: int = 32, mmax: int | None = None,
                          nbasis: int = 40, nquad: int = 160) -> np.ndarray:
    """The `count` largest eigenvalues (0 first, descending, with multiplicity) of
    L_{psi,c} on S^2 for psi ~ exp(kappa z), by Galerkin per azimuthal order."""
    mmax = int(np.ceil(np.sqrt(count))) + 2 if mmax is None else mmax
    out = []
    for m in range(mmax + 1):
        lam = _sector_galerkin(m, c * kappa, nbasis, nquad)
        out.extend(lam.tolist() * (1 if m == 0 else 2))
    out = np.sort(np.array(out))[::-1]
    return out[:count]


def _sector_fd(m: int, drift: float, ncell: int) -> np.ndarray:
    h = np.pi / ncell
    th = (np.arange(ncell) + 0.5) * h
    thf = np.arange(1, ncell) * h                       # interior faces
    wf = np.exp(drift * np.cos(thf)) * np.sin(thf) / h  # face conductances (w sin theta / h)
    wc = np.exp(drift * np.cos(th)) * np.sin(th) * h    # cell masses (w sin theta h)
    diag = np.zeros(ncell)
    diag[:-1] -= wf
    diag[1:] -= wf
    diag -= m * m * wc / np.sin(th) ** 2
    # symmetric tridiagonal pencil (A, diag(wc)) -> scale to a standard problem
    s = 1.0 / np.sqrt(wc)
    d = diag * s * s
    e = wf * s[:-1] * s[1:]
    lam = sla.eigh_tridiagonal(d, e, eigvals_only=True, select="i", select_range=(ncell - 12, ncell - 1))
    return np.sort(lam)[::-1]


def sphere_drift_spectrum_fd(kappa: float, c: float = 1.0, count: int = 32, mmax: int | None = None,
                             ncell: int = 4000) -> np.ndarray:
    """The same spectrum from finite volumes in theta (independent of the Galerkin code)."""
    mmax = int(np.ceil(np.sqrt(count))) + 2 if mmax is None else mmax
    out = []
    for m in range(mmax + 1):
        lam = _sector_fd(m, c * kappa, ncell)
        out.extend(lam.tolist() * (1 if m == 0 else 2))
    out = np.sort(np.array(out))[::-1]
    return out[:count]
