"""The variable-bandwidth kernel method in plain FP64 (TEST INFRASTRUCTURE ONLY;
see oracle/__init__.py).

Follows Davis & Giannakis (arXiv 2104.15124), Sec. 2 and Sec. 4, in the
paper's order and notation:

  b          bandwidth function, Eq. (bandwidth parameter), Sec. 2.1
  K_eps      density kernel matrix, Eq. (density kernel matrix)
  w, psi     KDE normalisation w = n (pi eps^2 b^2)^(d/2), psi = W^-1 K_eps 1
  K_eps,beta operator kernel, Eq. (variable-bandwidth kernel matrix), Sec. 2.2
  q, K~, D   q_{eps,beta} = psi^(-beta d) K 1, K~ = K / (q q^T)^alpha, D = K~ 1
  L, L-hat   L = eps^-2 P^-2 (D^-1 K~ - I), L-hat = eps^-2 (S^-1 K~ S^-1 - P^-2),
             S = P D^(1/2), P = psi^beta, c = 2 - 2 alpha + d beta + 2 beta
  chi, chi'  bandwidth sweep, eps_xi^2 = 2^xi, Eq. (bandwidth sensitivity), Sec. 2.3
  solve      f~ = Lambda^-1 g~, g~ = Q^T S^2 g / n, f = Q f~, Eqs. (LS minimiser, f_LS), Sec. 3.1
  gradient   grad u . grad v from the eigenpairs and C-hat_ljk = <phi_l, phi_j * phi_k>_S, Sec. 3.2

Readings where the paper is silent or ambiguous:
  R1 sparsity: the matrix lives on E = diagonal U kNN U kNN^T (no delta_tol drop).
  R2 self is excluded from the kNN lists and from b; k_bw = k unless given.
  R3 the diagonal (j = i) is part of every kernel sum, as in Algorithm 1 (j from i).
  R4 eps^2 = 2^xi on the grid xi = -10, -9.75, ..., 4 (57 points, delta = 0.25);
     eps is the left end of the forward difference; ties go to the smaller xi.
  R5 d-hat = 2 max chi'; the caller's d is used in w, q and alpha.
  R6 the operator kernel uses 4 eps^2 (P_i P_j) (rho = 2 psi^beta in Algorithm 1).
  R9 the operator sweep is centred at xi_c = round_quarter(log2(sum_E' t_op / sum_E' t_den)),
     t_den = d2 / (b_i b_j), t_op = d2 / (4 P_i P_j), E' = off-diagonal entries.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from . import knn as _knn

XI_LO, XI_HI, DXI = -10.0, 4.0, 0.25


def xi_grid(lo: float = XI_LO, hi: float = XI_HI, step: float = DXI) -> np.ndarray:
    """The sweep grid xi_g = lo + g * step, g = 0 .. (hi - lo) / step (R4)."""
    g = int(round((hi - lo) / step))
    return lo + step * np.arange(g + 1, dtype=np.float64)


def alpha_from(c: float, d: float, beta: float) -> float:
    """Sec. 2.2: the operator approximates L_{psi,c} with c = 2 - 2 alpha + d beta + 2 beta."""
    return (2.0 - c + d * beta + 2.0 * beta) / 2.0


# --------------------------------------------------------------------------- kNN, bandwidth, pattern

def bandwidth(nbr_d2: np.ndarray, k_bw: int) -> np.ndarray:
    """Eq. (bandwidth parameter): b^2(x_i) = sum_{r=1}^{k_bw} ||x_i - x_I(i,r)||^2,
    summed in rank order (nearest first); returns b (not b^2)."""
    b2 = nbr_d2[:, 0].astype(np.float64).copy()
    for r in range(1, k_bw):
        b2 = b2 + nbr_d2[:, r]
    return np.sqrt(b2)


@dataclasses.dataclass
class Pattern:
    """Sparse symmetric pattern E in CSR form: rows sorted by column, diagonal stored."""
    n: int
    row_ptr: np.ndarray   # int64 [n+1]
    col: np.ndarray       # int64 [nnz]
    row: np.ndarray       # int64 [nnz] (row of every entry)
    d2: np.ndarray        # float64 [nnz] canonical squared distances

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def offdiag(self) -> np.ndarray:
        return self.row != self.col


def sym_pattern(x: np.ndarray, nbr: np.ndarray) -> Pattern:
    """R1: E = {(i, i)} U {(i, j): j in N_k(i) or i in N_k(j)}, the entries a
    symmetric kernel matrix (K^ij = K^ji, Algorithm 1) keeps when every kNN
    pair is kept."""
    n, k = nbr.shape
    ar = np.arange(n, dtype=np.int64)
    own_r = np.repeat(ar, k)
    own_c = nbr.astype(np.int64).ravel()
    rows = np.concatenate([ar, own_r, own_c])
    cols = np.concatenate([ar, own_c, own_r])
    key = np.unique(rows * n + cols)
    row = key // n
    col = key % n
    row_ptr = np.searchsorted(row, np.arange(n + 1, dtype=np.int64)).astype(np.int64)
    d2 = _knn.pair_d2(x, row, col)
    return Pattern(n=n, row_ptr=row_ptr, col=col, row=row, d2=d2)


def full_pattern(x: np.ndarray) -> Pattern:
    """Every pair (i, j), for the dense all-pairs pin (Algorithm 1 with delta_tol = 0)."""
    n = x.shape[0]
    row = np.repeat(np.arange(n, dtype=np.int64), n)
    col = np.tile(np.arange(n, dtype=np.int64), n)
    row_ptr = np.arange(n + 1, dtype=np.int64) * n
    return Pattern(n=n, row_ptr=row_ptr, col=col, row=row, d2=_knn.pair_d2(x, row, col))


def row_sum(p: Pattern, v: np.ndarray) -> np.ndarray:
    return np.bincount(p.row, weights=v, minlength=p.n)


# --------------------------------------------------------------------------- bandwidth sweep (Sec. 2.3)

@dataclasses.dataclass
class Sweep:
    xi: np.ndarray        # grid xi_g (absolute, centre included)
    chi: np.ndarray       # chi_g
    chi_prime: np.ndarray # forward differences, length G - 1
    g_star: int
    eps2: float
    dim_est: float
    at_boundary: bool


def sweep(p: Pattern, rho: np.ndarray, scale: float, xi: np.ndarray) -> Sweep:
    """Eq. (bandwidth sensitivity): chi_xi = sum_ij exp(-d2_ij / (scale 2^xi rho_i rho_j)),
    chi'_xi = (log chi_{xi+delta} - log chi_xi) / (delta log 2), maximised over the grid.
    scale = 1, rho = b gives the density sweep; scale = 4, rho = P the operator sweep (R6)."""
    import torch
    t = torch.from_numpy(p.d2 / (scale * rho[p.row] * rho[p.col]))
    # one FP64 sum per grid point; torch's CPU ops spread the exponentials over the host cores
    chi = np.array([float(torch.exp(-t / 2.0 ** float(xg)).sum()) for xg in xi])
    delta = xi[1] - xi[0]
    chip = (np.log(chi[1:]) - np.log(chi[:-1])) / (delta * math.log(2.0))
    g = int(np.argmax(chip))
    return Sweep(xi=xi, chi=chi, chi_prime=chip, g_star=g, eps2=float(2.0 ** xi[g]),
                 dim_est=float(2.0 * chip[g]), at_boundary=(g == 0 or g == len(chip) - 1))


def operator_centre(p: Pattern, b: np.ndarray, P: np.ndarray) -> float:
    """R9: xi_c = round(4 log2(sum_E' d2/(4 P_i P_j) / sum_E' d2/(b_i b_j))) / 4."""
    off = p.offdiag
    r, c, d2 = p.row[off], p.col[off], p.d2[off]
    s_op = np.sum(d2 / (4.0 * P[r] * P[c]))
    s_den = np.sum(d2 / (b[r] * b[c]))
    return math.floor(4.0 * math.log2(s_op / s_den) + 0.5) / 4.0


# --------------------------------------------------------------------------- density and operator (Sec. 2.1-2.2)

def density(p: Pattern, b: np.ndarray, eps2: float, d: float) -> np.ndarray:
    """Eq. (density estimation): psi = W^-1 K_eps 1, K_eps^ij = exp(-d2/(eps^2 b_i b_j)),
    W_ii = n (pi eps^2 b_i^2)^(d/2)."""
    K = np.exp(-p.d2 / (eps2 * b[p.row] * b[p.col]))
    w = p.n * (math.pi * eps2 * b * b) ** (d / 2.0)
    return row_sum(p, K) / w


@dataclasses.dataclass
class Operator:
    eps2: float
    K: np.ndarray       # K_{eps,beta} on the pattern
    q: np.ndarray       # q_{eps,beta}
    Kt: np.ndarray      # K_{eps,beta,alpha} on the pattern
    D: np.ndarray       # q_{eps,beta,alpha} (diagonal of D)
    P: np.ndarray
    S: np.ndarray
    Lhat: np.ndarray    # L-hat on the pattern
    L: np.ndarray       # L on the pattern (not symmetric)


def operator(p: Pattern, psi: np.ndarray, eps2: float, d: float, c: float, beta: float) -> Operator:
    """Sec. 2.2 in order: K_{eps,beta}, q_{eps,beta}, K~ (alpha normalisation),
    D, P, S = P D^(1/2), then L = eps^-2 P^-2 (D^-1 K~ - I) and the symmetric
    L-hat = eps^-2 (S^-1 K~ S^-1 - P^-2)."""
    alpha = alpha_from(c, d, beta)
    r, col = p.row, p.col
    K = np.exp(-p.d2 / (4.0 * eps2 * (psi[r] * psi[col]) ** beta))
    q = psi ** (-beta * d) * row_sum(p, K)
    Kt = K / (q[r] * q[col]) ** alpha
    D = row_sum(p, Kt)
    P = psi ** beta
    S = P * np.sqrt(D)
    diag = (r == col).astype(np.float64)
    Lhat = (Kt / (S[r] * S[col]) - diag / P[r] ** 2) / eps2
    L = (Kt / D[r] - diag) / (eps2 * P[r] ** 2)
    return Operator(eps2=eps2, K=K, q=q, Kt=Kt, D=D, P=P, S=S, Lhat=Lhat, L=L)


# --------------------------------------------------------------------------- the whole build (Sec. 4 steps 1-3)

@dataclasses.dataclass
class Build:
    x: np.ndarray
    k: int
    k_bw: int
    d: float
    c: float
    beta: float
    nbr: np.ndarray
    nbr_d2: np.ndarray
    b: np.ndarray
    pattern: Pattern
    den: Sweep
    psi: np.ndarray
    P: np.ndarray
    xi_c: float
    op_sweep: Sweep
    op: Operator

    def lhat_csr(self) -> sp.csr_matrix:
        p = self.pattern
        return sp.csr_matrix((self.op.Lhat, p.col, p.row_ptr), shape=(p.n, p.n))


def build(x: np.ndarray, k: int, d: float, c: float, beta: float = -0.25, k_bw: int | None = None,
          eps2_den: float | None = None, eps2_op: float | None = None, nbr=None, nbr_d2=None,
          pattern: Pattern | None = None) -> Build:
    """Sec. 4, steps 1-3 up to L-hat: kNN, b, density sweep, psi, operator sweep,
    K_{eps,beta}, normalisations, L-hat.  eps2_den / eps2_op pin the bandwidths
    instead of tuning them; nbr / pattern may be passed to skip those steps."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    k_bw = k if k_bw is None else k_bw
    if nbr is None:
        nbr, nbr_d2 = _knn.knn(x, k)
    b = bandwidth(nbr_d2, k_bw)
    if np.any(b == 0):
        raise ValueError("bandwidth b_i = 0: more than k_bw duplicates of a point")
    p = sym_pattern(x, nbr) if pattern is None else pattern
    grid = xi_grid()
    den = sweep(p, b, 1.0, grid)
    e_den = den.eps2 if eps2_den is None else eps2_den
    psi = density(p, b, e_den, d)
    P = psi ** beta
    xi_c = operator_centre(p, b, P)
    ops = sweep(p, P, 4.0, grid + xi_c)
    e_op = ops.eps2 if eps2_op is None else eps2_op
    op = operator(p, psi, e_op, d, c, beta)
    return Build(x=x, k=k, k_bw=k_bw, d=d, c=c, beta=beta, nbr=nbr, nbr_d2=nbr_d2, b=b, pattern=p,
                 den=den, psi=psi, P=P, xi_c=xi_c, op_sweep=ops, op=op)


# --------------------------------------------------------------------------- dense all-pairs form (pin)

def dense_all_pairs(x: np.ndarray, k_bw: int, d: float, c: float, beta: float = -0.25,
                    eps2_den: float | None = None, eps2_op: float | None = None) -> dict:
    """Algorithm 1 with delta_tol = 0 (every pair kept) and the Sec. 2 formulas as
    dense n x n matrix algebra.  Squared distances come from the expansion
    |x|^2 + |y|^2 - 2 x.y in FP64 (clipped at 0), not from the canonical
    per-coordinate form, and b from a full row sort, so this shares no step
    with the sparse path beyond the formulas themselves."""
    X = np.asarray(x, dtype=np.float32).astype(np.float64)
    n = X.shape[0]
    sq = np.sum(X * X, axis=1)
    D2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * X @ X.T, 0.0)
    np.fill_diagonal(D2, 0.0)
    srt = np.sort(D2 + np.diag(np.full(n, np.inf)), axis=1)
    b = np.sqrt(np.sum(srt[:, :k_bw], axis=1))
    grid = xi_grid()

    def tune(arg):  # arg(eps2) -> kernel matrix
        chi = np.array([arg(2.0 ** g).sum() for g in grid])
        chip = np.diff(np.log(chi)) / (DXI * math.log(2.0))
        gs = int(np.argmax(chip))
        return chi, chip, gs

    Kden = lambda e2: np.exp(-D2 / (e2 * np.outer(b, b)))
    chi_d, chip_d, g_d = tune(Kden)
    e_den = 2.0 ** grid[g_d] if eps2_den is None else eps2_den
    W = n * (math.pi * e_den * b ** 2) ** (d / 2.0)
    psi = Kden(e_den) @ np.ones(n) / W
    P = psi ** beta
    off = ~np.eye(n, dtype=bool)
    xi_c = math.floor(4.0 * math.log2(np.sum((D2 / (4.0 * np.outer(P, P)))[off]) /
                                      np.sum((D2 / np.outer(b, b))[off])) + 0.5) / 4.0
    Kop = lambda e2: np.exp(-D2 / (4.0 * e2 * np.outer(psi, psi) ** beta))
    chi_o, chip_o, g_o = (None, None, None)
    chi = np.array([Kop(2.0 ** (xi_c + g)).sum() for g in grid])
    chip_o = np.diff(np.log(chi)) / (DXI * math.log(2.0))
    g_o = int(np.argmax(chip_o))
    e_op = 2.0 ** (xi_c + grid[g_o]) if eps2_op is None else eps2_op
    alpha = alpha_from(c, d, beta)
    K = Kop(e_op)
    q = psi ** (-beta * d) * K.sum(axis=1)
    Kt = K / np.outer(q, q) ** alpha
    Dv = Kt.sum(axis=1)
    S = P * np.sqrt(Dv)
    Lhat = (np.diag(1 / S) @ Kt @ np.diag(1 / S) - np.diag(P ** -2.0)) / e_op
    L = np.diag(P ** -2.0) @ (np.diag(1 / Dv) @ Kt - np.eye(n)) / e_op
    return dict(D2=D2, b=b, chi_den=chi_d, g_den=g_d, eps2_den=e_den, psi=psi, P=P, xi_c=xi_c,
                chi_op=chi, g_op=g_o, eps2_op=e_op, K=K, q=q, Kt=Kt, D=Dv, S=S, Lhat=Lhat, L=L)


# --------------------------------------------------------------------------- eigenpairs and the solve (Sec. 3.1, Sec. 4 step 3-4)

@dataclasses.dataclass
class Eigen:
    evals: np.ndarray     # ell + 1 leading eigenvalues, descending (lambda_0 ~ 0 first)
    phi_hat: np.ndarray   # [n, ell+1] eigenvectors of L-hat, phi_hat^T phi_hat = n
    phi: np.ndarray       # [n, ell+1] eigenvectors of L, phi = S^-1 phi_hat


def leading_eigenpairs(Lhat: sp.spmatrix, S: np.ndarray, ell: int, dense_max: int = 5000) -> Eigen:
    """Sec. 2.2 / Sec. 4 step 3: the ell + 1 largest (algebraic) eigenpairs of the
    symmetric L-hat, normalised to phi_hat^T phi_hat = n, mapped to L by S^-1.
    Dense symmetric solver up to dense_max points, else shift-invert Lanczos."""
    n = Lhat.shape[0]
    if n <= dense_max:
        w, v = np.linalg.eigh(Lhat.toarray())
        w, v = w[::-1][: ell + 1], v[:, ::-1][:, : ell + 1]
    else:
        import scipy.sparse.linalg as sla
        sigma = 1e-3 * abs(Lhat.diagonal().min())
        w, v = sla.eigsh(Lhat.tocsc(), k=ell + 1, sigma=sigma, which="LM", tol=1e-12)
        o = np.argsort(w)[::-1]
        w, v = w[o], v[:, o]
    v = v * math.sqrt(n)
    return Eigen(evals=w, phi_hat=v, phi=v / S[:, None])


def spectral_solve(e: Eigen, S: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Eqs. (LS minimiser) and (f_LS): g~ = Q^T S^2 g / n over the nonzero
    eigenpairs 1..ell (lambda_0 excluded), f~ = Lambda^-1 g~, f = Q f~."""
    n = g.shape[0]
    Q = e.phi[:, 1:]
    gt = Q.T @ (S * S * g) / n
    return Q @ (gt / e.evals[1:])


def triple_products(e: Eigen, S: np.ndarray) -> np.ndarray:
    """Sec. 3.2: C-hat_ljk = <phi_l, phi_j * phi_k>_S over the computed eigenvectors
    (l, j, k = 0..ell), the discrete counterpart of Eq. (C_ijk)."""
    n = S.shape[0]
    return np.einsum("il,ij,ik,i->ljk", e.phi, e.phi, e.phi, S * S / n, optimize=True)


def gradient_dot(e: Eigen, S: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Sec. 3.2, Eq. (gradient in the eigenbasis) truncated after the computed
    eigenpairs:  grad u . grad v = sum_{l,j,k} u_j v_k (C_ljk / 2)(lambda_l - lambda_j
    - lambda_k) phi_l, with u_j = <u, phi_j>_S and v_k = <v, phi_k>_S.  With v the
    coordinate x_s this is the derivative du/dx_s (Eq. gradient of u)."""
    n = S.shape[0]
    w = S * S / n
    uh = e.phi.T @ (w * u)
    vh = e.phi.T @ (w * v)
    lam = e.evals
    C = triple_products(e, S)
    fac = 0.5 * (lam[:, None, None] - lam[None, :, None] - lam[None, None, :])
    coef = np.einsum("ljk,j,k->l", C * fac, uh, vh)
    return e.phi @ coef


def carre_du_champ(L: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Lemma (Carre du Champ identity) for a matrix L: (L(uv) - u L v - v L u) / 2."""
    return 0.5 * (L @ (u * v) - u * (L @ v) - v * (L @ u))


def s_inner(S: np.ndarray, f: np.ndarray, g: np.ndarray) -> float:
    """Eq. (inner product): <f, g>_S = f^T S^2 g / n."""
    return float(f @ (S * S * g) / f.shape[0])
