"""FP64 CPU oracle for the sparse self-tuning variable-bandwidth kernel build
of Davis & Giannakis, "Graph-theoretic algorithms for Kolmogorov operators"
(arXiv 2104.15124).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / reference leg of `bench.py` may import, call, link or run
anything in this package.  The product path (the CUDA library and its Python
binding) never does, and this package imports nothing from it.

Contents
  knn_bf.c   plain C FP64 brute-force exact kNN (OpenMP), canonical distance
  knn.py     ctypes loader for knn_bf.c, plus a numpy brute force for tiny n
  method.py  the method's formulas in FP64 (bandwidth, pattern, epsilon sweeps,
             density, operator normalisations, symmetric operator L-hat),
             the dense all-pairs form of Algorithm 1 used as a pin, and the
             spectral solve of Sec. 3.1
  mlp.py     the learned radius network's forward and backward passes in FP64, for
             the training-kernel pins
  radius.py  the paper's delta_tol pattern (Algorithm 1, Sec. 4) and its per-grid-point
             sweep, the next row after the kNN pattern
  evolve.py  one explicit step of the particle evolution of a time-dependent density
             (Sec. 6): solve L_{1,psi} f = g, grad f by Sec. 3.2, move the samples

Every function cites the passage (section, equation, algorithm) it follows.
"""
