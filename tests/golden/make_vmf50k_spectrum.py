"""Writes vmf50k_spectrum.json: the FP64 oracle's 33 leading eigenvalues of L-hat for
the 50,000-point von Mises-Fisher workload (kappa = 2 about +z, k = 64, c = 1, d = 2,
beta = -1/4; Sec. 5.2's spherical example), with the tuned bandwidths and the mean
self weight of the Markov kernel, plus the continuum reference spectrum of L_{psi,1}
(oracle/spectra.py).  Calls only the oracle; rerun it to regenerate the file:

    python tests/golden/make_vmf50k_spectrum.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import method as M  # noqa: E402
from oracle import spectra as SP  # noqa: E402
from paper_2104_15124_gb300 import workloads as W  # noqa: E402


def main():
    w = W.VMF_50K
    B = M.build(w.sample(), w.k, d=w.d, c=w.c, beta=w.beta)
    e = M.leading_eigenpairs(B.lhat_csr(), B.op.S, 32)
    p = B.pattern
    dg = p.row == p.col
    out = {
        "cite": "Sec. 5.2 (spherical manifold, von Mises-Fisher density); eigenvalues of Eq. (symmetric discrete "
                "Kolmogorov operator) from the FP64 oracle; continuum from oracle/spectra.py",
        "workload": w.name, "n": w.n, "k": w.k, "c": w.c, "d": w.d, "beta": w.beta, "seed": w.seed,
        "eps2_den": B.den.eps2, "eps2_op": B.op_sweep.eps2,
        "self_weight": float(np.mean(B.op.Kt[dg] / B.op.D)),
        "evals": [float(v) for v in e.evals],
        "continuum": [float(v) for v in SP.sphere_drift_spectrum(2.0, w.c, 33)],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vmf50k_spectrum.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
