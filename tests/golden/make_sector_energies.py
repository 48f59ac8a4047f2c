"""Writes h10_sector_energies.json: the exact lowest energies of the H10
workload (linear H10, STO-3G, Loewdin basis, 1.2 A) in the c = c^T sector,
from the oracle alone (Lanczos on the symmetrised oracle sigma, tol 1e-12).

bench.py reads the file to state the per-state energy error of the GPU
solves; nothing here runs on the GPU or imports the CUDA library.  Run from the
repository root: ``python tests/golden/make_sector_energies.py``.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import eigen  # noqa: E402
from oracle import sigma as osg  # noqa: E402
from paper_2603_06101_gb300 import inputs  # noqa: E402


def sector_energies(I, k):
    sig = osg.StringSigma(I.h1, I.eri, I.nalpha, I.nbeta)
    na = sig.Na

    def apply(v):
        m = v.reshape(na, na)
        h = sig.apply(0.5 * (m + m.T))
        return 0.5 * (h + h.T)

    v0 = np.random.default_rng(7).standard_normal((na, na))
    v0 = (v0 + v0.T).reshape(-1)
    w, _ = eigen.lowest_lanczos(apply, na * na, k, v0=v0)
    return w


def main():
    I = inputs.h_chain(10, 1.2)
    w = sector_energies(I, 4)
    out = {
        "what": "lowest 4 energies of H10 (STO-3G, Loewdin, 1.2 A) in the c = c^T sector, hartree",
        "how": "oracle.eigen.lowest_lanczos (tol 1e-12) on S H S, S c = (c + c^T)/2, H the oracle "
               "string sigma; written by tests/golden/make_sector_energies.py",
        "e_core": float(I.e_core),
        "electronic": [float(x) for x in w],
        "total": [float(x + I.e_core) for x in w],
    }
    with open(os.path.join(HERE, "h10_sector_energies.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out["total"])


if __name__ == "__main__":
    main()
