"""The committed script that writes the bench's exact sector energies
(tests/golden/make_sector_energies.py) computes them by Lanczos on the
symmetrised oracle sigma.  Pinned here on H6 against the dense Slater-Condon
Hamiltonian: its eigenvectors with c = c^T (the singlet sector of reading
R10) carry the same energies; and the committed file is well formed."""
import importlib.util
import json
import os

import numpy as np

from paper_2603_06101_gb300 import inputs
from oracle import slater_condon as sc

HERE = os.path.dirname(os.path.abspath(__file__))


def _script():
    spec = importlib.util.spec_from_file_location("make_sector_energies",
                                                  os.path.join(HERE, "golden", "make_sector_energies.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sector_lanczos_equals_dense_symmetric_eigenvectors():
    I = inputs.h_chain(6, 1.0)
    w = _script().sector_energies(I, 4)
    H = sc.dense_hamiltonian(I.h1, I.eri, 3, 3)
    ev, V = np.linalg.eigh(H)
    sym = [i for i in range(len(ev))
           if np.abs(V[:, i].reshape(20, 20) - V[:, i].reshape(20, 20).T).max() < 1e-6]
    assert np.abs(w - ev[sym][:4]).max() < 1e-10


def test_committed_h10_sector_energies():
    with open(os.path.join(HERE, "golden", "h10_sector_energies.json")) as f:
        d = json.load(f)
    tot, el = np.array(d["total"]), np.array(d["electronic"])
    assert tot.size == 4 and np.all(np.diff(tot) > 0)
    assert np.allclose(tot - el, d["e_core"], atol=1e-12, rtol=0)
    I = inputs.h_chain(10, 1.2)
    assert abs(d["e_core"] - I.e_core) < 1e-10
