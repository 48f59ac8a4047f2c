"""Shared helpers of the GPU tests: build-on-demand and oracle caches."""
import functools
import os

import numpy as np
import pytest


def gpu_available() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def require_lib():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2603_06101_gb300 import build, sbci

    if not os.path.exists(sbci.LIB_PATH):
        build.build()
    return sbci


@functools.lru_cache(maxsize=None)
def oracle_sigma(key):
    from oracle import sigma as sg

    I = make_integrals(key)
    return sg.StringSigma(I.h1, I.eri, I.nalpha, I.nbeta)


@functools.lru_cache(maxsize=None)
def make_integrals(key):
    from paper_2603_06101_gb300 import inputs

    kind = key[0]
    if kind == "chain":
        _, nat, R = key
        return inputs.h_chain(nat, R)
    _, n, seed, na, nb = key
    return inputs.random_df(n, seed, na, nb)


def rel_err(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@functools.lru_cache(maxsize=None)
def oracle_sector_energies(key, k):
    """Lowest k electronic energies of H in the c = c^T sector (n_alpha =
    n_beta): Lanczos (oracle.eigen.lowest_lanczos) on S H S, S the
    symmetriser c -> (c + c^T)/2.  The antisymmetric complement maps to 0, so
    for the negative electronic energies of these systems the k lowest
    eigenvalues of S H S are the sector's."""
    from oracle import eigen

    ora = oracle_sigma(key)
    na, nb = ora.Na, ora.Nb
    assert na == nb

    def apply(v):
        m = v.reshape(na, nb)
        h = ora.apply(0.5 * (m + m.T))
        return 0.5 * (h + h.T)

    v0 = np.random.default_rng(7).standard_normal(na * nb).reshape(na, nb)
    v0 = (v0 + v0.T).reshape(-1)
    w, _ = eigen.lowest_lanczos(apply, na * nb, k, v0=v0)
    assert w.max() < -1e-3, "sector energies must be negative for the projection to isolate them"
    return w
