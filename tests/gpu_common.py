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
