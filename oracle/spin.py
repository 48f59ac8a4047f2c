"""<S^2> of a CI vector (oracle; test infrastructure only).

<S^2> = <S_- S_+> + S_z (S_z + 1) = |S_+ c|^2 + S_z (S_z + 1), with
S_+ = sum_p a+_{p alpha} a_{p beta} and S_z = (n_alpha - n_beta)/2.  The paper
reports <S^2> per state (Table 1); the operator is applied here determinant by
determinant with the spin-orbital operator code of ``oracle.slater_condon``.
"""
from __future__ import annotations

import numpy as np

from .slater_condon import apply_ops, determinants


def s_squared(c: np.ndarray, norb: int, nalpha: int, nbeta: int) -> float:
    c = np.asarray(c, dtype=np.float64).reshape(-1)
    dets = determinants(norb, nalpha, nbeta)
    splus: dict[int, float] = {}
    for coef, ket in zip(c, dets):
        if coef == 0.0:
            continue
        for p in range(norb):
            res = apply_ops(ket, [("+", p), ("-", norb + p)])
            if res is not None:
                splus[res[1]] = splus.get(res[1], 0.0) + res[0] * coef
    norm2 = float(c @ c)
    sz = 0.5 * (nalpha - nbeta)
    return (sum(v * v for v in splus.values())) / norm2 + sz * (sz + 1.0)
