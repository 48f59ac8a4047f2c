"""Occupation strings and single-excitation lists (oracle; test infrastructure only).

The paper represents H "in terms of Slater determinants" (Results, SBCI1
algorithm) and leaves the determinant machinery to PySCF.  The conventions
fixed here (and matched by the CUDA library) are:

* a string is an m-subset of the n spatial orbitals, stored as a bitmask;
  strings are ordered by increasing bitmask value;
* the address of a string with occupied orbitals o_1 < ... < o_m is
  sum_k C(o_k, k) (k = 1..m), the combinatorial number system, which is
  exactly its rank in that order;
* a determinant |Ia Ib> is prod_{p in Ia, ascending} a+_{p alpha}
  prod_{q in Ib, ascending} a+_{q beta} |0>, all alpha creators to the left;
* the excitation list of string I has, for every occupied l (ascending) and
  every k in unocc(I) U {l} (ascending), the entry (k, l, J, sign) with
  a+_k a_l |I> = sign |J>.  m(n-m+1) entries per string.
"""
from __future__ import annotations

from math import comb

import numpy as np


def enumerate_strings(norb: int, nelec: int) -> np.ndarray:
    """All bitmasks with ``nelec`` bits among ``norb`` bits, increasing order."""
    out = [mask for mask in range(1 << norb) if bin(mask).count("1") == nelec]
    return np.array(out, dtype=np.int64)


def occupied(mask: int, norb: int) -> list[int]:
    return [p for p in range(norb) if (mask >> p) & 1]


def address(mask: int, norb: int) -> int:
    """Rank of a string among equal-popcount bitmasks: sum_k C(o_k, k)."""
    occ = occupied(mask, norb)
    return sum(comb(o, k + 1) for k, o in enumerate(occ))


def apply_annihilate(occ: list[int], p: int):
    """a_p on an ordered occupation list: returns (sign, new list) or None."""
    if p not in occ:
        return None
    pos = occ.index(p)  # number of occupied orbitals before p
    return (-1) ** pos, occ[:pos] + occ[pos + 1:]


def apply_create(occ: list[int], p: int):
    """a+_p on an ordered occupation list: returns (sign, new list) or None."""
    if p in occ:
        return None
    pos = sum(1 for q in occ if q < p)
    return (-1) ** pos, occ[:pos] + [p] + occ[pos:]


def excite(occ: list[int], k: int, l: int):
    """a+_k a_l applied to an occupation list, operator by operator."""
    r = apply_annihilate(occ, l)
    if r is None:
        return None
    s1, o1 = r
    r = apply_create(o1, k)
    if r is None:
        return None
    s2, o2 = r
    return s1 * s2, o2


def excitation_list(norb: int, nelec: int):
    """Per string: list of (k, l, J, sign) in the order stated in the module doc.

    Returns an int64 array of shape [nstr, nlink, 4].
    """
    strs = enumerate_strings(norb, nelec)
    rank = {int(m): i for i, m in enumerate(strs)}
    nlink = nelec * (norb - nelec + 1)
    table = np.zeros((len(strs), nlink, 4), dtype=np.int64)
    for I, mask in enumerate(strs):
        occ = occupied(int(mask), norb)
        unocc = [p for p in range(norb) if p not in occ]
        e = 0
        for l in occ:
            for k in sorted(unocc + [l]):
                sign, new = excite(occ, k, l)
                J = rank[sum(1 << p for p in new)]
                table[I, e] = (k, l, J, sign)
                e += 1
        assert e == nlink
    return table


def pair_index(k: int, l: int) -> int:
    """Lower-triangle packed index of the unordered pair {k, l}."""
    a, b = (k, l) if k >= l else (l, k)
    return a * (a + 1) // 2 + b
