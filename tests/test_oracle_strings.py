"""Pins for occupation strings and excitation lists (counts, ranks, signs)."""
from math import comb

import numpy as np
import pytest

from oracle import slater_condon as sc
from oracle import strings as st


@pytest.mark.parametrize("n,m", [(2, 1), (4, 2), (6, 3), (7, 2), (8, 5), (10, 5)])
def test_counts_and_addresses(n, m):
    s = st.enumerate_strings(n, m)
    assert len(s) == comb(n, m)
    assert np.all(np.diff(s) > 0)
    for i, mask in enumerate(s):
        assert st.address(int(mask), n) == i


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (7, 3), (8, 4), (10, 5)])
def test_excitation_list_against_spin_orbital_operators(n, m):
    """Each (k, l, J, sign) must equal a+_k a_l applied to the bitmask by the
    independent operator code of the Slater-Condon module, in the stated order."""
    s = st.enumerate_strings(n, m)
    tab = st.excitation_list(n, m)
    assert tab.shape == (len(s), m * (n - m + 1), 4)
    for I, mask in enumerate(s):
        mask = int(mask)
        occ = [p for p in range(n) if mask >> p & 1]
        expect = []
        for l in occ:
            for k in sorted([p for p in range(n) if not mask >> p & 1] + [l]):
                sign, new = sc.apply_ops(mask, [("+", k), ("-", l)])
                expect.append((k, l, int(np.searchsorted(s, new)), sign))
        assert [tuple(int(v) for v in row) for row in tab[I]] == expect


def test_sign_parity_rule():
    """sign(a+_k a_l |I>) = (-1)^(number of occupied orbitals strictly between k and l)."""
    n, m = 9, 4
    s = st.enumerate_strings(n, m)
    tab = st.excitation_list(n, m)
    for I, mask in enumerate(s):
        for k, l, J, sign in tab[I]:
            lo, hi = min(k, l), max(k, l)
            between = bin(int(mask) & ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)).count("1")
            assert sign == (-1) ** between


def test_pair_index_is_a_bijection():
    n = 16
    seen = {st.pair_index(k, l) for k in range(n) for l in range(k + 1)}
    assert seen == set(range(n * (n + 1) // 2))
    assert all(st.pair_index(k, l) == st.pair_index(l, k) for k in range(n) for l in range(n))
