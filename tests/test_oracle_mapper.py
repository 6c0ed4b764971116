"""Pins of the oracle's interface configuration (Sec. 4.3, Eqs. subim and indices).

* the integer brute-force overlap search is checked against an exact rational search
  written here with fractions.Fraction;
* the closed form n = floor(Delta/l), s = Delta/l - n is checked bit for bit against the
  brute force over 10^5 random displacements and at exact multiples of l;
* the worked example of Appendix A (n = 1) is reproduced through Eq. indices.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rational_search(delta, l, n_par):
    """Exact overlap search on the rounded quotient q = fl(delta / l)."""
    q = Fraction(delta / l)
    pairs = np.zeros((n_par, 2), dtype=np.int32)
    ns, ss = set(), set()
    for i in range(n_par):
        lower = upper = None
        for j in range(n_par):
            for w in range(-3, 4):
                base = int(np.floor(float(i - j - q) / n_par)) + w
                a = q + j + base * n_par
                if a < i <= a + 1:
                    assert lower is None
                    lower = j
                if i <= a < i + 1:
                    assert upper is None
                    upper = j
                    ns.add(i - j - base * n_par)
                    ss.add(a - i)
        pairs[i] = (lower, upper)
    assert len(ns) == 1 and len(ss) == 1
    return ns.pop(), ss.pop(), pairs


@pytest.mark.parametrize("n_par", [1, 2, 3, 4, 7])
def test_bruteforce_matches_exact_rationals(n_par):
    rng = np.random.default_rng(n_par)
    l = 1.0 / n_par
    deltas = list(rng.uniform(-3.0, 3.0, 60)) + [0.0, l, 2 * l, -l, 0.37, -0.37, 1e-9, -1e-9]
    for d in deltas:
        rc, n, s, pairs = O.map_bruteforce(d, l, n_par)
        assert rc == 0
        nr, sr, pr = rational_search(d, l, n_par)
        assert n == nr
        assert Fraction(s) == sr or (sr > 0 and s == float(sr))  # s is representable
        assert np.array_equal(pairs, pr)


@pytest.mark.parametrize("n_par,l", [(4, 0.25), (64, 1.0 / 64), (48, np.pi / 192), (5, 0.3)])
def test_closed_form_bit_exact_vs_bruteforce(n_par, l):
    deltas = synth.random_displacements(seed=11 + n_par, count=25000, scale=7.0 * n_par * l)
    for d in deltas:
        n, s = O.map_closed(d, l)
        rc, nb, sb, pb = O.map_bruteforce(d, l, n_par)
        assert rc == 0
        assert n == nb
        assert np.float64(s).tobytes() == np.float64(sb).tobytes()
        assert np.array_equal(O.map_pairs(n, n_par), pb)
        assert 0.0 <= s < 1.0


@pytest.mark.parametrize("n_par", [1, 4, 9])
def test_exact_multiples_give_conforming_faces(n_par):
    l = 0.125
    for m in range(-3 * n_par, 3 * n_par + 1):
        d = m * l
        n, s = O.map_closed(d, l)
        assert (n, s) == (m, 0.0)
        rc, nb, sb, pb = O.map_bruteforce(d, l, n_par)
        assert rc == 0 and (nb, sb) == (m, 0.0)
        # conforming instant: the upper mortar (i_sub = 1) is the whole face, partner i - n
        for i in range(n_par):
            assert pb[i, 1] == (i - m) % n_par


def test_subim_lower_mortar_is_below_hanging_node():
    # Eq. subim: i_sub = 0 marks the part eta - i l < s l of static face i, which the
    # moving face i - n - 1 covers (its upper end sits at (i + s) l).
    l, n_par = 0.25, 4
    for d in (0.1, 0.3, 0.61, 1.2, -0.4):
        n, s = O.map_closed(d, l)
        pairs = O.map_pairs(n, n_par)
        for i in range(n_par):
            lower_partner_top = (pairs[i, 0] + n + s + 1)     # in face units, mod n_par
            r = (lower_partner_top - i - s) % n_par
            assert min(r, n_par - r) < 1e-12


def test_appendix_a_worked_example():
    """Appendix A: with n = 1 the moving partners (Eq. indices) of the five static faces
    reproduce the printed ranks r~, the sorted array A and the inverse map m."""
    g = json.load(open(os.path.join(GOLDEN, "appendix_a_mortar_sorting.json")))
    r_tilde = {}
    for row, vals in zip(g["r_tilde"]["rows_i_perp"], g["r_tilde"]["values"]):
        for c, r in enumerate(vals):
            r_tilde[(g["r_tilde"]["first_i_tilde"] + c, row)] = r
    n = g["n_delta"]
    n_par = 16                                                         # large enough: no wrap
    pairs = O.map_pairs(n, n_par)
    cols = []
    for ipar, iperp, iface in g["static_faces"]:
        for isub in (0, 1):
            it = int(pairs[ipar, isub])
            assert it == ipar - n + isub - 1
            cols.append((r_tilde[(it, iperp)], ipar, iperp, isub, iface))
    A = sorted(cols, key=lambda c: c[:4])
    assert np.array_equal(np.array(A).T, np.array(g["A"]))
    m = np.zeros((2, 5), dtype=int)
    for imortar, c in enumerate(A, start=1):
        m[c[3], c[4] - g["m_first_i_face"]] = imortar
    assert np.array_equal(m, g["m"])
