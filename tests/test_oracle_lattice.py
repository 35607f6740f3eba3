"""Pins of the oracle's lattice tables against what the paper fixes.

The D3Q19 weights and gradient tensors are printed in the LBM section (the
weight table beneath Eq. eqdistfbinary); the D2Q9 set is not in the paper.
Both must make the second moment of f_eq reproduce the pressure tensor of the
Equations-of-Motion section: the term kappa [d_a X d_b X - |grad X|^2 delta / 2]
requires sum_i w_i^{aa} e_ia^2 = c_s^2/2, sum_i w_i^{aa} e_ib^2 = -c_s^2/2 (b != a)
and sum_i w_i^{ab} e_ia e_ib = c_s^2 for a != b.  All identities are checked in
exact rationals.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

COMP = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (2, 0)]


def _rat(x):
    fr = Fraction(x).limit_denominator(1000)
    assert abs(float(fr) - x) < 1e-15, x
    return fr


@pytest.mark.parametrize("Q,D", [(9, 2), (19, 3)])
def test_velocity_set_and_weights(Q, D):
    e, w, t, opp = oracle.lattice(Q)
    W = [_rat(v) for v in w]
    cs2 = Fraction(1, 3)
    assert sum(W) == 1
    # only the expected speeds: 0, 1, sqrt(2)
    assert sorted(set(int((e[i] ** 2).sum()) for i in range(Q))) == [0, 1, 2]
    assert all(int(v) == 0 for v in e[0])
    # the D2Q9 set is planar
    if D == 2:
        assert np.all(e[:, 2] == 0)
    # isotropy up to fourth order (c_s^2 = 1/3)
    for a in range(3):
        assert sum(W[i] * e[i][a] for i in range(Q)) == 0
        for b in range(3):
            m2 = sum(W[i] * e[i][a] * e[i][b] for i in range(Q))
            assert m2 == (cs2 if (a == b and a < D) else 0)
    for a in range(D):
        for b in range(D):
            for c in range(D):
                for d in range(D):
                    m4 = sum(W[i] * e[i][a] * e[i][b] * e[i][c] * e[i][d] for i in range(Q))
                    want = cs2 * cs2 * ((a == b) * (c == d) + (a == c) * (b == d) + (a == d) * (b == c))
                    assert m4 == want
    # opposites
    for i in range(Q):
        assert np.all(e[opp[i]] == -e[i])
    # weight classes: rest, axis, diagonal/edge
    if Q == 19:
        assert W[0] == Fraction(1, 3)
        assert all(W[i] == Fraction(1, 18) for i in range(1, 7))
        assert all(W[i] == Fraction(1, 36) for i in range(7, 19))
    else:
        assert W[0] == Fraction(4, 9)
        assert all(W[i] == Fraction(1, 9) for i in range(1, 5))
        assert all(W[i] == Fraction(1, 36) for i in range(5, 9))


def test_d3q19_order_matches_weight_table():
    """The paper's tensor table puts xy-plane edges at 7-10, yz at 11-14, zx at 15-18,
    with w^{xy}_{7,10} = +1/12 (e_x e_y = +1) and w^{xy}_{8,9} = -1/12."""
    e, w, t, _ = oracle.lattice(19)
    assert [tuple(e[i]) for i in range(1, 7)] == [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                                 (0, 0, 1), (0, 0, -1)]
    for i in range(7, 11):
        assert e[i][2] == 0 and abs(e[i][0]) == 1 and abs(e[i][1]) == 1
    for i in range(11, 15):
        assert e[i][0] == 0
    for i in range(15, 19):
        assert e[i][1] == 0
    T = [[_rat(v) for v in row] for row in t]
    # printed entries
    assert T[1][0] == T[3][1] == T[5][2] == Fraction(5, 36)
    assert all(T[i][0] == Fraction(-1, 9) for i in (3, 4, 5, 6))
    assert all(T[i][0] == Fraction(-1, 72) for i in list(range(7, 11)) + list(range(15, 19)))
    assert all(T[i][0] == Fraction(1, 36) for i in range(11, 15))
    assert T[7][3] == T[10][3] == Fraction(1, 12) and T[8][3] == T[9][3] == Fraction(-1, 12)
    assert T[11][4] == T[14][4] == Fraction(1, 12) and T[12][4] == T[13][4] == Fraction(-1, 12)
    assert T[15][5] == T[18][5] == Fraction(1, 12) and T[16][5] == T[17][5] == Fraction(-1, 12)


@pytest.mark.parametrize("Q,D", [(9, 2), (19, 3)])
def test_gradient_tensors_reproduce_pressure_tensor(Q, D):
    e, w, t, _ = oracle.lattice(Q)
    T = [[_rat(v) for v in row] for row in t]
    cs2 = Fraction(1, 3)
    for c, (a, b) in enumerate(COMP):
        if a >= D or b >= D:
            assert all(T[i][c] == 0 for i in range(Q))
            continue
        for g in range(D):
            for d in range(D):
                m2 = sum(T[i][c] * e[i][g] * e[i][d] for i in range(Q))
                if a == b:
                    want = (cs2 / 2 if g == a else -cs2 / 2) if g == d else 0
                else:
                    want = cs2 if {g, d} == {a, b} else 0
                assert m2 == want, (Q, c, g, d, m2, want)
        # odd moments vanish: gradient terms must not change momentum
        for g in range(3):
            assert sum(T[i][c] * e[i][g] for i in range(Q)) == 0
            for d in range(3):
                for h in range(3):
                    assert sum(T[i][c] * e[i][g] * e[i][d] * e[i][h] for i in range(Q)) == 0
        # tensors are even: equal on opposite directions
        _, _, _, opp = oracle.lattice(Q)
        assert all(T[i][c] == T[opp[i]][c] for i in range(Q))
