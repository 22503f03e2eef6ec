"""RK443 tableau: order conditions of an IMEX pair (exact rational arithmetic).

The paper uses the RK443 scheme of Ascher, Ruuth & Spiteri for both propagators
(Sec. 3.2, Sec. 3.6).  A wrong coefficient fails one of these conditions.
"""
from fractions import Fraction as Fr

from oracle.rbc import RK443_AE, RK443_AI, RK443_C


def frac(M):
    return [[Fr(x).limit_denominator(1000) for x in row] for row in M]


AI, AE = frac(RK443_AI), frac(RK443_AE)
c = [Fr(x).limit_denominator(1000) for x in RK443_C]
bI, bE = AI[4], AE[4]                      # stiffly accurate: b = last row


def dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def matvec(A, v):
    return [dot(row, v) for row in A]


def test_row_sums_equal_c():
    for i in range(5):
        assert sum(AI[i]) == c[i]
        assert sum(AE[i]) == c[i]


def test_explicit_part_is_explicit_and_implicit_diagonal_constant():
    for i in range(5):
        assert all(AE[i][j] == 0 for j in range(i, 5))
        assert all(AI[i][j] == 0 for j in range(i + 1, 5))
    assert [AI[i][i] for i in range(1, 5)] == [Fr(1, 2)] * 4
    assert all(AI[i][0] == 0 for i in range(5))


def test_third_order_conditions():
    for A, b in ((AI, bI), (AE, bE)):
        assert sum(b) == 1
        assert dot(b, c) == Fr(1, 2)
        assert dot(b, [x * x for x in c]) == Fr(1, 3)
        assert dot(b, matvec(A, c)) == Fr(1, 6)


def test_coupling_conditions():
    # mixed conditions for order 3 of the additive pair
    assert dot(bI, matvec(AE, c)) == Fr(1, 6)
    assert dot(bE, matvec(AI, c)) == Fr(1, 6)
    assert dot(bI, matvec(AI, c)) == Fr(1, 6)
    assert dot(bE, matvec(AE, c)) == Fr(1, 6)
