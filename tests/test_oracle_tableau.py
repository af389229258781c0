"""Exact-rational pins of the tableaux (Table Butcher-O23; Dormand-Prince 1980)."""

from fractions import Fraction as Fr

from oracle.tableau import (BS3_A, BS3_B, BS3_BTILDE, BS3_C, BS3_E, DP5_A, DP5_B,
                            DP5_BSTAR, DP5_C)


def _full(A, s):
    return [[(A[i][j] if j < len(A[i]) else Fr(0)) for j in range(s)] for i in range(s)]


def _conditions(b, A, c):
    """Order conditions up to 4 as (lhs, rhs) pairs grouped by order."""
    s = len(b)
    A = _full(A, s)
    Ac = [sum(A[i][j] * c[j] for j in range(s)) for i in range(s)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(s)) for i in range(s)]
    dot = lambda u, v: sum(x * y for x, y in zip(u, v))  # noqa: E731
    return {
        1: [(sum(b), Fr(1))],
        2: [(dot(b, c), Fr(1, 2))],
        3: [(dot(b, [x * x for x in c]), Fr(1, 3)), (dot(b, Ac), Fr(1, 6))],
        4: [(dot(b, [x ** 3 for x in c]), Fr(1, 4)), (dot(b, [x * y for x, y in zip(c, Ac)]), Fr(1, 8)),
            (dot(b, Ac2), Fr(1, 12)), (dot(b, AAc), Fr(1, 24))],
    }


def test_bs3_row_sums_equal_c():
    for i, row in enumerate(BS3_A):
        assert sum(row, Fr(0)) == BS3_C[i]


def test_bs3_third_order_solution():
    cond = _conditions(BS3_B, BS3_A, BS3_C)
    for p in (1, 2, 3):
        for lhs, rhs in cond[p]:
            assert lhs == rhs
    assert any(lhs != rhs for lhs, rhs in cond[4])


def test_bs3_embedded_second_order():
    cond = _conditions(BS3_BTILDE, BS3_A, BS3_C)
    for p in (1, 2):
        for lhs, rhs in cond[p]:
            assert lhs == rhs
    assert any(lhs != rhs for lhs, rhs in cond[3])


def test_bs3_fsal_and_error_weights():
    assert tuple(BS3_A[3]) == tuple(BS3_B[:3]) and BS3_B[3] == 0
    assert sum(BS3_E) == 0
    assert BS3_E == (Fr(-5, 72), Fr(1, 12), Fr(1, 9), Fr(-1, 8))


def test_dopri5_orders():
    for i, row in enumerate(DP5_A):
        assert sum(row, Fr(0)) == DP5_C[i]
    for b in (DP5_B, DP5_BSTAR):
        cond = _conditions(b, DP5_A, DP5_C)
        for p in (1, 2, 3, 4):
            for lhs, rhs in cond[p]:
                assert lhs == rhs
    # FSAL: last row equals b
    assert tuple(DP5_A[6]) == tuple(DP5_B[:6])
