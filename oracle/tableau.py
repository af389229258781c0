"""Butcher tableaux in exact rationals.

* Bogacki-Shampine 3(2): Table Butcher-O23 (Sec. 2.2).  X^{n+1} uses b (third
  order, FSAL: the last row of A equals b); the embedded solution uses b~.
* Dormand-Prince 5(4): the pair behind the paper's ode45 reference solution
  (Sec. 2.4), from Dormand & Prince (1980), J. Comp. Appl. Math. 6(1).

Pinned by exact order-condition checks in tests/test_oracle_tableau.py.
"""

from fractions import Fraction as Fr

BS3_C = (Fr(0), Fr(1, 2), Fr(3, 4), Fr(1))
BS3_A = (
    (),
    (Fr(1, 2),),
    (Fr(0), Fr(3, 4)),
    (Fr(2, 9), Fr(1, 3), Fr(4, 9)),
)
BS3_B = (Fr(2, 9), Fr(1, 3), Fr(4, 9), Fr(0))
BS3_BTILDE = (Fr(7, 24), Fr(1, 4), Fr(1, 3), Fr(1, 8))
# X^{n+1} - X~^{n+1} = h * sum_l E_l K_l
BS3_E = tuple(b - bt for b, bt in zip(BS3_B, BS3_BTILDE))

DP5_C = (Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1))
DP5_A = (
    (),
    (Fr(1, 5),),
    (Fr(3, 40), Fr(9, 40)),
    (Fr(44, 45), Fr(-56, 15), Fr(32, 9)),
    (Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)),
    (Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)),
    (Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)),
)
DP5_B = (Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), Fr(0))
DP5_BSTAR = (Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200),
             Fr(187, 2100), Fr(1, 40))


def as_float(t):
    """Nested tuple of Fractions -> nested tuple of Python floats."""
    if isinstance(t, Fr):
        return float(t)
    return tuple(as_float(x) for x in t)
