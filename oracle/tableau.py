"""Butcher tableaus of the two embedded 5(4) pairs.

The paper delegates time stepping to DifferentialEquations.jl and names no
method; the integrator chosen here is an explicit 7-stage, first-same-as-last
5(4) pair: Dormand & Prince (1980), "A family of embedded Runge-Kutta
formulae", J. Comput. Appl. Math. 6, 19-26, and Tsitouras (2011),
"Runge-Kutta pairs of order 5(4) satisfying only the first column simplifying
assumption", Comput. Math. Appl. 62, 770-775.

Each tableau has: c (nodes), a (7x7 strictly lower), b (5th-order weights,
equal to the last row of a, so stage 7 is evaluated at the new solution and
reused as stage 1 of the next step), and e = b - bhat (weights of the
embedded error estimate).  Pinned by tests/test_oracle_tableau.py: all
rooted-tree order conditions to order 5 for b and order 4 for bhat, and the
row-sum condition c_i = sum_j a_ij.
"""
from fractions import Fraction as Fr

import numpy as np


class Tableau:
    def __init__(self, name, c, a, b, bhat):
        self.name = name
        self.c = np.array([float(x) for x in c])
        self.a = np.array([[float(x) for x in row] for row in a])
        self.b = np.array([float(x) for x in b])
        self.bhat = np.array([float(x) for x in bhat])
        self.e = np.array([float(x) - float(y) for x, y in zip(b, bhat)])
        self.exact = (c, a, b, bhat)
        self.stages = len(self.b)


def _dp5():
    c = [Fr(0), Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), Fr(1), Fr(1)]
    a = [[Fr(0)] * 7 for _ in range(7)]
    a[1][0] = Fr(1, 5)
    a[2][:2] = [Fr(3, 40), Fr(9, 40)]
    a[3][:3] = [Fr(44, 45), Fr(-56, 15), Fr(32, 9)]
    a[4][:4] = [Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)]
    a[5][:5] = [Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)]
    a[6][:6] = [Fr(35, 384), Fr(0), Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)]
    b = list(a[6][:6]) + [Fr(0)]
    bhat = [Fr(5179, 57600), Fr(0), Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200),
            Fr(187, 2100), Fr(1, 40)]
    # Store the error weights exactly: e = b - bhat.
    t = Tableau("dp5", c, a, b, bhat)
    t.e = np.array([float(x - y) for x, y in zip(b, bhat)])
    return t


def _tsit5():
    c = [0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0]
    a = [[0.0] * 7 for _ in range(7)]
    a[1][0] = 0.161
    a[2][:2] = [-0.008480655492356989, 0.335480655492357]
    a[3][:3] = [2.897153057105493, -6.359448489975075, 4.3622954328695815]
    a[4][:4] = [5.325864828439257, -11.748883564062828, 7.4955393428898365,
                -0.09249506636175525]
    a[5][:5] = [5.86145544294642, -12.92096931784711, 8.159367898576159,
                -0.071584973281401, -0.028269050394068383]
    a[6][:6] = [0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742,
                -3.290069515436081, 2.324710524099774]
    b = list(a[6][:6]) + [0.0]
    # Error weights e = b - bhat as published with the method.
    e = [-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995,
         -0.1447110071732629, 0.5823571654525552, -0.45808210592918697,
         0.015151515151515152]
    bhat = [bi - ei for bi, ei in zip(b, e)]
    t = Tableau("tsit5", c, a, b, bhat)
    t.e = np.array(e)
    return t


DP5 = _dp5()
TSIT5 = _tsit5()
TABLEAUS = {"dp5": DP5, "tsit5": TSIT5}
