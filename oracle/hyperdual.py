"""Hyper-dual numbers for exact first and second derivatives (oracle only).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline use this package; the product path never does.

A hyper-dual number a + b e1 + c e2 + d e1 e2 with e1^2 = e2^2 = 0 carries,
when seeded with b = c = 1 along coordinate i, the value f, the first
derivative df/dx_i (in b and c) and the second derivative d2f/dx_i^2 (in d),
exact up to rounding (Fike & Alonso, AIAA 2011-886).  The oracle uses them to
differentiate the full local basis function L * omega_j * tanh(R x_hat + b)
(Eq. (netdd)) without any hand-derived product or quotient rule.
"""
from __future__ import annotations

import numpy as np


class HD:
    __slots__ = ("a", "b", "c", "d")

    def __init__(self, a, b=0.0, c=0.0, d=0.0):
        self.a, self.b, self.c, self.d = a, b, c, d

    @staticmethod
    def var(x, seed: bool) -> "HD":
        """Independent variable x; seeded (derivative direction) or constant."""
        z = np.zeros_like(x)
        return HD(x, z + 1.0, z + 1.0, z) if seed else HD(x, z, z, z)

    @staticmethod
    def const(x) -> "HD":
        return HD(x, 0.0, 0.0, 0.0)

    def _wrap(o):
        return o if isinstance(o, HD) else HD(o, 0.0, 0.0, 0.0)

    def __add__(self, o):
        o = HD._wrap(o)
        return HD(self.a + o.a, self.b + o.b, self.c + o.c, self.d + o.d)

    __radd__ = __add__

    def __neg__(self):
        return HD(-self.a, -self.b, -self.c, -self.d)

    def __sub__(self, o):
        return self + (-HD._wrap(o))

    def __rsub__(self, o):
        return HD._wrap(o) + (-self)

    def __mul__(self, o):
        o = HD._wrap(o)
        return HD(self.a * o.a,
                  self.a * o.b + self.b * o.a,
                  self.a * o.c + self.c * o.a,
                  self.a * o.d + self.b * o.c + self.c * o.b + self.d * o.a)

    __rmul__ = __mul__

    def _chain(self, f0, f1, f2):
        """Apply a scalar function with derivatives f0 = f(a), f1 = f'(a), f2 = f''(a)."""
        return HD(f0, f1 * self.b, f1 * self.c, f1 * self.d + f2 * self.b * self.c)

    def recip(self):
        inv = 1.0 / self.a
        return self._chain(inv, -inv * inv, 2.0 * inv * inv * inv)

    def __truediv__(self, o):
        return self * HD._wrap(o).recip()

    def __rtruediv__(self, o):
        return HD._wrap(o) * self.recip()


def tanh(x: HD) -> HD:
    t = np.tanh(x.a)
    s = 1.0 - t * t
    return x._chain(t, s, -2.0 * t * s)


def sin(x: HD) -> HD:
    s, c = np.sin(x.a), np.cos(x.a)
    return x._chain(s, c, -s)


def cos(x: HD) -> HD:
    s, c = np.sin(x.a), np.cos(x.a)
    return x._chain(c, -s, -c)


def exp(x: HD) -> HD:
    e = np.exp(x.a)
    return x._chain(e, e, e)


def where(mask, x: HD, y: HD) -> HD:
    return HD(np.where(mask, x.a, y.a), np.where(mask, x.b, y.b),
              np.where(mask, x.c, y.c), np.where(mask, x.d, y.d))
