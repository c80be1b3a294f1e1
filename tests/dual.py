"""Forward-mode dual numbers (value + one tangent) for checking adjoints.

A dual a + b*eps with eps^2 = 0 propagates the directional derivative b through
+, -, *, / and log1p exactly (up to rounding), so f(x + e_j eps) has
df/dx_j as its tangent.  Test helper only.
"""
import math


class Dual:
    __slots__ = ("v", "d")

    def __init__(self, v, d=0.0):
        self.v = float(v)
        self.d = float(d)

    @staticmethod
    def lift(a):
        return a if isinstance(a, Dual) else Dual(a, 0.0)

    def __add__(self, o):
        o = Dual.lift(o)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = Dual.lift(o)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return Dual.lift(o) - self

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __mul__(self, o):
        o = Dual.lift(o)
        return Dual(self.v * o.v, self.d * o.v + self.v * o.d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = Dual.lift(o)
        return Dual(self.v / o.v, (self.d * o.v - self.v * o.d) / (o.v * o.v))


def log1p(a):
    a = Dual.lift(a)
    return Dual(math.log1p(a.v), a.d / (1.0 + a.v))


def seed(vals, j):
    """Duals for a vector with unit tangent on entry j."""
    return [Dual(v, 1.0 if i == j else 0.0) for i, v in enumerate(vals)]
