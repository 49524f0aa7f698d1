"""Forward-mode derivative numbers used by the oracle (test infrastructure only).

Two plain types, written for readability rather than speed:

* ``Dual``  -- value and first derivatives with respect to ``n`` inputs.  The
  arithmetic is generic over the scalar type, so the geometry code runs it over
  ``fractions.Fraction`` and gets *exact* rational values and gradients for the
  squared distances and the edge cross-product measure.
* ``Jet``   -- value, gradient and Hessian with respect to ``n`` inputs (second
  order).  Used over ``float`` for the barrier as a function of the gap function
  g, of the mollifier argument gamma, and of the entries of the constraint
  Jacobian J (the J-space Hessians of Eq. 17 and Eq. 31).

Only the product, quotient and chain rules appear here; nothing in this module
knows about contact, barriers or eigensystems.
"""
import math


class Dual:
    """Value ``v`` and gradient ``d`` (a list of length n)."""

    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = v
        self.d = d

    @staticmethod
    def variable(value, index, n, zero):
        d = [zero] * n
        d[index] = zero + 1
        return Dual(value, d)

    @staticmethod
    def const(value, n, zero):
        return Dual(value, [zero] * n)

    def _lift(self, o):
        return o if isinstance(o, Dual) else Dual(o, [o * 0] * len(self.d))

    def __add__(self, o):
        o = self._lift(o)
        return Dual(self.v + o.v, [a + b for a, b in zip(self.d, o.d)])

    __radd__ = __add__

    def __sub__(self, o):
        o = self._lift(o)
        return Dual(self.v - o.v, [a - b for a, b in zip(self.d, o.d)])

    def __rsub__(self, o):
        return self._lift(o) - self

    def __neg__(self):
        return Dual(-self.v, [-a for a in self.d])

    def __mul__(self, o):
        o = self._lift(o)
        return Dual(self.v * o.v, [a * o.v + self.v * b for a, b in zip(self.d, o.d)])

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = self._lift(o)
        q = self.v / o.v
        return Dual(q, [(a - q * b) / o.v for a, b in zip(self.d, o.d)])

    def __rtruediv__(self, o):
        return self._lift(o) / self


class Jet:
    """Value ``v``, gradient ``g`` (length n) and Hessian ``h`` (n x n lists)."""

    __slots__ = ("v", "g", "h")

    def __init__(self, v, g, h):
        self.v = v
        self.g = g
        self.h = h

    @staticmethod
    def variable(value, index, n):
        g = [0.0] * n
        g[index] = 1.0
        return Jet(value, g, [[0.0] * n for _ in range(n)])

    @staticmethod
    def const(value, n):
        return Jet(value, [0.0] * n, [[0.0] * n for _ in range(n)])

    def _lift(self, o):
        return o if isinstance(o, Jet) else Jet.const(o, len(self.g))

    def _compose(self, f0, f1, f2):
        """Chain rule for a scalar function with f(v)=f0, f'(v)=f1, f''(v)=f2."""
        n = len(self.g)
        g = [f1 * a for a in self.g]
        h = [[f1 * self.h[i][j] + f2 * self.g[i] * self.g[j] for j in range(n)] for i in range(n)]
        return Jet(f0, g, h)

    def __add__(self, o):
        o = self._lift(o)
        n = len(self.g)
        return Jet(self.v + o.v, [a + b for a, b in zip(self.g, o.g)],
                   [[self.h[i][j] + o.h[i][j] for j in range(n)] for i in range(n)])

    __radd__ = __add__

    def __neg__(self):
        n = len(self.g)
        return Jet(-self.v, [-a for a in self.g], [[-self.h[i][j] for j in range(n)] for i in range(n)])

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        o = self._lift(o)
        n = len(self.g)
        g = [a * o.v + self.v * b for a, b in zip(self.g, o.g)]
        h = [[self.h[i][j] * o.v + self.v * o.h[i][j] + self.g[i] * o.g[j] + o.g[i] * self.g[j]
              for j in range(n)] for i in range(n)]
        return Jet(self.v * o.v, g, h)

    __rmul__ = __mul__

    def reciprocal(self):
        v = self.v
        return self._compose(1.0 / v, -1.0 / (v * v), 2.0 / (v * v * v))

    def __truediv__(self, o):
        o = self._lift(o)
        return self * o.reciprocal()

    def __rtruediv__(self, o):
        return self._lift(o) * self.reciprocal()


def jlog(x):
    """Natural logarithm of a Jet (or a float)."""
    if not isinstance(x, Jet):
        return math.log(x)
    v = x.v
    return x._compose(math.log(v), 1.0 / v, -1.0 / (v * v))


def jsqrt(x):
    """Square root of a Jet (or a float)."""
    if not isinstance(x, Jet):
        return math.sqrt(x)
    s = math.sqrt(x.v)
    return x._compose(s, 0.5 / s, -0.25 / (s * x.v))
