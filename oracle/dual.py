"""Forward-mode dual numbers over numpy arrays, with a running magnitude bound.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this package;
only the tests, the smoke check and the benchmark's CPU-baseline leg use it.

A ``D`` holds, for every element of a 1-D batch (one entry per cell or per
face):

* ``v``  -- the value,
* ``g``  -- the exact derivative with respect to ``k`` seeded variables
  (shape ``(n, k)``),
* ``m``  -- the *magnitude* of the value: the same expression evaluated with
  every operand replaced by its absolute value and every subtraction turned
  into an addition,
* ``gm`` -- the same magnitude for each derivative.

``m`` and ``gm`` are the standard running bound of floating-point forward
error analysis: any evaluation order of the same expression in IEEE double
differs from the exact result by at most (a small multiple of) the unit
round-off times this magnitude.  The parity tests use them as the scale of
the relative tolerance, so that entries formed by cancellation (a pressure
difference, an accumulation change over one step) are judged against the size
of the terms that were cancelled rather than against the tiny result.

Branches (clamps, upwind choice) are decided on ``v`` only; the magnitude
follows the branch that the value takes.

Values may be complex: a complex input keeps ``v`` and ``g`` complex, so the
same code evaluated at u + i h e_j yields the complex-step derivative
Im R / h, which the tests use to pin the dual-number Jacobian.  Branches then
compare complex values lexicographically (real part first), which away from
exact ties is the comparison of the real parts.  Real inputs are unaffected.
"""
from __future__ import annotations

import numpy as np


def _arr(x):
    """float64 array, or complex128 where the input is complex."""
    return np.asarray(x, dtype=np.complex128 if np.iscomplexobj(x) else np.float64)


class D:
    __slots__ = ("v", "g", "m", "gm")
    __array_ufunc__ = None   # numpy scalars and arrays defer to D's operators

    def __init__(self, v, g, m=None, gm=None):
        self.v = _arr(v)
        self.g = _arr(g)
        self.m = np.abs(self.v) if m is None else np.asarray(m, dtype=np.float64)
        self.gm = np.abs(self.g) if gm is None else np.asarray(gm, dtype=np.float64)

    # ----------------------------------------------------------------- builders
    @staticmethod
    def const(c, n, k):
        c = np.broadcast_to(_arr(c), (n,)).copy()
        z = np.zeros((n, k))
        return D(c, z, np.abs(c), z.copy())

    @staticmethod
    def seed(v, k, j):
        """Independent variable number ``j`` of ``k``."""
        v = _arr(v)
        g = np.zeros((v.shape[0], k))
        g[:, j] = 1.0
        return D(v, g, np.abs(v), g.copy())

    @property
    def n(self):
        return self.v.shape[0]

    @property
    def k(self):
        return self.g.shape[1]

    def _lift(self, o):
        if isinstance(o, D):
            return o
        return D.const(o, self.n, self.k)

    def embed(self, k, offset):
        """Same number seen as a function of ``k`` variables: the current
        derivative block moves to columns ``offset .. offset+self.k``."""
        g = np.zeros((self.n, k), dtype=self.g.dtype)
        gm = np.zeros((self.n, k))
        g[:, offset:offset + self.k] = self.g
        gm[:, offset:offset + self.k] = self.gm
        return D(self.v.copy(), g, self.m.copy(), gm)

    def take(self, idx):
        return D(self.v[idx], self.g[idx], self.m[idx], self.gm[idx])

    # --------------------------------------------------------------- arithmetic
    def __add__(self, o):
        o = self._lift(o)
        return D(self.v + o.v, self.g + o.g, self.m + o.m, self.gm + o.gm)

    __radd__ = __add__

    def __sub__(self, o):
        o = self._lift(o)
        return D(self.v - o.v, self.g - o.g, self.m + o.m, self.gm + o.gm)

    def __rsub__(self, o):
        return self._lift(o) - self

    def __neg__(self):
        return D(-self.v, -self.g, self.m, self.gm)

    def __mul__(self, o):
        o = self._lift(o)
        v = self.v * o.v
        g = self.g * o.v[:, None] + self.v[:, None] * o.g
        m = self.m * o.m
        gm = self.gm * o.m[:, None] + self.m[:, None] * o.gm
        return D(v, g, m, gm)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = self._lift(o)
        v = self.v / o.v
        g = (self.g - v[:, None] * o.g) / o.v[:, None]
        ao = np.abs(o.v)
        m = self.m / ao
        gm = self.gm / ao[:, None] + (self.m / (ao * ao))[:, None] * o.gm
        return D(v, g, m, gm)

    def __rtruediv__(self, o):
        return self._lift(o) / self

    def __pow__(self, e):
        """Real, constant exponent ``e >= 1`` (used on clamped, non-negative
        bases only)."""
        e = float(e)
        v = self.v ** e
        dv = e * self.v ** (e - 1.0)
        m = self.m ** e
        dm = e * self.m ** (e - 1.0)
        return D(v, dv[:, None] * self.g, m, dm[:, None] * self.gm)


def where(cond, a: D, b: D) -> D:
    """Element-wise choice between two dual numbers (value-driven branch)."""
    c = np.asarray(cond, dtype=bool)
    return D(np.where(c, a.v, b.v), np.where(c[:, None], a.g, b.g),
             np.where(c, a.m, b.m), np.where(c[:, None], a.gm, b.gm))
