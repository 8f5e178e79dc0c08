"""Second-order forward-mode differentiation on batches (oracle; test
infrastructure only).

A ``Jet`` carries, for a batch of B independent evaluation points, a value
array ``v`` of shape (B, *S), its gradient ``g`` of shape (B, *S, n) and its
Hessian ``H`` of shape (B, *S, n, n) with respect to n seed variables. Only
the sum, product and reciprocal rules are used, so every derivative the
oracle reports is the exact derivative of the value computation (no
truncation, no finite differences). ``H`` is None for first-order jets.
"""
from __future__ import annotations

import numpy as np


class Jet:
    __slots__ = ("v", "g", "H")
    # keep numpy from broadcasting a Jet as an object array: ndarray * Jet
    # must dispatch to Jet.__rmul__
    __array_ufunc__ = None

    def __init__(self, v, g, H=None):
        self.v = v
        self.g = g
        self.H = H

    # ---- construction -------------------------------------------------
    @staticmethod
    def variables(values: np.ndarray, n: int, first: int, order: int) -> "Jet":
        """Seed jets for values of shape (B, *S); entry s (flattened over S)
        is seed variable ``first + s`` out of ``n``."""
        B = values.shape[0]
        S = values.shape[1:]
        m = int(np.prod(S)) if S else 1
        g = np.zeros((B, m, n))
        g[:, np.arange(m), first + np.arange(m)] = 1.0
        g = g.reshape((B,) + S + (n,))
        H = np.zeros((B,) + S + (n, n)) if order >= 2 else None
        return Jet(np.array(values, dtype=np.float64), g, H)

    @staticmethod
    def const(values: np.ndarray, n: int, order: int) -> "Jet":
        values = np.asarray(values, dtype=np.float64)
        g = np.zeros(values.shape + (n,))
        H = np.zeros(values.shape + (n, n)) if order >= 2 else None
        return Jet(values, g, H)

    @property
    def order(self) -> int:
        return 2 if self.H is not None else 1

    @property
    def n(self) -> int:
        return self.g.shape[-1]

    # ---- helpers -------------------------------------------------------
    def __getitem__(self, idx) -> "Jet":
        """Index the value shape S (the batch axis is kept): ``J[..., i, j]``."""
        if not isinstance(idx, tuple):
            idx = (idx,)
        full = (slice(None),) + idx
        return Jet(self.v[full], self.g[full], None if self.H is None else self.H[full])

    def __neg__(self):
        return Jet(-self.v, -self.g, None if self.H is None else -self.H)

    def __add__(self, o):
        if isinstance(o, Jet):
            return Jet(self.v + o.v, self.g + o.g, None if self.H is None else self.H + o.H)
        return Jet(self.v + o, self.g, self.H)

    __radd__ = __add__

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        """Elementwise product (value shapes broadcast like numpy)."""
        if not isinstance(o, Jet):
            c = np.asarray(o, dtype=np.float64)
            return Jet(self.v * c, self.g * c[..., None],
                       None if self.H is None else self.H * c[..., None, None])
        v = self.v * o.v
        g = self.v[..., None] * o.g + o.v[..., None] * self.g
        H = None
        if self.H is not None:
            H = (self.v[..., None, None] * o.H + o.v[..., None, None] * self.H
                 + self.g[..., :, None] * o.g[..., None, :] + o.g[..., :, None] * self.g[..., None, :])
        return Jet(v, g, H)

    __rmul__ = __mul__

    def reciprocal(self) -> "Jet":
        """1/x by the quotient rule."""
        r = 1.0 / self.v
        g = -(r * r)[..., None] * self.g
        H = None
        if self.H is not None:
            H = (2.0 * (r ** 3))[..., None, None] * self.g[..., :, None] * self.g[..., None, :] \
                - (r * r)[..., None, None] * self.H
        return Jet(r, g, H)

    def sqrt(self) -> "Jet":
        """sqrt(x) by the chain rule (x > 0)."""
        r = np.sqrt(self.v)
        d1 = 0.5 / r
        g = d1[..., None] * self.g
        H = None
        if self.H is not None:
            d2 = -0.25 / (r * self.v)
            H = d1[..., None, None] * self.H + d2[..., None, None] * self.g[..., :, None] * self.g[..., None, :]
        return Jet(r, g, H)

    def __truediv__(self, o):
        if isinstance(o, Jet):
            return self * o.reciprocal()
        return self * (1.0 / np.asarray(o, dtype=np.float64))

    def sum(self, axis: int) -> "Jet":
        """Sum over value axis ``axis`` (0-based within S)."""
        a = axis + 1
        return Jet(self.v.sum(axis=a), self.g.sum(axis=a), None if self.H is None else self.H.sum(axis=a))


def stack(jets, axis: int = 0) -> Jet:
    """Stack jets of equal value shape along a new value axis."""
    a = axis + 1
    v = np.stack([j.v for j in jets], axis=a)
    g = np.stack([j.g for j in jets], axis=a)
    H = None if jets[0].H is None else np.stack([j.H for j in jets], axis=a)
    return Jet(v, g, H)


def where_negative(x: Jet) -> np.ndarray:
    return x.v < 0.0


# ---- 3x3 matrix operations on jets of value shape (3, 3) -----------------

def mat(rows) -> Jet:
    """Build a (3,3) matrix jet from a 3x3 nested list of scalar jets."""
    return stack([stack(list(r), axis=0) for r in rows], axis=0)


def entry(A: Jet, i: int, j: int) -> Jet:
    return A[i, j]


def matmul(A, B) -> Jet:
    """C_ik = sum_j A_ij B_jk for 3x3 matrices; either factor may be a
    constant array of shape (3,3) or (B,3,3)."""
    rows = []
    for i in range(3):
        row = []
        for k in range(3):
            acc = None
            for j in range(3):
                a = A[i, j] if isinstance(A, Jet) else _const_entry(A, i, j)
                b = B[j, k] if isinstance(B, Jet) else _const_entry(B, j, k)
                t = a * b
                acc = t if acc is None else acc + t
            row.append(acc)
        rows.append(row)
    return mat(rows)


def _const_entry(C, i, j):
    C = np.asarray(C)
    return C[..., i, j]


def transpose(A: Jet) -> Jet:
    v = np.swapaxes(A.v, 1, 2)
    g = np.swapaxes(A.g, 1, 2)
    H = None if A.H is None else np.swapaxes(A.H, 1, 2)
    return Jet(v, g, H)


def det3(A: Jet) -> Jet:
    """Determinant by cofactor expansion along the first row."""
    a = lambda i, j: A[i, j]  # noqa: E731
    return (a(0, 0) * (a(1, 1) * a(2, 2) - a(1, 2) * a(2, 1))
            - a(0, 1) * (a(1, 0) * a(2, 2) - a(1, 2) * a(2, 0))
            + a(0, 2) * (a(1, 0) * a(2, 1) - a(1, 1) * a(2, 0)))


def inv3(A: Jet) -> Jet:
    """Inverse as adjugate / determinant (the classical cofactor formula)."""
    a = lambda i, j: A[i, j]  # noqa: E731
    c = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            r = [x for x in range(3) if x != i]
            s = [x for x in range(3) if x != j]
            minor = a(r[0], s[0]) * a(r[1], s[1]) - a(r[0], s[1]) * a(r[1], s[0])
            c[i][j] = minor if (i + j) % 2 == 0 else -minor
    rdet = det3(A).reciprocal()
    # inverse_ij = cofactor_ji / det
    return mat([[c[j][i] * rdet for j in range(3)] for i in range(3)])


def trace(A: Jet) -> Jet:
    return A[0, 0] + A[1, 1] + A[2, 2]
