"""The scan formulation of a block bi-diagonal system (Section II-B), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The recursion x_0 = c_0, x_i = b_{i-1} x_{i-1} + c_i is the bi-diagonal system of
Section II-B. Each step becomes the homogeneous matrix a_i = [[b_{i-1}, c_i],
[0, 1]] (a_0 = [[1, c_0], [0, 1]]), and a_{i-1} (+) a_i is the product a_i a_{i-1};
the inclusive scan of the a_i then carries x_i in its last column. The balanced
tree (Blelloch) schedule of the same scan is written out so that the tests can
check that re-association leaves the result unchanged.
"""
from __future__ import annotations

import numpy as np


def serial_recursion(b, c):
    """x_0 = c_0, x_i = b_{i-1} x_{i-1} + c_i.  b: [n-1, m, m] (b[i] = b_i), c: [n, m]."""
    n, m = c.shape
    x = np.empty_like(c)
    x[0] = c[0]
    for i in range(1, n):
        x[i] = b[i - 1] @ x[i - 1] + c[i]
    return x


def operators(b, c):
    """The homogeneous matrices a_i, [n, m+1, m+1]."""
    n, m = c.shape
    a = np.zeros((n, m + 1, m + 1))
    a[:, m, m] = 1.0
    a[0, :m, :m] = np.eye(m)
    a[1:, :m, :m] = b
    a[:, :m, m] = c
    return a


def combine(left, right):
    """left (+) right = right @ left (the operator of Section II-B)."""
    return right @ left


def inclusive_scan_serial(a):
    out = np.empty_like(a)
    out[0] = a[0]
    for i in range(1, a.shape[0]):
        out[i] = combine(out[i - 1], a[i])
    return out


def inclusive_scan_blelloch(a):
    """Balanced binary tree scan (up-sweep, down-sweep), then made inclusive."""
    n, k, _ = a.shape
    size = 1
    while size < n:
        size *= 2
    ident = np.eye(k)
    t = np.concatenate([a, np.broadcast_to(ident, (size - n, k, k))], axis=0).copy()
    d = 1
    while d < size:                       # up-sweep
        for i in range(2 * d - 1, size, 2 * d):
            t[i] = combine(t[i - d], t[i])
        d *= 2
    t[size - 1] = ident
    d = size // 2
    while d >= 1:                         # down-sweep (exclusive result)
        for i in range(2 * d - 1, size, 2 * d):
            left = t[i - d].copy()
            t[i - d] = t[i]
            t[i] = combine(t[i], left)
        d //= 2
    return np.stack([combine(t[i], a[i]) for i in range(n)])


def solve_by_scan(b, c, schedule="serial"):
    a = operators(b, c)
    s = inclusive_scan_serial(a) if schedule == "serial" else inclusive_scan_blelloch(a)
    m = c.shape[1]
    return s[:, :m, m]
