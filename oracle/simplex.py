"""Polynomial tools on simplices for the oracle (test infrastructure only).

V_h is the discontinuous space of degree-p polynomials per element (Sec. 3, the
DG space).  The oracle represents it in the Bernstein basis
    B_alpha = p!/alpha! * lambda^alpha,   |alpha| = p,
with lambda the element's barycentric coordinates.  Every bilinear form the
method needs is then an integral of a barycentric monomial times constants, and
    int_T lambda^gamma dx = |T| d! gamma! / (|gamma| + d)!
is exact (no quadrature).  Non-polynomial data (initial fields, exact solutions
in error norms) use a Duffy-collapsed tensor Gauss-Legendre rule.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def multi_indices(nvert: int, p: int):
    """All alpha in N^nvert with |alpha| = p, in a fixed (lexicographic) order."""
    out = [a for a in itertools.product(range(p + 1), repeat=nvert) if sum(a) == p]
    out.sort(reverse=True)
    return np.array(out, np.int64)


def factorial_vec(a):
    return np.vectorize(math.factorial, otypes=[float])(np.asarray(a))


def multinom(alpha):
    """p!/alpha! per row of alpha."""
    alpha = np.atleast_2d(alpha)
    p = alpha.sum(1)
    return factorial_vec(p) / np.prod(factorial_vec(alpha), axis=1)


def monomial_integral(gamma, d):
    """int over a d-simplex of measure 1 of lambda^gamma: d! gamma! / (|gamma| + d)!.
    gamma: [..., d+1] integer exponents."""
    gamma = np.asarray(gamma)
    num = math.factorial(d) * np.prod(factorial_vec(gamma), axis=-1)
    den = factorial_vec(gamma.sum(-1) + d)
    return num / den


def bernstein_eval(lam, p):
    """B_alpha(lambda) for barycentric points lam [..., d+1] -> [..., N_p]."""
    lam = np.asarray(lam, float)
    al = multi_indices(lam.shape[-1], p)
    c = multinom(al)
    vals = np.ones(lam.shape[:-1] + (len(al),))
    for i in range(lam.shape[-1]):
        vals = vals * lam[..., i:i + 1] ** al[:, i]
    return vals * c


# --------------------------------------------------------------------------
# Duffy-collapsed Gauss-Legendre rules on the unit simplex (projection / norms)
# --------------------------------------------------------------------------
@lru_cache(maxsize=None)
def duffy_rule(d: int, n: int):
    """Points (barycentric, [Q, d+1]) and weights summing to 1 (i.e. for a simplex of
    unit measure) of the collapsed n^d Gauss-Legendre rule.  Exact for total degree
    <= 2n - d (the collapse adds up to d-1 powers of the collapsed variable)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    if d == 1:
        lam = np.stack([1 - x, x], -1)
        return lam, w.copy()
    if d == 2:
        pts, wts = [], []
        for i in range(n):
            for j in range(n):
                u, v = x[i], x[j]
                # (u, v) in unit square -> (s, t) = (u (1 - v), v) in unit triangle
                s, t = u * (1 - v), v
                pts.append([1 - s - t, s, t])
                wts.append(w[i] * w[j] * (1 - v))
        wts = np.array(wts)
        return np.array(pts), wts / wts.sum()
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                u, v, z = x[i], x[j], x[k]
                s = u * (1 - v) * (1 - z)
                t = v * (1 - z)
                r = z
                pts.append([1 - s - t - r, s, t, r])
                wts.append(w[i] * w[j] * w[k] * (1 - v) * (1 - z) ** 2)
    wts = np.array(wts)
    return np.array(pts), wts / wts.sum()
