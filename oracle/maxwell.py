"""Maxwell pieces of the MTP scheme, pointwise (test infrastructure only).

Sec. 3: u = (E, H), g(u) = (eps E, mu H), f(u) = [-skew H ; skew E] (6 x 3), with
skew E the 3x3 matrix whose row-wise divergence is curl E.  The conservation law
d_t g(u) + div f(u) = 0 is Maxwell's system  d_t(eps E) = curl H, d_t(mu H) = -curl E.
After the tent map Phi (Sec. 3, transformed equation) the time-differentiated
quantity is g(u) - f(u) grad(phi) and the flux is delta f(u).

Readings of the paper used here:
* Numerical flux (Sec. 3, upwind flux).  The printed flux is for unit impedance and
  its facet term's sign convention does not match element-wise integration by
  parts.  We use, per element with outward unit normal n, interior trace (-) and
  exterior trace (+), the exact Riemann (upwind) flux for piecewise-constant
  eps, mu with impedance Z = sqrt(mu/eps):
      H* x n = (Z- H- x n + Z+ H+ x n + E-_t - E+_t) / (Z- + Z+)
      E*_t   = (Z+ E-_t + Z- E+_t + Z+ Z- (H- - H+) x n) / (Z- + Z+)
      F*     = [ H* x n ; -E* x n ]          (approximates f(u) n = [H x n ; -E x n])
  which for Z = 1 is {H} x n + (E-_t - E+_t)/2, -{E} x n + (H-_t - H+_t)/2, the
  upwind flux the paper cites.
* PEC boundary: mirror state E+ = -E-, H+ = H-, Z+ = Z-, giving E*_t = 0 and
  H* x n = H- x n + E-_t / Z.
"""
from __future__ import annotations

import numpy as np


def cross(a, b):
    """a x b for 3-vectors."""
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def skew(v):
    """The 3x3 matrix with (skew v) w = w x v, so div(skew E) (row-wise) = curl E (Sec. 3)."""
    x, y, z = v
    return np.array([[0.0, z, -y], [-z, 0.0, x], [y, -x, 0.0]])


def g_of(u, eps, mu):
    """g(u) = (eps E, mu H)."""
    return np.concatenate([eps * u[:3], mu * u[3:]])


def f_of(u):
    """f(u) = [-skew H ; skew E], a 6 x 3 matrix."""
    return np.vstack([-skew(u[3:]), skew(u[:3])])


def mass_pointwise(u, grad_phi, eps, mu):
    """The time-differentiated quantity of the transformed equation: g(u) - f(u) grad(phi)
    (Sec. 3).  Equals (eps E - H x grad phi, mu H + E x grad phi)."""
    return g_of(u, eps, mu) - f_of(u) @ np.asarray(grad_phi, float)


def mass_matrix_6(grad_phi, eps, mu):
    """6x6 matrix G with G u = g(u) - f(u) grad(phi), built by applying the map to unit vectors."""
    G = np.zeros((6, 6))
    for s in range(6):
        e = np.zeros(6)
        e[s] = 1.0
        G[:, s] = mass_pointwise(e, grad_phi, eps, mu)
    return G


def mass_inverse_closed_form(w, grad_phi, eps, mu):
    """Closed-form solution u of G u = w (end of Sec. 4):
    E = (eps mu - |g|^2)^-1 (I - g g^T/(eps mu)) (mu w_E + w_H x g),
    H = (eps mu - |g|^2)^-1 (I - g g^T/(eps mu)) (eps w_H - w_E x g),  g = grad(phi)."""
    g = np.asarray(grad_phi, float)
    wE, wH = w[:3], w[3:]
    P = np.eye(3) - np.outer(g, g) / (eps * mu)
    s = 1.0 / (eps * mu - g @ g)
    E = s * P @ (mu * wE + cross(wH, g))
    H = s * P @ (eps * wH - cross(wE, g))
    return np.concatenate([E, H])


def tangential(v, n):
    """v_t = -(v x n) x n."""
    return -cross(cross(v, n), n)


def upwind_flux(um, up, n, Zm, Zp):
    """Numerical flux F*(u-, u+) approximating f(u) n for outward normal n (see module doc)."""
    n = np.asarray(n, float)
    Em, Hm, Ep, Hp = um[:3], um[3:], up[:3], up[3:]
    Hxn = (Zm * cross(Hm, n) + Zp * cross(Hp, n) + tangential(Em, n) - tangential(Ep, n)) / (Zm + Zp)
    Et = (Zp * tangential(Em, n) + Zm * tangential(Ep, n) + Zp * Zm * cross(Hm - Hp, n)) / (Zm + Zp)
    return np.concatenate([Hxn, -cross(Et, n)])


def pec_flux(um, n, Z):
    """Flux on a PEC facet: the upwind flux against the mirror state (E+ = -E-, H+ = H-)."""
    up = np.concatenate([-um[:3], um[3:]])
    return upwind_flux(um, up, n, Z, Z)


def flux_matrices(n, Zm, Zp):
    """6x6 matrices (Cm, Cp) with F*(u-, u+) = Cm u- + Cp u+ (the flux is linear)."""
    Cm, Cp = np.zeros((6, 6)), np.zeros((6, 6))
    z = np.zeros(6)
    for s in range(6):
        e = np.zeros(6)
        e[s] = 1.0
        Cm[:, s] = upwind_flux(e, z, n, Zm, Zp)
        Cp[:, s] = upwind_flux(z, e, n, Zm, Zp)
    return Cm, Cp


def pec_matrix(n, Z):
    C = np.zeros((6, 6))
    for s in range(6):
        e = np.zeros(6)
        e[s] = 1.0
        C[:, s] = pec_flux(e, n, Z)
    return C


def flux_tensor():
    """F[r, k, s] with f(u)[r, k] = sum_s F[r, k, s] u[s]."""
    F = np.zeros((6, 3, 6))
    for s in range(6):
        e = np.zeros(6)
        e[s] = 1.0
        F[:, :, s] = f_of(e)
    return F


# 2D TE fields (Ex, Ey, Hz) inside the 6-vector (Ex, Ey, Ez, Hx, Hy, Hz)
TE_FIELDS = np.array([0, 1, 5])
ALL_FIELDS = np.arange(6)


def fields_for_dim(dim):
    return TE_FIELDS if dim == 2 else ALL_FIELDS
