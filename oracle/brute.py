"""Brute-force cross-checks of the MTP-SAT oracle (test infrastructure only).

Two solvers that reach the same PDE by other routes than the tent scheme:

* ``GlobalDG`` + ``rk4_global``: the standard (non-tent) method of lines for Maxwell's
  system d_t g(u) + div f(u) = 0 (Sec. 3) on the whole mesh at a flat front: upwind DG
  in space (the same flux definition, interior and PEC, with delta = 1 everywhere and no
  mapping), classical RK4 in time with a small step.  Every element and facet integral
  here is computed by Duffy-collapsed Gauss-Legendre quadrature, and facet points are
  matched between neighbours through physical coordinates, so no integral table or facet
  parametrisation is shared with the tent assembly (which integrates barycentric
  monomials exactly).  Both discretisations converge to the exact solution at
  O(h^{p+1}), so their distance shrinks at that rate (they are different discretisations:
  the distance is not round-off).

* ``substituted_rk4_tent`` / ``evolve_substituted_rk4``: the straightforward approach the
  paper sets against SAT (Sec. 3, the paragraph after eq. equ_ode): substitute Y = M U and
  integrate d/dt Y = A M(t)^-1 Y on each tent with the classical Runge-Kutta method
  (Sec. 5.1, Fig. 3 right, reports that its convergence stagnates at first order).  It
  uses the tent operators of ``mtp.Discretization``; only the time stepping differs.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import maxwell as mx
from .mesh import Mesh
from .simplex import bernstein_eval, duffy_rule, multi_indices, multinom


def bernstein_grad_lambda(lam, p):
    """dB_alpha / d lambda_i at barycentric points lam [Q, d+1] -> [Q, N_p, d+1]
    (B_alpha = p!/alpha! lambda^alpha, so dB_alpha/dlambda_i = alpha_i p!/alpha! lambda^(alpha - e_i))."""
    lam = np.asarray(lam, float)
    nv = lam.shape[-1]
    al = multi_indices(nv, p)
    c = multinom(al)
    out = np.zeros(lam.shape[:-1] + (len(al), nv))
    for i in range(nv):
        expo = al.copy()
        expo[:, i] -= 1
        val = np.ones(lam.shape[:-1] + (len(al),))
        for k in range(nv):
            val = val * lam[..., k:k + 1] ** np.maximum(expo[:, k], 0)
        out[..., i] = c * al[:, i] * val          # alpha_i = 0 gives 0
    return out


class GlobalDG:
    """Upwind DG semi-discretisation M dU/dt = A U on the whole mesh (flat front, delta = 1).

    Unknowns U[e][r][a]: Bernstein coefficients of field r (2D TE: Ex, Ey, Hz; 3D: E, H) on
    element e.  M = diag(eps | mu per field) (x) element mass;
    (A U) . v = sum_T int_T f(u) : grad v  -  sum_T sum_{F in dT} int_F F*_T(u-, u+) . v
    with the upwind flux against the neighbour and the PEC flux on the boundary (Sec. 3)."""

    def __init__(self, mesh: Mesh, p: int):
        self.mesh, self.p = mesh, p
        d = self.d = mesh.dim
        self.fs = mx.fields_for_dim(d)
        nf = self.nf = len(self.fs)
        nb = self.nb = len(multi_indices(d + 1, p))
        ne = mesh.ne
        N = nf * nb
        qe = p + 2                                       # exact for degree <= 2p + 4 - d
        lam, w = duffy_rule(d, qe)
        B = bernstein_eval(lam, p)                       # [Q, nb]
        dB = bernstein_grad_lambda(lam, p)               # [Q, nb, d+1]
        Ften = mx.flux_tensor()                          # f(u)[r, k] = F[r, k, s] u[s]
        rows, cols, vals = [], [], []
        mass_blocks = []

        def add(e1, e2, blk):
            r0, c0 = e1 * N, e2 * N
            ii, jj = np.nonzero(blk)
            rows.append(r0 + ii)
            cols.append(c0 + jj)
            vals.append(blk[ii, jj])

        # facet rule: (d-1)-simplex Gauss rule on the facet's own barycentrics
        if d == 2:
            fl, fw = duffy_rule(1, p + 2)
        else:
            fl, fw = duffy_rule(2, p + 2)
        for e in range(ne):
            vol = mesh.vol[e]
            gl = mesh.grad_lam[e]                        # [d+1, d]
            Mloc = vol * np.einsum("q,qa,qb->ab", w, B, B)
            mat = np.array([mesh.eps[e] if r < 3 else mesh.mu[e] for r in self.fs])
            mass_blocks.append(np.kron(np.diag(mat), Mloc))
            # volume: int_T f(u) : grad v  ->  sum_k F[r, k, s] int_T B_b d_k B_a
            gradB = np.einsum("qai,ik->qak", dB, gl)     # physical gradients [Q, nb, d]
            K = vol * np.einsum("q,qb,qak->kab", w, B, gradB)
            blk = np.zeros((N, N))
            for k in range(d):
                blk += np.kron(Ften[np.ix_(self.fs, [k], self.fs)][:, 0, :], K[k])
            # facets: - int_F F*_T . v
            verts = mesh.verts[mesh.elems[e]]
            for f in range(d + 1):
                n = np.zeros(3)
                n[:d] = mesh.normal[e, f]
                keep = [i for i in range(d + 1) if i != f]
                lam_e = np.zeros((len(fw), d + 1))
                lam_e[:, keep] = fl
                X = lam_e @ verts                        # physical facet points
                Be = bernstein_eval(lam_e, p)            # [Qf, nb]
                area = mesh.face_area[e, f]
                own = area * np.einsum("q,qa,qb->ab", fw, Be, Be)
                e2 = int(mesh.nbr[e, f])
                if e2 < 0:
                    C = mx.pec_matrix(n, math.sqrt(mesh.mu[e] / mesh.eps[e]))
                    blk -= np.kron(C[np.ix_(self.fs, self.fs)], own)
                    continue
                Cm, Cp = mx.flux_matrices(n, math.sqrt(mesh.mu[e] / mesh.eps[e]),
                                          math.sqrt(mesh.mu[e2] / mesh.eps[e2]))
                blk -= np.kron(Cm[np.ix_(self.fs, self.fs)], own)
                lam2 = self._barycentric(e2, X)
                B2 = bernstein_eval(lam2, p)
                cross = area * np.einsum("q,qa,qb->ab", fw, Be, B2)
                add(e, e2, -np.kron(Cp[np.ix_(self.fs, self.fs)], cross))
            add(e, e, blk)
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(ne * N, ne * N))
        inv_rows, inv_cols, inv_vals = [], [], []
        for e, Mb in enumerate(mass_blocks):
            ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
            inv_rows.append(e * N + ii.ravel())
            inv_cols.append(e * N + jj.ravel())
            inv_vals.append(np.linalg.inv(Mb).ravel())
        self.Minv = sp.csr_matrix((np.concatenate(inv_vals), (np.concatenate(inv_rows), np.concatenate(inv_cols))),
                                  shape=(ne * N, ne * N))
        self.mass_blocks = mass_blocks

    def _barycentric(self, e, X):
        """Barycentric coordinates of physical points X [Q, d] in element e."""
        m = self.mesh
        v0 = m.verts[m.elems[e, 0]]
        gl = m.grad_lam[e]                               # rows: grad lambda_0..d
        lam = np.empty((len(X), self.d + 1))
        lam[:, 1:] = (X - v0) @ gl[1:].T
        lam[:, 0] = 1.0 - lam[:, 1:].sum(1)
        return lam

    def project(self, fn, t=0.0):
        """L2 projection of the fields (E, H) = fn(x, t) -> U [ne, nf, nb]."""
        m, d, p = self.mesh, self.d, self.p
        lam, w = duffy_rule(d, p + 8)
        B = bernstein_eval(lam, p)
        X = np.einsum("qi,eid->eqd", lam, m.verts[m.elems])
        E, H = fn(X, t)
        u = np.concatenate([E, H], -1)[..., self.fs]     # [ne, Q, nf]
        U = np.empty((m.ne, self.nf, self.nb))
        for e in range(m.ne):
            Mloc = m.vol[e] * np.einsum("q,qa,qb->ab", w, B, B)
            rhs = m.vol[e] * np.einsum("q,qa,qr->ra", w, B, u[e])
            U[e] = np.linalg.solve(Mloc, rhs.T).T
        return U

    def rate(self, U):
        """dU/dt = M^-1 A U."""
        return self.Minv @ (self.A @ U)

    def l2_error(self, U, fn, t):
        m, d, p = self.mesh, self.d, self.p
        lam, w = duffy_rule(d, p + 8)
        B = bernstein_eval(lam, p)
        X = np.einsum("qi,eid->eqd", lam, m.verts[m.elems])
        E, H = fn(X, t)
        u = np.concatenate([E, H], -1)[..., self.fs]
        uh = np.einsum("qa,era->eqr", B, U)
        return math.sqrt(float((np.einsum("eqr,q->e", (uh - u) ** 2, w) * m.vol).sum()))

    def energy(self, U):
        """(1/2) U . M U = (1/2) int eps |E|^2 + mu |H|^2."""
        x = U.reshape(self.mesh.ne, -1)
        return 0.5 * sum(float(x[e] @ Mb @ x[e]) for e, Mb in enumerate(self.mass_blocks))


def rk4_global(dg: GlobalDG, U0, T, n_steps):
    """Classical RK4 with n_steps equal steps on dU/dt = M^-1 A U from 0 to T."""
    h = T / n_steps
    x = np.asarray(U0, float).reshape(-1).copy()
    for _ in range(n_steps):
        k1 = dg.rate(x)
        k2 = dg.rate(x + 0.5 * h * k1)
        k3 = dg.rate(x + 0.5 * h * k2)
        k4 = dg.rate(x + h * k3)
        x += h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return x.reshape(np.shape(U0))


# ---------------------------------------------------------------------------------------
# the Y-substituted classical RK4 tent stepper (the approach SAT replaces)
# ---------------------------------------------------------------------------------------
def substituted_rk4_tent(disc, V, dt, tau, Ypatch, msub):
    """Sec. 3 after eq. equ_ode: d/dt Y = A M(t)^-1 Y on the tent at V (t in [0, 1]),
    integrated with msub classical RK4 steps; M(t) = M(0) + t M' as in the tent assembly.
    Returns (patch slots, tent-top Y)."""
    slots, M0, Mp, A = disc.tent_operators(V, dt, tau)
    ns = len(slots)

    def f(t, Y):
        U = np.stack([np.linalg.solve(M0[k] + t * Mp[k], Y[k]) for k in range(ns)])
        out = np.zeros_like(U)
        for (a, b), blk in A.items():
            out[a] += blk @ U[b]
        return out

    h = 1.0 / msub
    Y = np.array(Ypatch, float)
    for i in range(msub):
        t = i * h
        k1 = f(t, Y)
        k2 = f(t + 0.5 * h, Y + 0.5 * h * k1)
        k3 = f(t + 0.5 * h, Y + 0.5 * h * k2)
        k4 = f(t + h, Y + h * k3)
        Y = Y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return slots, Y


def evolve_substituted_rk4(disc, Y, tents, msub):
    """Every tent in (layer, vertex) order with ``substituted_rk4_tent`` (global state Y)."""
    m = disc.mesh
    Y = np.array(Y, float).reshape(m.ne, disc.nf * disc.nb)
    tau = np.zeros(m.nv)
    for t in range(len(tents["vertex"])):
        V = int(tents["vertex"][t])
        tb, tt = float(tents["t_bot"][t]), float(tents["t_top"][t])
        slots, Yp = substituted_rk4_tent(disc, V, tt - tb, tau, Y[m.patch[V]], msub)
        Y[slots] = Yp
        tau[V] = tt
    return Y.reshape(m.ne, disc.nf, disc.nb)


def rk4_order_table(ps=(1, 2, 3, 4), ns=(2, 4, 8, 16), T=0.25, cf=0.5):
    """Rows (p, n, SAT error vs the exact TE cavity mode, distance between the Y-substituted RK4
    and the SAT results on the same tents) for the 2D convergence study of Sec. 5.1."""
    import mtp_synth as S
    from .mtp import Discretization
    from .pitch import pitch_tents
    zero = lambda X, t: (np.zeros(X.shape[:-1] + (3,)), np.zeros(X.shape[:-1] + (3,)))
    rows = []
    for p in ps:
        for n in ns:
            w = S.te_square(n, p, T)
            disc = Discretization(Mesh(w.verts, w.elems, w.eps, w.mu), p)
            tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, cf)
            Y0 = disc.project_initial(w.init)
            Ys, _ = disc.evolve(Y0, tents)
            Yr = evolve_substituted_rk4(disc, Y0, tents, 2 * p)
            Us, Ur = disc.fields_at_flat_front(Ys), disc.fields_at_flat_front(Yr)
            rows.append((p, n, disc.l2_error(Us, w.exact, w.T), disc.l2_error(Ur, w.exact, w.T),
                         disc.l2_error(Ur - Us, zero, 0.0)))
    return rows


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="2D TE cavity: SAT vs Y-substituted classical RK4 on the same tents")
    ap.add_argument("--p", default="1,2,3,4")
    ap.add_argument("--n", default="2,4,8,16")
    args = ap.parse_args()
    rows = rk4_order_table([int(x) for x in args.p.split(",")], [int(x) for x in args.n.split(",")])
    print("| p | n | SAT error | RK4 error | RK4 - SAT |")
    print("|---|---|---|---|---|")
    for p, n, es, er, d in rows:
        print(f"| {p} | {n} | {es:.3e} | {er:.3e} | {d:.3e} |")
