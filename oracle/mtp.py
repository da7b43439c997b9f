"""Per-tent MTP discretization and SAT time stepping, FP64 (test infrastructure only).

Follows the paper step by step:

* Sec. 3 (tent map):  phi(x, t) = (1 - t) phi_b(x) + t phi_t(x), delta = phi_t - phi_b.
  For the tent at vertex V, phi_t - phi_b = (t_top - t_bot) lambda_V, so on every
  element T of the patch grad(phi)(t) = grad(phi_b) + t * dt * grad(lambda_V) is constant.
* Sec. 3 (semi-discrete system, eq. d/dt[M U] - A U = 0) on the patch omega_V with
      (M(t) U) . v = int g(u) - f(u) grad(phi) . v
      (A U) . v   = sum_T int_T delta f(u) : grad v  -  sum_T sum_{F in dT, V in F} int_F delta F*_T . v
  (the facet term only over facets containing V: delta = dt lambda_V vanishes on
  the others).  F*_T is the upwind / PEC flux of ``maxwell`` with T's outward normal.
* Sec. 4 (SAT, eqs. taylor_pol, coeff_rec, recursion-init):  m sub-intervals,
  q stages; per sub-interval i
      M_i U_{i,0} = Y_{i,0};   Y_{i,n} = A U_{i,n-1} (1 <= n <= q);
      M_i U_{i,n} = Y_{i,n} - n M' U_{i,n-1} (1 <= n <= q-1);
      Y_{i+1,0}   = sum_{n=0..q} (1/m)^n / n! Y_{i,n}.
  M_i is solved by dense LU of each element's block (the closed form of Sec. 4 is an
  independent check in the tests).
* Sec. 3/4 (hand-off): the tent top value Y_{m-1}(1) is the next tent's bottom
  value; the global state is Y (the moments of g(u) - f(u) grad(phi)) per element.

The state is stored as Bernstein moments Y[e][field][a] = int_T y_field B_a.
The polynomial y = M_T^{-1} Y is the "conserved variable" field; at a flat front
y = (eps E, mu H).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import maxwell as mx
from .mesh import Mesh
from .simplex import (bernstein_eval, duffy_rule, monomial_integral, multi_indices, multinom)


def dof_counts(dim, p):
    nb = (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6
    nf = 3 if dim == 2 else 6
    return nf, nb


class Discretization:
    """DG space of degree p on a mesh, Bernstein basis, exact element/facet integrals."""

    def __init__(self, mesh: Mesh, p: int):
        self.mesh, self.p = mesh, p
        d = self.d = mesh.dim
        self.fs = mx.fields_for_dim(d)
        self.nf, self.nb = len(self.fs), dof_counts(d, p)[1]
        al = self.alpha = multi_indices(d + 1, p)
        c = self.c = multinom(al)
        nb = self.nb
        cc = np.outer(c, c)
        # element mass on unit measure: c_a c_b int lambda^(alpha_a + alpha_b)
        self.mass_ref = cc * monomial_integral(al[:, None, :] + al[None, :, :], d)
        # volume: int lambda_j B_b d_k B_a = sum_i vol_ref[j, a, b, i] d_k lambda_i  (unit measure)
        vol_ref = np.zeros((d + 1, nb, nb, d + 1))
        eye = np.eye(d + 1, dtype=np.int64)
        for j in range(d + 1):
            for i in range(d + 1):
                g = eye[j][None, None, :] + al[None, :, :] + al[:, None, :] - eye[i][None, None, :]
                val = monomial_integral(np.maximum(g, 0), d)
                vol_ref[j, :, :, i] = cc * al[:, i][:, None] * val
        self.vol_ref = vol_ref
        # own-own facet integrals: int_F lambda_j B_a B_b on facet f (unit measure)
        fown = np.zeros((d + 1, d + 1, nb, nb))
        for f in range(d + 1):
            keep = [k for k in range(d + 1) if k != f]
            onface = (al[:, f] == 0)
            for j in range(d + 1):
                if j == f:
                    continue
                g = eye[j][None, None, :] + al[:, None, :] + al[None, :, :]
                val = monomial_integral(g[..., keep], d - 1)
                fown[j, f] = cc * val * np.outer(onface, onface)
        self.fown_ref = fown
        self.F = mx.flux_tensor()
        self._cross_cache = {}
        self._mass_lu = {}

    # ------------------------------------------------------------------
    def mass(self, e):
        return self.mesh.vol[e] * self.mass_ref

    def stiff(self, e, j):
        """K_k[a, b] = int_T lambda_j B_b d_k B_a, k = 0..d-1."""
        gl = self.mesh.grad_lam[e]                          # [d+1, d]
        return self.mesh.vol[e] * np.einsum("abi,ik->kab", self.vol_ref[j], gl)

    def face_cross(self, e, f, v):
        """C[a, b] = int_F lambda_v B^e_a B^{e2}_b with e2 the neighbour across facet f of e."""
        key = (e, f, v)
        if key in self._cross_cache:
            return self._cross_cache[key]
        m, d, al, c = self.mesh, self.d, self.alpha, self.c
        e2, f2 = int(m.nbr[e, f]), int(m.nbr_face[e, f])
        gverts = [int(x) for i, x in enumerate(m.elems[e]) if i != f]
        loc1 = [m.local_index(e, g) for g in gverts]
        loc2 = [m.local_index(e2, g) for g in gverts]
        wv = np.array([1 if g == v else 0 for g in gverts])
        g = al[:, None, loc1] + al[None, :, loc2] + wv[None, None, :]
        ok = np.outer(al[:, f] == 0, al[:, f2] == 0)
        C = np.outer(c, c) * monomial_integral(g, d - 1) * ok * m.face_area[e, f]
        self._cross_cache[key] = C
        return C

    # ------------------------------------------------------------------
    def z(self, e):
        return math.sqrt(self.mesh.mu[e] / self.mesh.eps[e])

    def flux_pair(self, e, f):
        """(Cm, Cp) of facet f of e with e's outward normal (PEC: (C, None)); cached, tent-independent."""
        key = ("flux", e, f)
        if key not in self._cross_cache:
            m = self.mesh
            n = self.emb(m.normal[e, f])
            e2 = int(m.nbr[e, f])
            if e2 >= 0:
                self._cross_cache[key] = mx.flux_matrices(n, self.z(e), self.z(e2))
            else:
                self._cross_cache[key] = (mx.pec_matrix(n, self.z(e)), None)
        return self._cross_cache[key]

    @staticmethod
    def emb(vec):
        out = np.zeros(3)
        out[: len(vec)] = vec
        return out

    def tent_operators(self, V, dt, tau):
        """Patch slots, per-element M(0), M', and the block operator A of the tent at V."""
        m, d, fs = self.mesh, self.d, self.fs
        slots = list(m.patch[V])
        slot_of = {e: k for k, e in enumerate(slots)}
        M0, Mp, A = [], [], {}
        for k, e in enumerate(slots):
            j = m.local_index(e, V)
            gl = m.grad_lam[e]
            gphi_b = self.emb(sum(tau[int(m.elems[e, i])] * gl[i] for i in range(d + 1)))
            gdelta = self.emb(dt * gl[j])
            Me = self.mass(e)
            G0 = mx.mass_matrix_6(gphi_b, m.eps[e], m.mu[e])[np.ix_(fs, fs)]
            G1 = mx.mass_matrix_6(gdelta, 0.0, 0.0)[np.ix_(fs, fs)]
            M0.append(np.kron(G0, Me))
            Mp.append(np.kron(G1, Me))
            K = self.stiff(e, j)
            blk = np.zeros((self.nf * self.nb,) * 2)
            for kk in range(d):
                blk += np.kron(self.F[np.ix_(fs, [kk], fs)][:, 0, :], dt * K[kk])
            for f in range(d + 1):
                if f == j:
                    continue
                n = self.emb(m.normal[e, f])
                Fo = m.face_area[e, f] * self.fown_ref[j, f]
                e2 = int(m.nbr[e, f])
                if e2 >= 0:
                    Cm, Cp = self.flux_pair(e, f)
                    blk -= dt * np.kron(Cm[np.ix_(fs, fs)], Fo)
                    key = (k, slot_of[e2])
                    cross = -dt * np.kron(Cp[np.ix_(fs, fs)], self.face_cross(e, f, V))
                    A[key] = A.get(key, 0) + cross
                else:
                    C = self.flux_pair(e, f)[0]
                    blk -= dt * np.kron(C[np.ix_(fs, fs)], Fo)
            A[(k, k)] = A.get((k, k), 0) + blk
        return slots, M0, Mp, A

    # ------------------------------------------------------------------
    def sat_tent(self, V, dt, tau, Ypatch, q=None, msub=None):
        """q-stage SAT with m sub-intervals on the tent at V (Sec. 4).  Ypatch: [ns, nf*nb]."""
        p = self.p
        q = p + 1 if q is None else q
        msub = 2 * p if msub is None else msub
        slots, M0, Mp, A = self.tent_operators(V, dt, tau)
        ns = len(slots)

        def apply_A(U):
            out = np.zeros_like(U)
            for (a, b), blk in A.items():
                out[a] += blk @ U[b]
            return out

        Y = Ypatch.copy()
        for i in range(msub):
            ti = i / msub
            lus = [sla.lu_factor(M0[k] + ti * Mp[k]) for k in range(ns)]
            solve = lambda R: np.stack([sla.lu_solve(lus[k], R[k]) for k in range(ns)])
            U = solve(Y)
            acc = Y.copy()
            for n in range(1, q + 1):
                Yn = apply_A(U)
                acc += (1.0 / msub) ** n / math.factorial(n) * Yn
                if n <= q - 1:
                    R = Yn - n * np.stack([Mp[k] @ U[k] for k in range(ns)])
                    U = solve(R)
            Y = acc
        return slots, Y

    # ------------------------------------------------------------------
    def evolve(self, Y, tents, tau0=None, layers=None, q=None, msub=None):
        """Apply the tents (in (layer, vertex) order) to the global state Y [ne, nf, nb].
        ``layers``: optional (begin, end) layer range; tau0: front before the first tent."""
        m = self.mesh
        Y = Y.copy().reshape(m.ne, self.nf * self.nb)
        tau = np.zeros(m.nv) if tau0 is None else np.array(tau0, float)
        lp = tents["layer_ptr"]
        lb, le = (0, len(lp) - 1) if layers is None else layers
        for t in range(int(lp[lb]), int(lp[le])):
            V = int(tents["vertex"][t])
            tb, tt = float(tents["t_bot"][t]), float(tents["t_top"][t])
            assert tau[V] == tb
            slots, Yp = self.sat_tent(V, tt - tb, tau, Y[m.patch[V]], q, msub)
            Y[slots] = Yp
            tau[V] = tt
        return Y.reshape(m.ne, self.nf, self.nb), tau

    # ------------------------------------------------------------------
    def project_initial(self, fn, t=0.0, nq=None):
        """Y at a flat front: moments of g(u0) = (eps E0, mu H0) against B_a (Sec. 4: on flat
        fronts M is the material-weighted mass matrix)."""
        m, d = self.mesh, self.d
        nq = nq or (self.p + 8)
        lam, w = duffy_rule(d, nq)
        B = bernstein_eval(lam, self.p)                      # [Q, nb]
        P = m.verts[m.elems]                                 # [ne, d+1, d]
        X = np.einsum("qi,eid->eqd", lam, P)
        E, H = fn(X, t)
        u = np.concatenate([E, H], -1)[..., self.fs]         # [ne, Q, nf]
        scale = np.where(np.isin(self.fs, [0, 1, 2]), 1.0, 0.0)
        mat = scale[None, :] * m.eps[:, None] + (1 - scale[None, :]) * m.mu[:, None]
        Y = np.einsum("eqr,q,qa->era", u, w, B) * m.vol[:, None, None]
        return Y * mat[:, :, None]

    def y_coeffs(self, Y):
        """Bernstein coefficients of the polynomial y with moments Y (y = M_T^-1 Y per element)."""
        out = np.zeros_like(Y)
        for e in range(self.mesh.ne):
            out[e] = np.linalg.solve(self.mass(e), Y[e].T).T
        return out

    def material(self):
        scale = np.isin(self.fs, [0, 1, 2])
        return np.where(scale[None, :], self.mesh.eps[:, None], self.mesh.mu[:, None])

    def fields_at_flat_front(self, Y):
        """U coefficients (E, H) at a flat front: y / (eps | mu)."""
        return self.y_coeffs(Y) / self.material()[:, :, None]

    def eval_lattice(self, coeffs):
        """Values of per-element polynomials at the sorted-vertex lattice -> [ne, N_p, nf]."""
        from mtp_synth import lattice_multi_indices
        m = self.mesh
        mi = lattice_multi_indices(self.d, self.p)
        out = np.zeros((m.ne, len(mi), self.nf))
        for e in range(m.ne):
            lam = m.barycentric_of_sorted_lattice(e, mi, self.p)
            B = bernstein_eval(lam, self.p)
            out[e] = B @ coeffs[e].T
        return out

    def moments_from_lattice(self, vals):
        """Inverse of eval_lattice followed by M_T: lattice values of y -> moments Y."""
        from mtp_synth import lattice_multi_indices
        m = self.mesh
        mi = lattice_multi_indices(self.d, self.p)
        Y = np.zeros((m.ne, self.nf, self.nb))
        for e in range(m.ne):
            lam = m.barycentric_of_sorted_lattice(e, mi, self.p)
            B = bernstein_eval(lam, self.p)
            coef = np.linalg.solve(B, vals[e])              # [nb, nf]
            Y[e] = (self.mass(e) @ coef).T
        return Y

    def l2_error(self, U, fn, t, nq=None):
        """sqrt(sum_T int_T |u_h - u|^2) over the fields of this dimension (Sec. 5)."""
        m, d = self.mesh, self.d
        nq = nq or (self.p + 8)
        lam, w = duffy_rule(d, nq)
        B = bernstein_eval(lam, self.p)
        P = m.verts[m.elems]
        X = np.einsum("qi,eid->eqd", lam, P)
        E, H = fn(X, t)
        u = np.concatenate([E, H], -1)[..., self.fs]
        uh = np.einsum("qa,era->eqr", B, U)
        err = np.einsum("eqr,q->e", (uh - u) ** 2, w) * m.vol
        return math.sqrt(err.sum())

    def energy(self, U):
        """(1/2) sum_T int eps |E_h|^2 + mu |H_h|^2 (U at a flat front)."""
        mat = self.material()
        tot = 0.0
        for e in range(self.mesh.ne):
            Me = self.mass(e)
            tot += sum(mat[e, r] * U[e, r] @ Me @ U[e, r] for r in range(self.nf))
        return 0.5 * tot


def spacetime_dofs(disc_or_counts, tents, patch_sizes, p, nrhs=1):
    """Sec. 5: sum_i N_dof,i * m * q with N_dof,i = n_f N_p |omega_V| and m = 2p, q = p+1."""
    nf, nb = disc_or_counts
    sizes = np.asarray(patch_sizes)[np.asarray(tents["vertex"])]
    return int(sizes.sum()) * nf * nb * (2 * p) * (p + 1) * nrhs


def front_before_layer(tents, nv, layer):
    """Vertex times of the front before ``layer``: each vertex's last t_top in earlier layers."""
    tau = np.zeros(nv)
    lp = tents["layer_ptr"]
    end = int(lp[layer])
    v = np.asarray(tents["vertex"][:end])
    np.maximum.at(tau, v, np.asarray(tents["t_top"][:end]))   # a vertex's times only increase
    return tau
