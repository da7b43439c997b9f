"""Discrete adjoint of the MTP-SAT evolution, FP64 (test infrastructure only).

The paper has no adjoint; this is the transpose of the oracle's own discrete map, written
out step by step so that it can be checked against central finite differences:

* Each tent applies the linear SAT map of Sec. 4 to the patch state.  Per sub-interval i
  (M_i = M(i/m), A and M' from Sec. 3):
      U_0 = M_i^-1 Y_0,  Y_n = A U_{n-1} (n = 1..q),  U_n = M_i^-1 (Y_n - n M' U_{n-1}) (n < q),
      Y_out = Y_0 + sum_n c_n Y_n,  c_n = (1/m)^n / n!.
  Reverse, with lam = dJ/dY_out and mu_n = dJ/dU_n:
      for n = q..1:  nu_n = M_i^-T mu_n (n < q),  lamY_n = c_n lam + nu_n,
                     mu_{n-1} += A^T lamY_n - n M'^T nu_n
      nu_0 = M_i^-T mu_0,  dJ/dY_0 = lam + nu_0.
* Material derivatives of the tent map: M_i depends on eps_T (E block) and mu_T (H block)
  through g(u) = (eps E, mu H):  dJ/dp += -nu_n^T (dM/dp) U_n for every solve; A depends on
  eps and mu only through the facet impedances Z = sqrt(mu/eps) of the upwind / PEC flux:
  dJ/dZ_T += lamY_n^T (dA/dZ_T) U_{n-1}, with dZ/deps = -Z/(2 eps), dZ/dmu = Z/(2 mu).
  The flux-matrix derivatives dC/dZ are taken by complex step (exact, no cancellation).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import maxwell as mx


def _flux_dz(n, Zm, Zp, h=1e-30):
    """d(Cm, Cp)/dZm and d(Cm, Cp)/dZp by complex step."""
    def mats(zm, zp):
        Cm = np.zeros((6, 6), complex)
        Cp = np.zeros((6, 6), complex)
        z = np.zeros(6, complex)
        for s in range(6):
            e = np.zeros(6, complex)
            e[s] = 1.0
            Cm[:, s] = mx.upwind_flux(e, z, n, zm, zp)
            Cp[:, s] = mx.upwind_flux(z, e, n, zm, zp)
        return Cm, Cp
    a = mats(Zm + 1j * h, Zp)
    b = mats(Zm, Zp + 1j * h)
    return (a[0].imag / h, a[1].imag / h), (b[0].imag / h, b[1].imag / h)


def _pec_dz(n, Z, h=1e-30):
    C = np.zeros((6, 6), complex)
    for s in range(6):
        e = np.zeros(6, complex)
        e[s] = 1.0
        up = np.concatenate([-e[:3], e[3:]])
        C[:, s] = mx.upwind_flux(e, up, n, Z + 1j * h, Z + 1j * h)
    return C.imag / h


def tent_dA_dZ(disc, V, dt):
    """{slot k: {(row slot, col slot): dA/dZ_{e_k} block}} for the tent at V."""
    m, fs = disc.mesh, disc.fs
    slots = list(m.patch[V])
    slot_of = {e: k for k, e in enumerate(slots)}
    out = {k: {} for k in range(len(slots))}

    def add(k, key, blk):
        out[k][key] = out[k].get(key, 0) + blk

    for k, e in enumerate(slots):
        j = m.local_index(e, V)
        for f in range(m.dim + 1):
            if f == j:
                continue
            n = disc.emb(m.normal[e, f])
            Fo = m.face_area[e, f] * disc.fown_ref[j, f]
            e2 = int(m.nbr[e, f])
            if e2 >= 0:
                k2 = slot_of[e2]
                (dCm_m, dCp_m), (dCm_p, dCp_p) = _flux_dz(n, disc.z(e), disc.z(e2))
                Fc = disc.face_cross(e, f, V)
                sel = np.ix_(fs, fs)
                add(k, (k, k), -dt * np.kron(dCm_m[sel], Fo))
                add(k, (k, k2), -dt * np.kron(dCp_m[sel], Fc))
                add(k2, (k, k), -dt * np.kron(dCm_p[sel], Fo))
                add(k2, (k, k2), -dt * np.kron(dCp_p[sel], Fc))
            else:
                dC = _pec_dz(n, disc.z(e))
                add(k, (k, k), -dt * np.kron(dC[np.ix_(fs, fs)], Fo))
    return out


def tent_adjoint(disc, V, dt, tau, Ybot, lam_top, q=None, msub=None):
    """Returns (lam_bot, dJ/deps, dJ/dmu) for the patch elements of the tent at V, given the
    bottom state Ybot [ns, nf*nb] and lam_top = dJ/dY_top."""
    p = disc.p
    q = p + 1 if q is None else q
    msub = 2 * p if msub is None else msub
    slots, M0, Mp, A = disc.tent_operators(V, dt, tau)
    dA = tent_dA_dZ(disc, V, dt)
    ns = len(slots)
    m = disc.mesh
    isE = np.isin(disc.fs, [0, 1, 2])
    dM_eps = [np.kron(np.diag(isE.astype(float)), disc.mass(e)) for e in slots]
    dM_mu = [np.kron(np.diag((~isE).astype(float)), disc.mass(e)) for e in slots]

    def apply(blocks, U, transpose=False):
        out = np.zeros_like(U)
        for (a, b), blk in blocks.items():
            if transpose:
                out[b] += blk.T @ U[a]
            else:
                out[a] += blk @ U[b]
        return out

    # forward tape
    tape = []
    Y = Ybot.copy()
    for i in range(msub):
        ti = i / msub
        Mi = [M0[k] + ti * Mp[k] for k in range(ns)]
        lus = [sla.lu_factor(Mi[k]) for k in range(ns)]
        solve = lambda R, lus=lus: np.stack([sla.lu_solve(lus[k], R[k]) for k in range(ns)])
        Us = [solve(Y)]
        acc = Y.copy()
        for n in range(1, q + 1):
            Yn = apply(A, Us[-1])
            acc += (1.0 / msub) ** n / math.factorial(n) * Yn
            if n <= q - 1:
                Us.append(solve(Yn - n * np.stack([Mp[k] @ Us[-1][k] for k in range(ns)])))
        tape.append((lus, Us))
        Y = acc
    # reverse
    lam = lam_top.copy()
    gZ = np.zeros(ns)
    geps = np.zeros(ns)
    gmu = np.zeros(ns)
    for i in reversed(range(msub)):
        lus, Us = tape[i]
        solveT = lambda R, lus=lus: np.stack([sla.lu_solve(lus[k], R[k], trans=1) for k in range(ns)])
        mu_next = np.zeros_like(lam)            # mu_n for the current n
        lam_in = lam.copy()
        for n in range(q, 0, -1):
            cn = (1.0 / msub) ** n / math.factorial(n)
            lamY = cn * lam
            if n < q:
                nu = solveT(mu_next)
                lamY = lamY + nu
                for k in range(ns):
                    geps[k] -= nu[k] @ dM_eps[k] @ Us[n][k]
                    gmu[k] -= nu[k] @ dM_mu[k] @ Us[n][k]
            Uprev = Us[n - 1]
            for k in range(ns):
                gZ[k] += np.sum(lamY * apply(dA[k], Uprev))
            mu_prev = apply(A, lamY, transpose=True)
            if n < q:
                mu_prev -= n * np.stack([Mp[k].T @ nu[k] for k in range(ns)])
            mu_next = mu_prev
        nu0 = solveT(mu_next)
        for k in range(ns):
            geps[k] -= nu0[k] @ dM_eps[k] @ Us[0][k]
            gmu[k] -= nu0[k] @ dM_mu[k] @ Us[0][k]
        lam = lam_in + nu0
    for k, e in enumerate(slots):
        z = disc.z(e)
        geps[k] += gZ[k] * (-z / (2 * m.eps[e]))
        gmu[k] += gZ[k] * (z / (2 * m.mu[e]))
    return slots, lam, geps, gmu


def evolve_adjoint(disc, tents, Y0, lam_T):
    """Reverse sweep over all tents.  Returns (dJ/dY0, dJ/deps, dJ/dmu) of the tent maps only
    (the caller adds the explicit dependence of its initial state and functional)."""
    m = disc.mesh
    Y = Y0.copy().reshape(m.ne, -1)
    tau = np.zeros(m.nv)
    store = []
    for t in range(len(tents["vertex"])):
        V = int(tents["vertex"][t])
        tb, tt = float(tents["t_bot"][t]), float(tents["t_top"][t])
        patch = m.patch[V]
        tau_patch = {int(v): tau[int(v)] for e in patch for v in m.elems[e]}
        store.append((V, tt - tb, tau_patch, Y[patch].copy()))
        _, Yp = disc.sat_tent(V, tt - tb, tau, Y[patch])
        Y[patch] = Yp
        tau[V] = tt
    lam = lam_T.copy().reshape(m.ne, -1)
    geps = np.zeros(m.ne)
    gmu = np.zeros(m.ne)
    for V, dt, tau_patch, Ybot in reversed(store):
        tau_l = np.zeros(m.nv)
        for v, x in tau_patch.items():
            tau_l[v] = x
        slots, lb, ge, gm = tent_adjoint(disc, V, dt, tau_l, Ybot, lam[m.patch[V]])
        lam[slots] = lb
        geps[slots] += ge
        gmu[slots] += gm
    return lam.reshape(Y0.shape), geps, gmu


def l2_misfit(disc, Y_T, U_target):
    """J = 1/2 sum_T int_T |E_h(T) - E_target,h|^2 (flat front: E_h = M^-1 Y_E / eps) and its
    partial derivatives dJ/dY_T (E block) and dJ/deps (explicit, through E = Y_E/eps)."""
    m = disc.mesh
    isE = np.isin(disc.fs, [0, 1, 2])
    J = 0.0
    lam = np.zeros_like(Y_T)
    geps = np.zeros(m.ne)
    for e in range(m.ne):
        Me = disc.mass(e)
        for r in np.nonzero(isE)[0]:
            U = np.linalg.solve(Me, Y_T[e, r]) / m.eps[e]
            d = U - U_target[e, r]
            Md = Me @ d
            J += 0.5 * d @ Md
            lam[e, r] = np.linalg.solve(Me.T, Md) / m.eps[e]       # = d / eps
            geps[e] += -(Md @ U) / m.eps[e]
    return J, lam, geps
