"""Helpers that run the oracle on the same seeded inputs the GPU tests use.
Only numbers computed by ``oracle/`` come out of here (test infrastructure)."""
import numpy as np

import mtp_synth as S
from oracle.mesh import Mesh as OMesh
from oracle.mtp import Discretization, front_before_layer
from oracle.pitch import pitch_tents


def oracle_setup(w):
    mesh = OMesh(w.verts, w.elems, w.eps, w.mu)
    return Discretization(mesh, w.p)


def oracle_full_run(w, wavespeed=None):
    """Initial L2 projection, full evolve; returns (initial y lattice values, final y lattice values,
    final energy, initial energy)."""
    disc = oracle_setup(w)
    tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, w.causality, wavespeed)
    Y0 = disc.project_initial(w.init)
    Y, _ = disc.evolve(Y0, tents)
    vals0 = disc.eval_lattice(disc.y_coeffs(Y0))
    vals = disc.eval_lattice(disc.y_coeffs(Y))
    e0 = disc.energy(disc.fields_at_flat_front(Y0))
    e1 = disc.energy(disc.fields_at_flat_front(Y))
    return vals0, vals, e0, e1


def oracle_single_tents(w, disc, tents, layer, vals, sample, elems_needed=None):
    """Run the sampled tents of ``layer`` on the state given by lattice values ``vals``
    [ne, Np, nf] (front before ``layer``); returns {tent index: lattice values of its patch}."""
    m = disc.mesh
    tau = front_before_layer(tents, m.nv, layer)
    out = {}
    for t in sample:
        V = int(tents["vertex"][t])
        dt = float(tents["t_top"][t] - tents["t_bot"][t])
        patch = m.patch[V]
        Yp = _moments_subset(disc, vals, patch)
        _, Y = disc.sat_tent(V, dt, tau, Yp.reshape(len(patch), -1))
        Y = Y.reshape(len(patch), disc.nf, disc.nb)
        coef = np.stack([np.linalg.solve(disc.mass(e), Y[k].T).T for k, e in enumerate(patch)])
        out[t] = _eval_subset(disc, coef, patch)
    return out


def _moments_subset(disc, vals, elems):
    from oracle.simplex import bernstein_eval
    mi = S.lattice_multi_indices(disc.d, disc.p)
    Y = np.zeros((len(elems), disc.nf, disc.nb))
    for k, e in enumerate(elems):
        lam = disc.mesh.barycentric_of_sorted_lattice(e, mi, disc.p)
        B = bernstein_eval(lam, disc.p)
        coef = np.linalg.solve(B, vals[e])
        Y[k] = (disc.mass(e) @ coef).T
    return Y


def _eval_subset(disc, coef, elems):
    from oracle.simplex import bernstein_eval
    mi = S.lattice_multi_indices(disc.d, disc.p)
    out = np.zeros((len(elems), len(mi), disc.nf))
    for k, e in enumerate(elems):
        lam = disc.mesh.barycentric_of_sorted_lattice(e, mi, disc.p)
        out[k] = bernstein_eval(lam, disc.p) @ coef[k].T
    return out


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
