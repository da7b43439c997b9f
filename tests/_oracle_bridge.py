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


def max_rel(a, b):
    """Largest pointwise difference over the largest reference magnitude: unlike one L2 norm
    over a whole mesh, a local error confined to one element (one facet, one patch) shows up
    at full size."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.abs(a - b).max() / np.abs(b).max())


# ---------------------------------------------------------------------------------------
# several layers of a full-size workload, the tents of each layer spread over host processes
# ---------------------------------------------------------------------------------------
_POOL_DISC = {}


def _pool_init(workload_name, verts, elems, eps, mu, p):
    from oracle.mesh import Mesh as OMesh
    _POOL_DISC["disc"] = Discretization(OMesh(verts, elems, eps, mu), p)


def _pool_tent(job):
    V, dt, tau, Yp = job
    return _POOL_DISC["disc"].sat_tent(V, dt, tau, Yp)


def oracle_layers(w, tents, layer_begin, layer_end, vals, procs=None):
    """Apply the tents of layers [layer_begin, layer_end) with the oracle to the state given by
    lattice values ``vals`` [ne, Np, nf] on the front before ``layer_begin``; returns the lattice
    values after them.  Tents of one layer are independent (Sec. 2), so each layer is spread
    over a pool of spawned processes (spawn: safe after the parent has used the GPU)."""
    import multiprocessing as mp
    import os
    disc = oracle_setup(w)
    m = disc.mesh
    tau = front_before_layer(tents, m.nv, layer_begin)
    Y = disc.moments_from_lattice(vals).reshape(m.ne, -1)
    procs = procs or max(1, min(16, (os.cpu_count() or 2) - 1))
    lp = tents["layer_ptr"]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_pool_init, initargs=(w.name, w.verts, w.elems, w.eps, w.mu, w.p)) as pool:
        for L in range(layer_begin, layer_end):
            idx = range(int(lp[L]), int(lp[L + 1]))
            jobs = []
            for t in idx:
                V = int(tents["vertex"][t])
                assert tau[V] == tents["t_bot"][t]
                jobs.append((V, float(tents["t_top"][t] - tents["t_bot"][t]), tau, Y[m.patch[V]]))
            for t, (slots, Yp) in zip(idx, pool.map(_pool_tent, jobs, chunksize=1)):
                Y[slots] = Yp
                tau[int(tents["vertex"][t])] = float(tents["t_top"][t])
    Y = Y.reshape(m.ne, disc.nf, disc.nb)
    return disc.eval_lattice(disc.y_coeffs(Y))
