"""Pins of the oracle's discrete adjoint (CPU): the transpose identity of one tent map and
central finite differences of the oracle's own forward map (tents frozen by pitching with
wave speed 1, an upper bound of 1/sqrt(eps mu) for eps >= 1, mu = 1)."""
import numpy as np
import pytest

import mtp_synth as S
from oracle.adjoint import evolve_adjoint, l2_misfit, tent_adjoint
from oracle.mesh import Mesh
from oracle.mtp import Discretization
from oracle.pitch import pitch_tents


def _disc(w, eps=None, mu=None):
    return Discretization(Mesh(w.verts, w.elems, w.eps if eps is None else eps,
                               w.mu if mu is None else mu), w.p)


def _tent_case(p=2):
    w = S.adjoint_cube(n=2, p=p, T=0.1)
    V = 13                                                  # centre vertex, 24 tets
    tau = np.zeros(len(w.verts))
    tau[[4, 10, 12, 14]] = 0.01
    return w, V, tau, 0.03


@pytest.mark.parametrize("p", [1, 2])
def test_tent_adjoint_transpose_identity(p):
    w, V, tau, dt = _tent_case(p)
    disc = _disc(w)
    ns = len(disc.mesh.patch[V])
    rng = np.random.default_rng(p)
    x = rng.standard_normal((ns, disc.nf * disc.nb))
    y = rng.standard_normal((ns, disc.nf * disc.nb))
    _, Phix = disc.sat_tent(V, dt, tau, x)
    _, PhiTy, _, _ = tent_adjoint(disc, V, dt, tau, x, y)
    assert abs(np.sum(Phix * y) - np.sum(x * PhiTy)) < 1e-12 * np.abs(np.sum(Phix * y))


def test_tent_material_derivatives_match_fd():
    w, V, tau, dt = _tent_case(2)
    disc = _disc(w)
    patch = disc.mesh.patch[V]
    rng = np.random.default_rng(7)
    x = rng.standard_normal((len(patch), disc.nf * disc.nb))
    y = rng.standard_normal((len(patch), disc.nf * disc.nb))
    _, _, geps, gmu = tent_adjoint(disc, V, dt, tau, x, y)
    for k in (0, 5, 17):
        e = patch[k]
        for which, g in (("eps", geps), ("mu", gmu)):
            h = 1e-6
            vals = []
            for s in (1, -1):
                eps, mu = w.eps.copy(), w.mu.copy()
                (eps if which == "eps" else mu)[e] += s * h
                _, Yp = _disc(w, eps, mu).sat_tent(V, dt, tau, x)
                vals.append(np.sum(Yp * y))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (which, k, fd, g[k])


def _J_and_grad(w, eps, target_U, tents):
    disc = _disc(w, eps)
    Y0 = disc.project_initial(w.init)
    Y, _ = disc.evolve(Y0, tents)
    J, lamT, geps_final = l2_misfit(disc, Y, target_U)
    return disc, Y0, J, lamT, geps_final


def test_full_gradient_matches_central_fd():
    w = S.adjoint_cube(n=2, p=1, T=0.08, width=0.3)
    ws = np.ones(len(w.elems))
    tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, 0.5, ws)
    tgt_disc = _disc(w, w.extra["eps_target"])
    Yt, _ = tgt_disc.evolve(tgt_disc.project_initial(w.init), tents)
    Ut = tgt_disc.fields_at_flat_front(Yt)
    disc, Y0, J, lamT, geps_final = _J_and_grad(w, w.eps, Ut, tents)
    lam0, geps_tent, gmu_tent = evolve_adjoint(disc, tents, Y0, lamT)
    isE = np.isin(disc.fs, [0, 1, 2])
    geps_init = np.einsum("era,era->e", lam0[:, isE], Y0[:, isE]) / w.eps
    grad = geps_final + geps_tent + geps_init
    h = 1e-6
    for e in (0, 11, 30, 47):
        Js = []
        for s in (1, -1):
            eps = w.eps.copy()
            eps[e] += s * h
            Js.append(_J_and_grad(w, eps, Ut, tents)[2])
        fd = (Js[0] - Js[1]) / (2 * h)
        assert abs(fd - grad[e]) <= 1e-6 * np.abs(grad).max(), (e, fd, grad[e])
