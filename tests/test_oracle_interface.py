"""Pins of the oracle at a material interface (eps, mu jump), CPU only.

The impedance-weighted upwind flux (Sec. 3, upwind flux, read for piecewise-constant eps and
mu) is consistent: for fields whose tangential components are continuous it equals f(u) n
whatever impedances it is given.  So the smooth-field pins cannot see which side's impedance
the assembly passes where.  These pins use fields with a jump at the interface:

* the assembled tent operator A at a vertex on a plane interface, applied to piecewise-
  constant data (an incident plane wave on one side, nothing on the other), must produce
  the exact Riemann (Fresnel) flux on the interface facets: for piecewise constants the
  upwind flux is the flux of the exact interface state, whose tangential E is the
  transmitted wave 2 Z2 / (Z1 + Z2) E_inc;
* the whole scheme, run on a strip with an eps jump, must reflect a smooth pulse with the
  normal-incidence coefficient (Z2 - Z1) / (Z2 + Z1) and converge to the exact
  reflected + transmitted solution.

Planted mistakes (the neighbour's and the own impedance swapped in the assembly; the
impedance inverted) fail them.
"""
import math

import numpy as np
import pytest

import mtp_synth as S
from oracle import maxwell as mx
from oracle.mesh import Mesh
from oracle.mtp import Discretization
from oracle.pitch import pitch_tents
from oracle.simplex import bernstein_eval, duffy_rule


# ----------------------------------------------------------------------------- assembled flux
def _facet_geometry(verts, el, f):
    """Outward unit normal and measure of facet f (opposite local vertex f) of a tetrahedron,
    from the vertex coordinates alone."""
    P = verts[el]
    F = [P[i] for i in range(4) if i != f]
    n = np.cross(F[1] - F[0], F[2] - F[0])
    area = 0.5 * np.linalg.norm(n)
    n = n / np.linalg.norm(n)
    if n @ (P[f] - F[0]) > 0:                  # point away from the opposite vertex
        n = -n
    return n, area


def _interface_flux_mismatch(eps_l, mu_l, eps_r, mu_r):
    """Largest mismatch, relative to the largest expected value, between the constant moments
    of A U (the tent at the centre vertex of a 2 x 2 x 2 Kuhn cube, interface plane x = 1/2)
    and the exact Riemann flux."""
    v, e = S.cube_mesh(2)
    left = v[e].mean(1)[:, 0] < 0.5
    eps = np.where(left, eps_l, eps_r)
    mu = np.where(left, mu_l, mu_r)
    disc = Discretization(Mesh(v, e, eps, mu), 1)
    V = 13                                     # (1/2, 1/2, 1/2)
    dt = 0.05
    slots, M0, Mp, A = disc.tent_operators(V, dt, np.zeros(len(v)))
    Z1, Z2 = math.sqrt(mu_l / eps_l), math.sqrt(mu_r / eps_r)
    nx = np.array([1.0, 0.0, 0.0])
    Einc = np.array([0.0, 0.7, -0.4])          # tangential to the interface
    uL = np.concatenate([Einc, np.cross(nx, Einc) / Z1])      # wave travelling along +x
    Est = 2.0 * Z2 / (Z1 + Z2) * Einc                           # exact interface state
    ustar = np.concatenate([Est, np.cross(nx, Est) / Z2])
    nb = disc.nb
    U = [np.kron(uL if left[el] else np.zeros(6), np.ones(nb)) for el in slots]
    AU = [np.zeros(6 * nb) for _ in slots]
    for (a, b), blk in A.items():
        AU[a] += blk @ U[b]
    worst, scale = 0.0, 0.0
    for k, el in enumerate(slots):
        got = AU[k].reshape(6, nb).sum(1)      # moments against sum_a B_a = 1
        expect = np.zeros(6)
        j = int(np.nonzero(e[el] == V)[0][0])
        for f in range(4):
            if f == j:
                continue                       # the facet opposite V has delta = 0
            n, area = _facet_geometry(v, e[el], f)
            centre = v[[x for i, x in enumerate(e[el]) if i != f]].mean(0)
            on_interface = abs(centre[0] - 0.5) < 1e-12 and abs(abs(n[0]) - 1) < 1e-12
            uF = ustar if on_interface else (uL if left[el] else np.zeros(6))
            # int_F delta = dt |F| / 3 (lambda_V averages 1/3 on a triangle containing V)
            expect -= dt * area / 3.0 * (mx.f_of(uF) @ n)
        worst = max(worst, np.abs(got - expect).max())
        scale = max(scale, np.abs(expect).max())
    return worst / scale


@pytest.mark.parametrize("mats", [(1.0, 1.0, 4.0, 1.0), (1.0, 1.0, 2.0, 3.0), (3.0, 0.5, 1.0, 2.0)])
def test_assembled_operator_gives_exact_riemann_flux_at_interface(mats):
    assert _interface_flux_mismatch(*mats) < 1e-13


def test_interface_flux_pin_detects_swapped_impedances(monkeypatch):
    orig = mx.flux_matrices
    monkeypatch.setattr(mx, "flux_matrices", lambda n, Zm, Zp: orig(n, Zp, Zm))
    assert _interface_flux_mismatch(1.0, 1.0, 4.0, 1.0) > 1e-3


def test_interface_flux_pin_detects_inverted_impedance(monkeypatch):
    monkeypatch.setattr(Discretization, "z", lambda self, e: math.sqrt(self.mesh.eps[e] / self.mesh.mu[e]))
    assert _interface_flux_mismatch(1.0, 1.0, 4.0, 1.0) > 1e-3


# ----------------------------------------------------------------------------- reflection
def _strip(k):
    """[0, 2] x [0, 1/4], 8k x k squares each split along its (i, j)-(i+1, j+1) diagonal."""
    nx, ny = 8 * k, k
    xs, ys = np.linspace(0, 2, nx + 1), np.linspace(0, 0.25, ny + 1)
    vid = lambda i, j: i + (nx + 1) * j
    V = np.array([[xs[i], ys[j]] for j in range(ny + 1) for i in range(nx + 1)])
    E = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            E += [[a, b, c], [a, c, d]]
    return V, np.array(E)


EPS2, X0, WIDTH, T_END = 4.0, 0.5, 0.15, 1.0
Z1, Z2 = 1.0, math.sqrt(1.0 / EPS2)
R_EXACT, TAU_EXACT = (Z2 - Z1) / (Z2 + Z1), 2 * Z2 / (Z1 + Z2)


def _pulse(s):
    return np.exp(-(s / WIDTH) ** 2)


def _interface_solution(X, t):
    """TE fields (Ey, Hz) of a pulse travelling along +x from eps = 1 (x < 1) into eps = 4:
    incident + reflected (coefficient R) on the left, transmitted (coefficient TAU, speed 1/2)
    on the right; y-independent, so the PEC walls y = 0, 1/4 hold it exactly."""
    x = X[..., 0]
    left = x < 1.0
    inc = _pulse(x - X0 - t)
    ref = R_EXACT * _pulse(2.0 - x - X0 - t)
    c2 = 1.0 / math.sqrt(EPS2)
    tra = TAU_EXACT * _pulse(1.0 - X0 - (t - (x - 1.0) / c2))
    Ey = np.where(left, inc + ref, tra)
    Hz = np.where(left, (inc - ref) / Z1, tra / Z2)
    z = np.zeros_like(x)
    return np.stack([z, Ey, z], -1), np.stack([z, z, Hz], -1)


def _reflection_run(k, p=2):
    V, E = _strip(k)
    cen = V[E].mean(1)
    eps = np.where(cen[:, 0] > 1.0, EPS2, 1.0)
    mu = np.ones(len(E))
    mesh = Mesh(V, E, eps, mu)
    disc = Discretization(mesh, p)
    tents = pitch_tents(V, E, eps, mu, T_END, 0.5)
    Y, _ = disc.evolve(disc.project_initial(_interface_solution), tents)
    U = disc.fields_at_flat_front(Y)
    rel = disc.l2_error(U, _interface_solution, T_END) / disc.l2_error(0 * U, _interface_solution, T_END)
    lam, w = duffy_rule(2, p + 8)
    B = bernstein_eval(lam, p)
    X = np.einsum("qi,eid->eqd", lam, V[E])
    Ey = np.einsum("qa,ea->eq", B, U[:, 1, :])
    shape = _pulse(2.0 - X[..., 0] - X0 - T_END)       # unit reflected pulse at t = T
    left = (cen[:, 0] < 1.0)[:, None]
    num = np.einsum("eq,q,e->", Ey * shape * left, w, mesh.vol)
    den = np.einsum("eq,q,e->", shape * shape * left, w, mesh.vol)
    return rel, num / den


def test_reflection_coefficient_at_eps_jump_converges():
    """Normal incidence on eps 1 | 4 (Z 1 | 1/2): reflected amplitude -> -1/3, and the L2
    error against the exact reflected + transmitted solution falls like O(h^3) at p = 2."""
    (e1, r1), (e2, r2) = _reflection_run(1), _reflection_run(2)
    assert abs(r2 - R_EXACT) < 1.5e-3, (r1, r2)
    assert abs(r2 - R_EXACT) < abs(r1 - R_EXACT) / 4
    assert e2 < e1 / 2.5 and e2 < 0.12, (e1, e2)


def test_reflection_pin_detects_inverted_impedance(monkeypatch):
    monkeypatch.setattr(Discretization, "z", lambda self, e: math.sqrt(self.mesh.eps[e] / self.mesh.mu[e]))
    _, r = _reflection_run(1)
    assert abs(r - R_EXACT) > 0.3, r
