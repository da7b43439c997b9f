"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only *describes problems*: structured simplicial meshes of the unit
square / cube (optionally perturbed or graded), per-element material values,
and closed-form field functions used as initial data or as exact solutions.
It contains none of the MTP / SAT arithmetic, so both the CPU oracle and the
GPU path may import it without sharing any part of the method.

Conventions
-----------
* 2D meshes: vertex (i, j) has index ``i + (n+1) j``; square (i, j) is split
  along its diagonal (i, j)-(i+1, j+1) into two triangles.
* 3D meshes: vertex (i, j, k) has index ``i + (n+1) (j + (n+1) k)``; every cube
  is split into the 6 Kuhn (Freudenthal) tetrahedra along the (0,0,0)-(1,1,1)
  diagonal, which gives a conforming mesh with 24 tetrahedra around every
  interior vertex.
* Field functions take points ``x`` of shape ``[..., dim]`` and a time ``t`` and
  return ``(E, H)`` with 3-component E and H (2D: z-invariant, so TE fields are
  ``E = (Ex, Ey, 0)``, ``H = (0, 0, Hz)``).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def square_mesh(n: int, coords=None):
    """Unit square, n x n squares each split into 2 right triangles."""
    xs = np.linspace(0.0, 1.0, n + 1) if coords is None else np.asarray(coords, float)
    vid = lambda i, j: i + (n + 1) * j
    verts = np.array([[xs[i], xs[j]] for j in range(n + 1) for i in range(n + 1)], float)
    elems = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            elems.append([a, b, c])
            elems.append([a, c, d])
    return verts, np.array(elems, np.int32)


def cube_mesh(n: int, coords=None):
    """Unit cube, n^3 cubes each split into 6 Kuhn tetrahedra."""
    xs = np.linspace(0.0, 1.0, n + 1) if coords is None else np.asarray(coords, float)
    vid = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    verts = np.array([[xs[i], xs[j], xs[k]]
                      for k in range(n + 1) for j in range(n + 1) for i in range(n + 1)], float)
    unit = [np.array(e) for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    elems = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                base = np.array([i, j, k])
                for perm in itertools.permutations(range(3)):
                    path = [base.copy()]
                    cur = base.copy()
                    for ax in perm:
                        cur = cur + unit[ax]
                        path.append(cur.copy())
                    elems.append([vid(*q) for q in path])
    return verts, np.array(elems, np.int32)


def interior_mask(verts: np.ndarray) -> np.ndarray:
    """Vertices strictly inside the unit box (tolerance 1e-12)."""
    return np.all((verts > 1e-12) & (verts < 1.0 - 1e-12), axis=1)


def perturb_interior(verts: np.ndarray, h: float, amount: float, seed: int) -> np.ndarray:
    """Add U(-amount*h, amount*h) to every coordinate of every interior vertex."""
    rng = np.random.default_rng(seed)
    out = verts.copy()
    shift = rng.uniform(-amount * h, amount * h, size=verts.shape)
    mask = interior_mask(verts)
    out[mask] += shift[mask]
    return out


def graded_coords(n: int, ratio: float) -> np.ndarray:
    """Per-axis coordinates with geometric cell sizes h_i = h0 r^i, r = ratio^(1/(n-1)),
    smallest cell at 0, sizes summing to 1."""
    r = ratio ** (1.0 / (n - 1))
    sizes = r ** np.arange(n)
    sizes = sizes / sizes.sum()
    x = np.concatenate([[0.0], np.cumsum(sizes)])
    x[-1] = 1.0
    return x


def centroids(verts, elems):
    return verts[elems].mean(axis=1)


# --------------------------------------------------------------------------
# closed-form fields
# --------------------------------------------------------------------------
def te_cavity_mode(x, t):
    """2D TE mode of the unit-square PEC cavity (omega = sqrt(2) pi):
    Hz = cos(pi x) cos(pi y) cos(w t), Ex = -cos(pi x) sin(pi y) sin(w t)/sqrt2,
    Ey = sin(pi x) cos(pi y) sin(w t)/sqrt2."""
    x = np.asarray(x, float)
    w = math.sqrt(2.0) * math.pi
    cx, sx = np.cos(math.pi * x[..., 0]), np.sin(math.pi * x[..., 0])
    cy, sy = np.cos(math.pi * x[..., 1]), np.sin(math.pi * x[..., 1])
    z = np.zeros_like(cx)
    E = np.stack([-cx * sy * math.sin(w * t) / math.sqrt(2.0),
                  sx * cy * math.sin(w * t) / math.sqrt(2.0), z], -1)
    H = np.stack([z, z, cx * cy * math.cos(w * t)], -1)
    return E, H


def cube_cavity_mode(x, t, A=(1.0, 1.0, -2.0)):
    """3D (1,1,1) mode of the unit-cube PEC cavity, omega = sqrt(3) pi, div E = 0."""
    x = np.asarray(x, float)
    w = math.sqrt(3.0) * math.pi
    a1, a2, a3 = A
    c = [np.cos(math.pi * x[..., d]) for d in range(3)]
    s = [np.sin(math.pi * x[..., d]) for d in range(3)]
    ct, st = math.cos(w * t), math.sin(w * t)
    E = np.stack([a1 * c[0] * s[1] * s[2], a2 * s[0] * c[1] * s[2], a3 * s[0] * s[1] * c[2]], -1) * ct
    H = -np.stack([(a3 - a2) * s[0] * c[1] * c[2], (a1 - a3) * c[0] * s[1] * c[2],
                   (a2 - a1) * c[0] * c[1] * s[2]], -1) * (st / math.sqrt(3.0))
    return E, H


def gaussian_pulse(centres, width=0.05):
    """E = curl(psi e_z) = (d_y psi, -d_x psi, 0), psi = sum_c exp(-|x - c|^2 / w^2); H = 0."""
    centres = np.atleast_2d(np.asarray(centres, float))

    def fn(x, t=0.0):
        x = np.asarray(x, float)
        E = np.zeros(x.shape[:-1] + (3,))
        for c in centres:
            d = x - c[: x.shape[-1]]
            psi = np.exp(-np.sum(d * d, -1) / width ** 2)
            E[..., 0] += -2.0 * d[..., 1] / width ** 2 * psi
            E[..., 1] += 2.0 * d[..., 0] / width ** 2 * psi
        return E, np.zeros_like(E)
    return fn


def plane_wave_x(g):
    """E_z = g(x - t), H_y = -g(x - t): exact solution for eps = mu = 1 (g any callable)."""
    def fn(x, t):
        x = np.asarray(x, float)
        v = g(x[..., 0] - t)
        z = np.zeros_like(v)
        return np.stack([z, z, v], -1), np.stack([z, -v, z], -1)
    return fn


# --------------------------------------------------------------------------
# workloads (the five problem configurations)
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    dim: int
    verts: np.ndarray
    elems: np.ndarray
    eps: np.ndarray
    mu: np.ndarray
    p: int
    T: float
    causality: float = 0.5
    init: object = None          # callable (x, t) -> (E, H)
    exact: object = None         # callable or None
    extra: dict = field(default_factory=dict)

    @property
    def n_fields(self):
        return 3 if self.dim == 2 else 6

    @property
    def n_basis(self):
        p = self.p
        return (p + 1) * (p + 2) // 2 if self.dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6


def te_square(n=8, p=2, T=0.5):
    """2D TE unit-square PEC cavity, n x n x 2 triangles (n = 8: 128 triangles)."""
    v, e = square_mesh(n)
    one = np.ones(len(e))
    return Workload(f"te_square_n{n}_p{p}", 2, v, e, one, one.copy(), p, T,
                    init=te_cavity_mode, exact=te_cavity_mode)


def cube_mode(n=16, p=3, T=1.0, perturb=0.15, seed=11029):
    """3D unit-cube PEC cavity, n^3 x 6 tets, interior vertices perturbed by U(+-0.15 h)."""
    v, e = cube_mesh(n)
    if perturb:
        v = perturb_interior(v, 1.0 / n, perturb, seed)
    one = np.ones(len(e))
    return Workload(f"cube_mode_n{n}_p{p}", 3, v, e, one, one.copy(), p, T,
                    init=cube_cavity_mode, exact=cube_cavity_mode)


def graded_sphere(n=32, p=4, T=0.5, ratio=8.0, seed=1906, eps_in=4.0, radius=0.25, width=0.05):
    """3D unit cube graded toward (0,0,0) with size ratio 8, eps = 4 in a ball of radius 0.25
    around the centre (by element centroid), Gaussian E pulse at a seeded centre."""
    v, e = cube_mesh(n, graded_coords(n, ratio))
    c = centroids(v, e)
    eps = np.where(np.linalg.norm(c - 0.5, axis=1) <= radius, eps_in, 1.0)
    rng = np.random.default_rng(seed)
    centre = rng.uniform(0.3, 0.7, size=3)
    return Workload(f"graded_sphere_n{n}_p{p}", 3, v, e, eps, np.ones(len(e)), p, T,
                    init=gaussian_pulse(centre, width), extra={"centre": centre})


def adjoint_cube(n=8, p=2, T=0.5, seed_eps=1, seed_target=2, seed_pulse=11029, width=0.05):
    """3D unit cube, per-element eps ~ U[1, 3] (seeded) and a second seeded target eps."""
    v, e = cube_mesh(n)
    eps = np.random.default_rng(seed_eps).uniform(1.0, 3.0, len(e))
    eps_t = np.random.default_rng(seed_target).uniform(1.0, 3.0, len(e))
    centre = np.random.default_rng(seed_pulse).uniform(0.3, 0.7, size=3)
    return Workload(f"adjoint_cube_n{n}_p{p}", 3, v, e, eps, np.ones(len(e)), p, T,
                    init=gaussian_pulse(centre, width),
                    extra={"eps_target": eps_t, "centre": centre})


def many_instances(count=64, seed=4, n_rhs=4, width=0.05, T=0.5):
    """Sizes n ~ U{6..20}, orders p ~ U{2,3,4}, 4 pulse centres per instance (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(6, 21))
        p = int(rng.choice([2, 3, 4]))
        centres = rng.uniform(0.3, 0.7, size=(n_rhs, 3))
        out.append({"n": n, "p": p, "centres": centres, "T": T, "width": width})
    return out


def random_state(n_elems, n_fields, n_basis, seed, dtype=np.float64):
    """Seeded smooth-free random coefficients (standard normal) for single-layer checks."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_elems, n_fields, n_basis)).astype(dtype)


def lattice_multi_indices(dim: int, p: int):
    """Equispaced degree-p lattice of a simplex, as integer tuples (i_1..i_dim), sum <= p,
    enumerated with i_dim outermost and i_1 innermost.  The point is
    v_s0 + sum_l (i_l / p) (v_sl - v_s0), with s the element's vertex ids sorted ascending."""
    out = []
    if dim == 2:
        for i2 in range(p + 1):
            for i1 in range(p + 1 - i2):
                out.append((i1, i2))
    else:
        for i3 in range(p + 1):
            for i2 in range(p + 1 - i3):
                for i1 in range(p + 1 - i3 - i2):
                    out.append((i1, i2, i3))
    return np.array(out, np.int64)


def lattice_points(verts, elems, p):
    """Physical lattice points [n_elems, N_p, dim] (see lattice_multi_indices)."""
    dim = verts.shape[1]
    s = np.sort(elems, axis=1)
    P = verts[s]                      # [ne, dim+1, dim]
    mi = lattice_multi_indices(dim, p).astype(float) / p
    base = P[:, 0, :]
    out = base[:, None, :].repeat(len(mi), 1)
    for l in range(dim):
        out = out + mi[None, :, l, None] * (P[:, l + 1, :] - base)[:, None, :]
    return out
