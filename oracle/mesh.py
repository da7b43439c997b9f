"""Conforming simplicial mesh for the oracle (test infrastructure only).

Sec. 2 starts from a conforming spatial mesh of elements T and vertices V; each
tent's spatial footprint is the vertex patch omega_V (all elements containing V).
This module holds the affine geometry of each element (barycentric gradients,
measure), the facet table (each facet shared by two elements, or on the domain
boundary, which is PEC everywhere in this implementation), and vertex adjacency.
Element vertex order is kept exactly as given; orientation does not matter
because only |det| and outward normals are used.
"""
from __future__ import annotations

import math

import numpy as np


class Mesh:
    def __init__(self, verts, elems, eps, mu):
        self.verts = np.asarray(verts, float)
        self.elems = np.asarray(elems, np.int64)
        self.dim = self.verts.shape[1]
        self.ne = len(self.elems)
        self.nv = len(self.verts)
        self.eps = np.asarray(eps, float).copy()
        self.mu = np.asarray(mu, float).copy()
        d = self.dim
        P = self.verts[self.elems]                              # [ne, d+1, d]
        J = np.stack([P[:, l + 1] - P[:, 0] for l in range(d)], -1)   # columns = edges
        self.detJ = np.linalg.det(J)
        if np.any(np.abs(self.detJ) < 1e-300):
            raise ValueError("degenerate element")
        Jinv = np.linalg.inv(J)                                 # rows = grad lambda_1..d
        g = np.zeros((self.ne, d + 1, d))
        g[:, 1:, :] = Jinv
        g[:, 0, :] = -Jinv.sum(1)
        self.grad_lam = g                                       # [ne, d+1, d]
        self.vol = np.abs(self.detJ) / math.factorial(d)
        self._faces()
        self._adjacency()

    # ------------------------------------------------------------------
    def _faces(self):
        d = self.dim
        key_to = {}
        self.nbr = -np.ones((self.ne, d + 1), np.int64)        # neighbour element across local facet f
        self.nbr_face = -np.ones((self.ne, d + 1), np.int64)
        for e in range(self.ne):
            for f in range(d + 1):
                key = tuple(sorted(int(v) for i, v in enumerate(self.elems[e]) if i != f))
                if key in key_to:
                    e2, f2 = key_to.pop(key)
                    self.nbr[e, f], self.nbr_face[e, f] = e2, f2
                    self.nbr[e2, f2], self.nbr_face[e2, f2] = e, f
                else:
                    key_to[key] = (e, f)
        # outward unit normal and measure of facet f (opposite local vertex f):
        # grad lambda_f points into the element, normal to facet f.
        gl = self.grad_lam
        nrm = np.linalg.norm(gl, axis=-1)                       # [ne, d+1] = 1/height_f
        self.normal = -gl / nrm[..., None]
        # |F_f| = d |T| / height_f
        self.face_area = d * self.vol[:, None] * nrm

    def _adjacency(self):
        nb = [set() for _ in range(self.nv)]
        patch = [[] for _ in range(self.nv)]
        for e, el in enumerate(self.elems):
            for i, v in enumerate(el):
                patch[int(v)].append(e)
                for w in el:
                    if w != v:
                        nb[int(v)].add(int(w))
        self.neighbours = [sorted(s) for s in nb]
        self.patch = patch                                      # elements containing V, ascending

    # ------------------------------------------------------------------
    def local_index(self, e, v):
        return int(np.nonzero(self.elems[e] == v)[0][0])

    def barycentric_of_sorted_lattice(self, e, mi, p):
        """Barycentric coordinates (w.r.t. this element's own vertex order) of the lattice
        points defined on the ascending-sorted vertex ids (mtp_synth.lattice_points)."""
        el = self.elems[e]
        order = np.argsort(el, kind="stable")                 # order[k] = local index of k-th smallest
        lam_sorted = np.zeros((len(mi), self.dim + 1))
        lam_sorted[:, 1:] = mi / p
        lam_sorted[:, 0] = 1.0 - mi.sum(1) / p
        lam = np.zeros_like(lam_sorted)
        lam[:, order] = lam_sorted
        return lam
