"""Tent pitching for the oracle (test infrastructure only).

Sec. 2: fronts tau_i are vertex-valued (P1) times; a tent moves one vertex V
forward in time, its footprint is the vertex patch omega_V; vertices at graph
distance >= 2 move independently; heights are limited by the causality condition
|grad tau| < 1/c.  Sec. 5 uses slopes |grad phi| <= 1/(2c).

The paper gives no algorithm.  Reading used here (deterministic, exact in FP64
with every operation written out so that an independent implementation with
the same arithmetic order reproduces it bit for bit):

* Element geometry on the ascending-sorted vertex ids s_0 < ... < s_d:
  2D  det = (x1-x0)(y2-y0) - (x2-x0)(y1-y0);  height_i = |det| / |edge opposite i|
  3D  det = e1 . (e2 x e3) written out;        height_i = |det| / |(Pb-Pa) x (Pc-Pa)|
  where (a, b[, c]) are the other local indices in increasing order.
* k_V = min over elements containing V of the height at V.
* c_T = wavespeed[T] if given else 1/sqrt(eps_T mu_T); c_VW = max c_T over the
  elements containing edge VW.
* Edge bound b_VW = (cf * min(k_V, k_W)) / (d * c_VW).  Keeping
  |tau_V - tau_W| <= b_VW on every edge gives |grad tau|_T <= cf / c_T on every
  element (grad tau = sum_{j != i} (tau_j - tau_i) grad lambda_j and
  |grad lambda_j| = 1/height_j), i.e. the paper's slope bound for cf = 1/2.
* Rounds: select every V with tau_V < T that is a strict local minimum of
  (tau, index) among its neighbours (an independent set, so all selected tents
  are independent); its new time is min(T, min_W tau_W + b_VW) from the
  start-of-round times.  Tent layer = 1 + max(last layer of V and of its
  neighbours), starting at 0.  Output sorted by (layer, vertex).
"""
from __future__ import annotations

import math

import numpy as np


def element_heights(verts, elems):
    """heights[e, k] = height of element e at its k-th smallest vertex id; returns (heights, sorted ids)."""
    s = np.sort(np.asarray(elems, np.int64), axis=1)
    d = verts.shape[1]
    H = np.zeros(s.shape)
    for e in range(len(s)):
        P = [tuple(float(c) for c in verts[v]) for v in s[e]]
        if d == 2:
            det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1])
            adet = abs(det)
            for i in range(3):
                a, b = [k for k in range(3) if k != i]
                dx = P[b][0] - P[a][0]
                dy = P[b][1] - P[a][1]
                H[e, i] = adet / math.sqrt(dx * dx + dy * dy)
        else:
            e1 = [P[1][c] - P[0][c] for c in range(3)]
            e2 = [P[2][c] - P[0][c] for c in range(3)]
            e3 = [P[3][c] - P[0][c] for c in range(3)]
            det = (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1])
                   - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0])
                   + e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]))
            adet = abs(det)
            for i in range(4):
                a, b, c = [k for k in range(4) if k != i]
                u = [P[b][q] - P[a][q] for q in range(3)]
                w = [P[c][q] - P[a][q] for q in range(3)]
                cx = u[1] * w[2] - u[2] * w[1]
                cy = u[2] * w[0] - u[0] * w[2]
                cz = u[0] * w[1] - u[1] * w[0]
                H[e, i] = adet / math.sqrt(cx * cx + cy * cy + cz * cz)
    return H, s


def pitch_tents(verts, elems, eps, mu, T, cf=0.5, wavespeed=None, max_rounds=None):
    """Returns dict(vertex, t_bot, t_top, layer, layer_ptr) sorted by (layer, vertex).
    ``max_rounds`` stops after that many rounds (the front is then not at T)."""
    verts = np.asarray(verts, float)
    nv, d = verts.shape
    H, s = element_heights(verts, elems)
    ne = len(s)
    if wavespeed is None:
        c = np.array([1.0 / math.sqrt(float(eps[e]) * float(mu[e])) for e in range(ne)])
    else:
        c = np.asarray(wavespeed, float)
    k = np.full(nv, np.inf)
    edge_c = {}
    for e in range(ne):
        for i in range(d + 1):
            v = int(s[e, i])
            if H[e, i] < k[v]:
                k[v] = H[e, i]
            for j in range(i + 1, d + 1):
                key = (v, int(s[e, j]))
                if key not in edge_c or c[e] > edge_c[key]:
                    edge_c[key] = c[e]
    # directed-edge CSR (rows ascending by V, columns ascending by W)
    src, dst, bnd = [], [], []
    for (a, b), cab in edge_c.items():
        bab = (cf * min(k[a], k[b])) / (d * cab)
        src += [a, b]
        dst += [b, a]
        bnd += [bab, bab]
    order = np.lexsort((np.array(dst), np.array(src)))
    src = np.array(src, np.int64)[order]
    dst = np.array(dst, np.int64)[order]
    bnd = np.array(bnd, float)[order]
    ptr = np.zeros(nv + 1, np.int64)
    np.add.at(ptr, src + 1, 1)
    ptr = np.cumsum(ptr)
    starts = ptr[:-1]

    tau = np.zeros(nv)
    last = np.full(nv, -1, np.int64)
    tv, tb, tt, tl = [], [], [], []
    rounds = 0
    while max_rounds is None or rounds < max_rounds:
        rounds += 1
        active = tau < T
        if not active.any():
            break
        tv_src, tv_dst = tau[src], tau[dst]
        less = (tv_src < tv_dst) | ((tv_src == tv_dst) & (src < dst))
        is_min = np.logical_and.reduceat(less, starts) & active
        sel = np.nonzero(is_min)[0]
        cand = np.minimum.reduceat(tau[dst] + bnd, starts)
        lmax = np.maximum.reduceat(last[dst], starts)
        new = np.minimum(T, cand[sel])
        lay = 1 + np.maximum(last[sel], lmax[sel])
        tv.append(sel)
        tb.append(tau[sel].copy())
        tt.append(new)
        tl.append(lay)
        tau[sel] = new
        last[sel] = lay
    v = np.concatenate(tv)
    b = np.concatenate(tb)
    t = np.concatenate(tt)
    lay = np.concatenate(tl)
    o = np.lexsort((v, lay))
    v, b, t, lay = v[o], b[o], t[o], lay[o]
    nl = int(lay.max()) + 1 if len(lay) else 0
    layer_ptr = np.zeros(nl + 1, np.int64)
    np.add.at(layer_ptr, lay + 1, 1)
    layer_ptr = np.cumsum(layer_ptr)
    return {"vertex": v.astype(np.int32), "t_bot": b, "t_top": t, "layer": lay.astype(np.int32),
            "layer_ptr": layer_ptr, "k": k}


def pitch_first_round(verts, elems, eps, mu, T, cf=0.5, wavespeed=None):
    """Tents of the first round (all in layer 0, from the flat front t = 0): [(V, t_bot, t_top)]."""
    r = pitch_tents(verts, elems, eps, mu, T, cf, wavespeed, max_rounds=1)
    return [(int(v), float(b), float(t)) for v, b, t in zip(r["vertex"], r["t_bot"], r["t_top"])]
