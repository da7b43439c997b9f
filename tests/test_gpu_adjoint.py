"""Adjoint sweep (mtp_adjoint / MtpEvolveFunction) on the GPU, FP64.

* small mesh: dJ/deps and dJ/dmu against the oracle's discrete adjoint (same functional,
  states exchanged through the lattice)
* the adjoint workload at full size (8^3 x 6 tets, p = 2, eps ~ U[1, 3], T = 0.5): dJ/deps
  against central finite differences (h = 1e-6) of the GPU forward map, tents frozen
* <Phi x, y> = <x, Phi^T y> for the whole evolve; independence of the checkpoint interval
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from _oracle_bridge import rel_l2
from oracle.adjoint import evolve_adjoint, l2_misfit
from oracle.mesh import Mesh as OMesh
from oracle.mtp import Discretization
from oracle.pitch import pitch_tents

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _gpu_problem(w, eps, base_vals, target_vals):
    """Mesh with the given eps, frozen tents (wave speed 1), base coefficients of (E0, H0) and
    target E coefficients in the library basis."""
    m = mtp.Mesh(3, w.verts, w.elems, eps, w.mu, p=w.p)
    t = m.pitch(w.T, 0.5, wavespeed=np.ones(len(w.elems)))
    base = m.state_from_lattice(torch.tensor(base_vals[None], device=DEV))
    tgt = m.state_from_lattice(torch.tensor(target_vals[None], device=DEV))[:, :, :3, :]
    return m, t, base, tgt


def _J(m, t, base, tgt, eps_t, mu_t, grad=False):
    scale = torch.cat([eps_t[:, None].expand(-1, 3), mu_t[:, None].expand(-1, 3)], 1)   # [ne, 6]
    Y0 = base * scale[None, :, :, None]
    YT = mtp.mtp_evolve_autograd(Y0, eps_t, mu_t, t)
    E = YT[:, :, :3, :] / eps_t[None, :, None, None]
    return 0.5 * ((E - tgt) ** 2).sum()


def test_adjoint_matches_oracle_small():
    w = S.adjoint_cube(n=2, p=2, T=0.06, width=0.3)
    ws = np.ones(len(w.elems))
    tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, 0.5, ws)
    od = Discretization(OMesh(w.verts, w.elems, w.eps, w.mu), w.p)
    td = Discretization(OMesh(w.verts, w.elems, w.extra["eps_target"], w.mu), w.p)
    Yt, _ = td.evolve(td.project_initial(w.init), tents)
    Ut = td.fields_at_flat_front(Yt)
    Y0 = od.project_initial(w.init)
    YT, _ = od.evolve(Y0, tents)
    Jo, lamT, geps_final = l2_misfit(od, YT, Ut)
    lam0, geps_tent, gmu_tent = evolve_adjoint(od, tents, Y0, lamT)
    isE = np.isin(od.fs, [0, 1, 2])
    g_oracle = geps_final + geps_tent + np.einsum("era,era->e", lam0[:, isE], Y0[:, isE]) / w.eps
    # same discrete initial field and target on the GPU (through the lattice)
    base_vals = od.eval_lattice(od.fields_at_flat_front(Y0))          # (E0, H0) at the lattice
    tgt_vals = np.concatenate([od.eval_lattice(Ut)[..., :3], np.zeros(base_vals.shape[:-1] + (3,))], -1)
    m, t, base, tgt = _gpu_problem(w, w.eps, base_vals, tgt_vals)
    eps_t = torch.tensor(w.eps, device=DEV, requires_grad=True)
    mu_t = torch.tensor(w.mu, device=DEV, requires_grad=True)
    J = _J(m, t, base, tgt, eps_t, mu_t)
    J.backward()
    assert abs(J.item() - Jo) <= 1e-10 * Jo
    g = eps_t.grad.cpu().numpy()
    assert np.abs(g - g_oracle).max() <= 1e-9 * np.abs(g_oracle).max()
    gm = mu_t.grad.cpu().numpy()
    assert np.abs(gm - gmu_tent).max() <= 1e-9 * np.abs(gmu_tent).max()


def test_adjoint_workload_gradient_matches_central_fd():
    """8^3 x 6 tets, p = 2, eps ~ U[1,3] (seed 1), target from eps seed 2, Gaussian pulse, T = 0.5."""
    w = S.adjoint_cube(n=8, p=2, T=0.5)
    import mtp_synth
    pts = mtp_synth.lattice_points(w.verts, w.elems, w.p)
    E0, H0 = w.init(pts, 0.0)
    base_vals = np.ascontiguousarray(np.concatenate([E0, H0], -1))
    # target: E(T) of the GPU forward run with the second seeded eps
    mt, tt, bt, _ = _gpu_problem(w, w.extra["eps_target"], base_vals, base_vals)
    scale = torch.tensor(np.concatenate([np.repeat(w.extra["eps_target"][:, None], 3, 1),
                                         np.repeat(w.mu[:, None], 3, 1)], 1), device=DEV)
    Yt = (bt * scale[None, :, :, None]).contiguous()
    tt.evolve(Yt)
    Et = Yt[:, :, :3, :] / torch.tensor(w.extra["eps_target"], device=DEV)[None, :, None, None]
    tgt_vals = mt.state_to_lattice(torch.cat([Et, torch.zeros_like(Et)], 2).contiguous()).cpu().numpy()[0]

    def J_of(eps, grad=False):
        m, t, base, tgt = _gpu_problem(w, eps, base_vals, tgt_vals)
        eps_t = torch.tensor(eps, device=DEV, requires_grad=grad)
        mu_t = torch.tensor(w.mu, device=DEV)
        J = _J(m, t, base, tgt, eps_t, mu_t)
        if grad:
            J.backward()
            return J.item(), eps_t.grad.cpu().numpy()
        return J.item()

    J0, g = J_of(w.eps, grad=True)
    assert J0 > 0
    rng = np.random.default_rng(3)
    for e in rng.choice(len(w.elems), 4, replace=False):
        h = 1e-6
        ep, em = w.eps.copy(), w.eps.copy()
        ep[e] += h
        em[e] -= h
        fd = (J_of(ep) - J_of(em)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * np.abs(g).max(), (e, fd, g[e])


def test_adjoint_transpose_identity_and_checkpoint_interval():
    w = S.adjoint_cube(n=3, p=2, T=0.2)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2)
    t = m.pitch(w.T, 0.5, wavespeed=np.ones(len(w.elems)))
    rng = np.random.default_rng(9)
    x = torch.tensor(rng.standard_normal(m.state_shape), device=DEV)
    y = torch.tensor(rng.standard_normal(m.state_shape), device=DEV)
    Phix = x.clone()
    t.evolve(Phix)
    ne = len(w.elems)
    outs = []
    nl = t.info["n_layers"]
    for k in (0, 1, 7, nl):
        lam0 = torch.empty_like(x)
        ge = torch.empty(ne, dtype=torch.float64, device=DEV)
        gm = torch.empty(ne, dtype=torch.float64, device=DEV)
        mtp.mtp_adjoint(t.h, x, y, lam0, ge, gm, k)
        outs.append((lam0.cpu().numpy(), ge.cpu().numpy(), gm.cpu().numpy()))
    lhs = float((Phix * y).sum())
    rhs = float((x * torch.tensor(outs[0][0], device=DEV)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    for o in outs[1:]:
        assert rel_l2(o[0], outs[0][0]) < 1e-13
        assert rel_l2(o[1], outs[0][1]) < 1e-12
        assert rel_l2(o[2], outs[0][2]) < 1e-12
