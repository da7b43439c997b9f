"""The Y-substituted classical RK4 tent stepper (MTP_FLAG_SUBSTITUTED_RK4) on the GPU, FP64:
the negative control of Sec. 3 (after eq. equ_ode) and Sec. 5.1 (Fig. 3 right).

* parity: the same tents advanced by the oracle's ``evolve_substituted_rk4`` (1e-11, L2 and
  element-wise);
* order loss on the 2D TE cavity at p = 4: SAT's error falls like h^5, while the RK4
  time-stepping error (its distance from SAT on the same tents) falls at an order near 1 to 2
  and overtakes SAT's whole error on the finer meshes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from _oracle_bridge import max_rel, oracle_setup, rel_l2
from oracle.brute import evolve_substituted_rk4
from oracle.pitch import pitch_tents

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _gpu(w, vals0, flags):
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=mtp.MTP_FP64, flags=flags)
    t = m.pitch(w.T, w.causality)
    st = m.state_from_lattice(torch.tensor(vals0[None], device=DEV))
    t.evolve(st)
    return m.state_to_lattice(st).cpu().numpy()[0]


@pytest.mark.parametrize("case", ["te_square_n4_p2", "cube_n2_p2", "graded_n3_p2"])
def test_substituted_rk4_matches_oracle(case):
    w = {"te_square_n4_p2": lambda: S.te_square(4, 2, 0.25), "cube_n2_p2": lambda: S.cube_mode(2, 2, 0.1),
         "graded_n3_p2": lambda: S.graded_sphere(n=3, p=2, T=0.06, width=0.3)}[case]()
    disc = oracle_setup(w)
    tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, w.causality)
    Y0 = disc.project_initial(w.init)
    vals0 = disc.eval_lattice(disc.y_coeffs(Y0))
    Y = evolve_substituted_rk4(disc, Y0, tents, 2 * w.p)
    ref = disc.eval_lattice(disc.y_coeffs(Y))
    out = _gpu(w, vals0, mtp.MTP_FLAG_SUBSTITUTED_RK4)
    err, emax = rel_l2(out, ref), max_rel(out, ref)
    print(f"{case}: rel l2 {err:.2e}, element-wise max {emax:.2e}")
    assert err <= 1e-11 and emax <= 1e-11, (err, emax)
    # and it is a different scheme from SAT
    assert rel_l2(_gpu(w, vals0, 0), ref) > 1e-9


def test_substituted_rk4_loses_order_on_te_cavity_p4():
    p, rows = 4, []
    for n in (4, 8, 16, 32):
        w = S.te_square(n, p, 0.25)
        pts = S.lattice_points(w.verts, w.elems, p)
        E0, H0 = w.exact(pts, 0.0)
        ET, HT = w.exact(pts, w.T)
        vals0 = np.ascontiguousarray(np.concatenate([E0, H0], -1)[..., [0, 1, 5]])
        exact = np.concatenate([ET, HT], -1)[..., [0, 1, 5]]
        sat = _gpu(w, vals0, 0)
        rk = _gpu(w, vals0, mtp.MTP_FLAG_SUBSTITUTED_RK4)
        rows.append((n, rel_l2(sat, exact), rel_l2(rk, exact), rel_l2(rk, sat)))
    for r in rows:
        print("n %d  SAT %.3e  RK4 %.3e  RK4-SAT %.3e" % r)
    sat_rate = np.log2(rows[1][1] / rows[3][1]) / 2
    rk_rate = np.log2(rows[1][3] / rows[3][3]) / 2
    assert sat_rate > p + 0.5, rows
    assert rk_rate < 2.5, rows
    assert rows[3][2] > 3 * rows[3][1], rows
