"""Tent pitching with the rounds on the GPU (mtp_pitch_tents_device): the tent list must be
bit-identical to the oracle's pitcher (Sec. 2 rule, fixed FP64 operations) and to the host
pitcher, including when the device output buffers have to grow (millions of tents)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from oracle.pitch import pitch_tents

pytestmark = pytest.mark.gpu


def _same(got, ref):
    for k in ("vertex", "layer", "layer_ptr"):
        assert np.array_equal(got[k], ref[k]), k
    for k in ("t_bot", "t_top"):
        assert np.array_equal(got[k].view(np.uint64), ref[k].view(np.uint64)), k   # bit-exact


def _square_perturbed():
    v, e = S.square_mesh(6)
    return S.Workload("sq_pert", 2, S.perturb_interior(v, 1 / 6, 0.2, 3), e, np.ones(len(e)), np.ones(len(e)), 1, 0.3)


def _one_triangle():
    v = np.array([[0.0, 0.0], [1.0, 0.1], [0.3, 0.8]])
    return S.Workload("tri", 2, v, np.array([[0, 1, 2]], np.int32), np.ones(1), np.ones(1), 1, 0.4)


CASES = {
    "te_square8": lambda: S.te_square(8, 2, 0.5),
    "square_perturbed": _square_perturbed,
    "one_triangle": _one_triangle,
    "cube6_perturbed": lambda: S.cube_mode(6, 1, 0.3),
    "graded6_eps_jump": lambda: S.graded_sphere(n=6, p=1, T=0.2),
    "cube4_random_eps": lambda: S.adjoint_cube(n=4, p=1, T=0.3),
    "cube4_short_T": lambda: S.cube_mode(4, 1, 1e-3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_device_pitcher_matches_oracle_and_host(name):
    w = CASES[name]()
    ref = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, 0.5, None)
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=1)
    td = m.pitch(w.T, 0.5, device=True)
    th = m.pitch(w.T, 0.5)
    _same(td.get(), ref)
    _same(td.get(), th.get())
    assert td.info == th.info


def test_device_pitcher_with_wavespeed_and_factor():
    w = S.adjoint_cube(n=3, p=1, T=0.2)
    ws = np.linspace(0.5, 1.5, len(w.elems))
    ref = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, 0.4, ws)
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=1)
    _same(m.pitch(w.T, 0.4, ws, device=True).get(), ref)


def test_device_pitched_tents_evolve_identically():
    w = S.te_square(6, 2, 0.3)
    m = mtp.Mesh(2, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=mtp.MTP_FP64)
    pts = S.lattice_points(w.verts, w.elems, w.p)
    E, H = w.init(pts, 0.0)
    y = np.ascontiguousarray(np.concatenate([E, H], -1)[..., [0, 1, 5]])
    out = []
    for device in (False, True):
        t = m.pitch(w.T, 0.5, device=device)
        st = m.state_from_lattice(torch.tensor(y[None], device="cuda"))
        t.evolve(st)
        out.append(m.state_to_lattice(st).cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_device_pitcher_graded32_matches_host():
    """The benchmarked mesh: 9.0 M tents in 10 091 layers, so the device output arrays and
    the layer pointers are grown several times during the rounds."""
    w = S.graded_sphere(32, 4, 0.5)
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=mtp.MTP_FP32)
    t0 = time.perf_counter()
    th = m.pitch(w.T, w.causality)
    t1 = time.perf_counter()
    td = m.pitch(w.T, w.causality, device=True)
    t2 = time.perf_counter()
    _same(td.get(), th.get())
    assert td.info == th.info
    print(f"graded 32^3: {td.info['n_tents']} tents, host pitch {t1 - t0:.2f} s, device pitch {t2 - t1:.2f} s")
