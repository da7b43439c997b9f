"""Launch configurations and the autotuner on the GPU, and the paper's convergence claim
(Sec. 5.1, Fig. 3 left) reproduced with the CUDA path: O(h^{p+1}) for p = 1..4 with
(p+1)-stage SAT and m = 2p on the 2D cavity, and for p = 1..3 on the 3D (1,1,1) cavity mode."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from paper_1906_11029_gb300 import tune

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _vals(w):
    pts = S.lattice_points(w.verts, w.elems, w.p)
    E, H = w.init(pts, 0.0)
    fs = [0, 1, 5] if w.dim == 2 else list(range(6))
    return np.ascontiguousarray(np.concatenate([E, H], -1)[..., fs][None])


def test_launch_configurations_agree_and_window_evolve():
    """DAG walk (two CTA counts) and per-layer launches give bit-identical FP64 results, for a
    full evolve and for a window of layers started mid-run."""
    w = S.cube_mode(3, 2, 0.3)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2)
    t = m.pitch(w.T)
    v = torch.tensor(_vals(w), device=DEV)
    outs = []
    nl = t.info["n_layers"]
    for launch in (0, 1, 2):
        t.set_launch(launch)
        st = m.state_from_lattice(v)
        t.evolve(st)
        s2 = m.state_from_lattice(v)
        t.evolve_layers(s2, 0, nl // 3)
        t.evolve_layers(s2, nl // 3, nl)
        outs.append((st.cpu().numpy(), s2.cpu().numpy()))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[1], outs[0][1])
    assert np.array_equal(outs[0][0], outs[0][1])


def test_autotuner_picks_and_caches(tmp_path):
    w = S.graded_sphere(6, 3, 0.1)
    cache = str(tmp_path / "tune.json")
    prec, launch, rec = tune.autotune(3, w.verts, w.elems, w.eps, w.mu, w.p, w.T, _vals(w),
                                      accuracy="fp32", cache=cache)
    assert prec in (mtp.MTP_FP32, mtp.MTP_TF32X3) and launch in (0, 1, 2)
    assert os.path.exists(cache)
    assert len(rec["candidates"]) == 6 and all(len(c["launch_ms"]) == 3 for c in rec["candidates"])
    assert rec["variant"] in (0, 1, 2, 3, 4)
    assert {(c["precision"], c["variant"]) for c in rec["candidates"]} == {
        (mtp.MTP_FP32, 0), (mtp.MTP_FP32, 1), (mtp.MTP_FP32, 2), (mtp.MTP_FP32, 3), (mtp.MTP_FP32, 4),
        (mtp.MTP_TF32X3, 0)}
    again = tune.autotune(3, w.verts, w.elems, w.eps, w.mu, w.p, w.T, _vals(w), accuracy="fp32", cache=cache)
    assert again[0] == prec and again[1] == launch


def _lattice_error(p, n):
    w = S.te_square(n, p, 0.5)
    m = mtp.Mesh(2, w.verts, w.elems, w.eps, w.mu, p=p)
    t = m.pitch(w.T)
    st = m.state_from_lattice(torch.tensor(_vals(w), device=DEV))
    t.evolve(st)
    got = m.state_to_lattice(st).cpu().numpy()[0]
    pts = S.lattice_points(w.verts, w.elems, p)
    E, H = w.exact(pts, w.T)
    ref = np.concatenate([E, H], -1)[..., [0, 1, 5]]
    return float(np.linalg.norm(got - ref) / math.sqrt(ref.size))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cavity_convergence_rate_gpu(p):
    ns = (4, 8, 16, 32) if p <= 2 else (4, 8, 16)
    errs = [_lattice_error(p, n) for n in ns]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print(f"p={p} errors {['%.2e' % e for e in errs]} rates {['%.2f' % r for r in rates]}")
    assert rates[-1] > p + 0.7, (errs, rates)


def _lattice_error_3d(p, n):
    w = S.cube_mode(n, p, 0.25, perturb=0.0)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=p)
    t = m.pitch(w.T)
    st = m.state_from_lattice(torch.tensor(_vals(w), device=DEV))
    t.evolve(st)
    got = m.state_to_lattice(st).cpu().numpy()[0]
    pts = S.lattice_points(w.verts, w.elems, p)
    E, H = w.exact(pts, w.T)
    ref = np.concatenate([E, H], -1)
    return float(np.linalg.norm(got - ref) / math.sqrt(ref.size))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_cube_cavity_convergence_rate_gpu(p):
    ns = (4, 8, 16)
    errs = [_lattice_error_3d(p, n) for n in ns]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print(f"3D p={p} errors {['%.2e' % e for e in errs]} rates {['%.2f' % r for r in rates]}")
    assert rates[-1] > p + 0.7, (errs, rates)
