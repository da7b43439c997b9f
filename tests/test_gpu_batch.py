"""Many instances (different meshes, degrees and right-hand-side counts) in one persistent
launch: each instance's result equals its own evolve (same tent maps; the batch kernel is a
separate compilation, so agreement is to rounding, not bit for bit)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from _oracle_bridge import rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _instances(precision):
    """The many-instance recipe at reduced size: n ~ U{2..4}, p ~ U{1..4}, 1-4 pulse RHS."""
    rng = np.random.default_rng(44)
    out = []
    for i in range(6):
        n = int(rng.integers(2, 5))
        p = [1, 2, 3, 4, 2, 3][i]
        nrhs = int(rng.integers(1, 5))
        v, e = S.cube_mesh(n)
        one = np.ones(len(e))
        m = mtp.Mesh(3, v, e, one, one, p=p, precision=precision, n_rhs=nrhs)
        t = m.pitch(0.1)
        centres = rng.uniform(0.3, 0.7, size=(nrhs, 3))
        pts = S.lattice_points(v, e, p)
        vals = np.stack([np.concatenate(S.gaussian_pulse(c, 0.3)(pts), -1) for c in centres])
        st = m.state_from_lattice(torch.tensor(np.ascontiguousarray(vals), device=DEV))
        out.append((m, t, st))
    return out


@pytest.mark.parametrize("precision", [mtp.MTP_FP64, mtp.MTP_FP32])
def test_batch_equals_individual_evolves(precision):
    inst = _instances(precision)
    refs = []
    for m, t, st in inst:
        r = st.clone()
        t.evolve(r)
        refs.append(r.cpu().numpy())
    b = mtp.Batch([t for _, t, _ in inst])
    assert b.info["n_instances"] == len(inst)
    assert b.info["n_tents"] == sum(t.info["n_tents"] for _, t, _ in inst)
    states = [st.clone() for _, _, st in inst]
    b.evolve(states)
    tol = 1e-13 if precision == mtp.MTP_FP64 else 2e-6
    for s, r in zip(states, refs):
        assert rel_l2(s.cpu().numpy(), r) <= tol
    # second evolve from the same inputs gives the same result (counters and fronts reset)
    states2 = [st.clone() for _, _, st in inst]
    b.evolve(states2)
    for s, s2 in zip(states, states2):
        assert np.array_equal(s.cpu().numpy(), s2.cpu().numpy())


def test_batch_rejects_mixed_precision():
    a = mtp.Mesh(3, *S.cube_mesh(2), np.ones(48), np.ones(48), p=2, precision=mtp.MTP_FP64)
    c = mtp.Mesh(3, *S.cube_mesh(2), np.ones(48), np.ones(48), p=2, precision=mtp.MTP_FP32)
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Batch([a.pitch(0.1), c.pitch(0.1)])
    assert ex.value.code == mtp.MTP_EINVAL
