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
from _oracle_bridge import max_rel, oracle_setup, rel_l2
from oracle.pitch import pitch_tents

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


@pytest.mark.parametrize("precision", [mtp.MTP_FP64, mtp.MTP_FP32])
def test_batch_matches_oracle_two_instances(precision):
    """Two instances of different size and degree (2^3 x 6 tets at p = 2 with 2 right-hand
    sides, 3^3 x 6 tets at p = 3 with 1) in one batch launch; every right-hand side is compared
    with the oracle's evolve of the same lattice data on the oracle's own tents."""
    rng = np.random.default_rng(45)
    tol = 1e-11 if precision == mtp.MTP_FP64 else 1e-5
    inst = []
    for n, p, nrhs in ((2, 2, 2), (3, 3, 1)):
        v, e = S.cube_mesh(n)
        one = np.ones(len(e))
        m = mtp.Mesh(3, v, e, one, one, p=p, precision=precision, n_rhs=nrhs)
        t = m.pitch(0.1)
        pts = S.lattice_points(v, e, p)
        vals = np.stack([np.concatenate(S.gaussian_pulse(c, 0.3)(pts), -1)
                         for c in rng.uniform(0.3, 0.7, size=(nrhs, 3))])
        st = m.state_from_lattice(torch.tensor(np.ascontiguousarray(vals), device=DEV))
        inst.append((m, t, st, S.Workload(f"batch_n{n}_p{p}", 3, v, e, one, one.copy(), p, 0.1), vals))
    b = mtp.Batch([t for _, t, _, _, _ in inst])
    b.evolve([st for _, _, st, _, _ in inst])
    for m, t, st, w, vals in inst:
        out = m.state_to_lattice(st).cpu().numpy()
        disc = oracle_setup(w)
        tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, w.causality)
        for r in range(len(vals)):
            Y, _ = disc.evolve(disc.moments_from_lattice(vals[r]), tents)
            ref = disc.eval_lattice(disc.y_coeffs(Y))
            err, emax = rel_l2(out[r], ref), max_rel(out[r], ref)
            print(f"{w.name} rhs {r}: rel l2 {err:.2e}, element-wise max {emax:.2e}")
            assert err <= tol and emax <= tol, (w.name, r, err, emax)
