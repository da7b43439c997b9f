"""Edge cases and failure paths on the GPU: one-element meshes, a single-layer evolve,
non-causal tents, non-finite input, and a device-side wait that is made to expire (the
kernel's bounded wait returns MTP_ETIMEOUT and the context stays usable)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from _oracle_bridge import oracle_full_run, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _one_element(dim):
    if dim == 2:
        v = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]])
        e = np.array([[0, 1, 2]], np.int32)
    else:
        v = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.1, 0.9, 0.1], [0.2, 0.1, 0.8]])
        e = np.array([[0, 1, 2, 3]], np.int32)
    one = np.ones(1)
    init = S.gaussian_pulse(np.full(dim, 0.3), 0.5)
    return S.Workload(f"one_element_{dim}d", dim, v, e, one, one.copy(), 3, 0.05, init=init)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", [mtp.MTP_FP64, mtp.MTP_FP32])
def test_single_element_mesh_matches_oracle(dim, precision):
    w = _one_element(dim)
    vals0, ref, _, _ = oracle_full_run(w)
    m = mtp.Mesh(dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=precision)
    t = m.pitch(w.T)
    st = m.state_from_lattice(torch.tensor(vals0[None], device=DEV))
    t.evolve(st)
    err = rel_l2(m.state_to_lattice(st).cpu().numpy()[0], ref)
    assert err <= (1e-11 if precision == mtp.MTP_FP64 else 1e-5), err


def test_short_evolve_with_few_layers():
    w = S.cube_mode(3, 2, 1e-3)
    vals0, ref, _, _ = oracle_full_run(w)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2)
    t = m.pitch(w.T)
    st = m.state_from_lattice(torch.tensor(vals0[None], device=DEV))
    t.evolve(st)
    assert rel_l2(m.state_to_lattice(st).cpu().numpy()[0], ref) <= 1e-11


def test_non_causal_tents_are_reported():
    """Tents pitched for a wave speed 4x too slow violate |grad phi| < sqrt(eps mu) (their tops
    are about 1.2x too steep)."""
    w = S.cube_mode(2, 2, 1.0)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2)
    t = m.pitch(w.T, causality_factor=0.9, wavespeed=0.25 * np.ones(len(w.elems)))
    st = m.new_state()
    with pytest.raises(mtp.MtpError) as ex:
        t.evolve(st)
    assert ex.value.code == mtp.MTP_ECAUSAL


def test_non_finite_state_is_reported():
    w = S.cube_mode(2, 2, 0.05)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2)
    t = m.pitch(w.T)
    st = m.new_state()
    st[0, 3, 1, 2] = float("nan")
    with pytest.raises(mtp.MtpError) as ex:
        t.evolve(st)
    assert ex.value.code == mtp.MTP_ENUMERIC


def test_expired_wait_returns_timeout_and_context_survives():
    w = S.cube_mode(2, 2, 0.1)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2, flags=mtp.MTP_FLAG_TEST_STALL)
    t = m.pitch(w.T)
    with pytest.raises(mtp.MtpError) as ex:
        t.evolve(m.new_state())
    assert ex.value.code == mtp.MTP_ETIMEOUT
    # the same process keeps working: a normal evolve afterwards
    m2 = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2)
    t2 = m2.pitch(w.T)
    st = m2.new_state()
    t2.evolve(st)
    torch.cuda.synchronize()
    assert float(st.abs().sum()) == 0.0
