"""CUDA path vs the FP64 oracle, through the C ABI (GB300).

States are exchanged through lattice values of the conserved variable y (basis
independent), so the oracle (Bernstein basis, dense LU, exact integrals) and the
CUDA path (orthonormal basis, closed-form mass inverse) share no arithmetic.

Tolerances (per the required precision contract): FP64 mode <= 1e-11, FP32 mode <= 1e-5,
asserted twice: as one relative L2 over all compared lattice values, and element-wise as the
largest pointwise difference over the largest reference value (so that an error confined to
one element, one facet or one patch of a large mesh cannot hide in the global norm).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from _oracle_bridge import max_rel, oracle_full_run, oracle_layers, oracle_setup, oracle_single_tents, rel_l2
from oracle.pitch import pitch_tents

pytestmark = pytest.mark.gpu
TOL = {mtp.MTP_FP64: 1e-11, mtp.MTP_FP32: 1e-5, mtp.MTP_FP32_SPLIT: 1e-5}
DEV = "cuda:0"


def _gpu_full(w, precision, vals0, n_rhs=1, wavespeed=None):
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=precision, n_rhs=n_rhs)
    t = m.pitch(w.T, w.causality, wavespeed)
    v0 = torch.tensor(np.broadcast_to(vals0, (n_rhs,) + vals0.shape).copy(), device=DEV)
    st = m.state_from_lattice(v0)
    e0 = m.energy(st)
    t.evolve(st)
    out = m.state_to_lattice(st).cpu().numpy()
    e1 = m.energy(st)
    torch.cuda.synchronize()
    return out, e0, e1


_CASES = {
    "te_square_n8_p2": lambda: S.te_square(8, 2, 0.5),            # the 2D TE cavity workload in full
    "te_square_n4_p1": lambda: S.te_square(4, 1, 0.3),
    "te_square_n3_p4": lambda: S.te_square(3, 4, 0.15),
    "cube_n2_p2": lambda: S.cube_mode(2, 2, 0.12),
    "cube_n2_p3": lambda: S.cube_mode(2, 3, 0.1),
    "cube_n2_p1": lambda: S.cube_mode(2, 1, 0.15),
    "graded_n3_p2": lambda: S.graded_sphere(n=3, p=2, T=0.06, width=0.3),   # eps jump + grading
    "cube_n2_p4": lambda: S.cube_mode(2, 4, 0.04),
    "te_square_n3_p5": lambda: S.te_square(3, 5, 0.1),
    "cube_n2_p5": lambda: S.cube_mode(2, 5, 0.015),
}
_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        _ORACLE[name] = oracle_full_run(_CASES[name]())
    return _ORACLE[name]


@pytest.mark.parametrize("precision", [mtp.MTP_FP64, mtp.MTP_FP32, mtp.MTP_FP32_SPLIT])
@pytest.mark.parametrize("name", list(_CASES))
def test_full_evolve_matches_oracle(name, precision):
    w = _CASES[name]()
    if name == "cube_n2_p5" and precision == mtp.MTP_FP64:
        # a 24-tet patch of degree 5 in FP64 needs more shared memory than one block may have
        m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=5, precision=precision)
        with pytest.raises(mtp.MtpError) as ex:
            m.pitch(w.T).evolve(m.new_state())
        assert ex.value.code == mtp.MTP_EUNSUPPORTED
        return
    vals0, ref, oe0, oe1 = _oracle(name)
    out, e0, e1 = _gpu_full(w, precision, vals0)
    err = rel_l2(out[0], ref)
    emax = max_rel(out[0], ref)
    print(f"{name} precision {precision}: rel l2 {err:.2e}, element-wise max {emax:.2e}")
    assert err <= TOL[precision], (name, precision, err)
    assert emax <= TOL[precision], (name, precision, emax)
    assert abs(e0[0] - oe0) <= 10 * TOL[precision] * oe0
    assert abs(e1[0] - oe1) <= 10 * TOL[precision] * oe1
    assert e1[0] <= e0[0] * (1 + 1e-12 if precision == mtp.MTP_FP64 else 1 + 1e-5)


def test_multi_rhs_equals_single():
    w = S.cube_mode(2, 2, 0.12)
    vals0, _, _, _ = _oracle("cube_n2_p2")
    rng = np.random.default_rng(5)
    stack = np.stack([vals0, rng.standard_normal(vals0.shape), 0.5 * vals0])
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2, n_rhs=3)
    t = m.pitch(w.T)
    st = m.state_from_lattice(torch.tensor(stack, device=DEV))
    t.evolve(st)
    many = m.state_to_lattice(st).cpu().numpy()
    for r in range(3):
        one, _, _ = _gpu_full(w, mtp.MTP_FP64, stack[r])
        assert np.array_equal(one[0], many[r])


def test_fp64_deterministic_and_host_entry_point():
    w = S.cube_mode(2, 3, 0.1)
    vals0, _, _, _ = _oracle("cube_n2_p3")
    a, _, _ = _gpu_full(w, mtp.MTP_FP64, vals0)
    b, _, _ = _gpu_full(w, mtp.MTP_FP64, vals0)
    assert np.array_equal(a, b)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=3)
    t = m.pitch(w.T)
    st = m.state_from_lattice(torch.tensor(vals0[None], device=DEV))
    host_in = st.cpu().numpy().copy()
    host_out = np.empty_like(host_in)
    t.evolve_host(host_in, host_out)
    t.evolve(st)
    assert np.array_equal(host_out, st.cpu().numpy())


def test_lattice_roundtrip_and_T_mismatch():
    w = S.graded_sphere(n=3, p=4, T=0.05)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=4)
    v = torch.tensor(np.random.default_rng(1).standard_normal(m.lattice_shape), device=DEV)
    back = m.state_to_lattice(m.state_from_lattice(v))
    assert rel_l2(back.cpu().numpy(), v.cpu().numpy()) < 1e-12
    t = m.pitch(w.T)
    with pytest.raises(mtp.MtpError) as ex:
        mtp.mtp_evolve(t.h, m.new_state(), w.T * 2)
    assert ex.value.code == mtp.MTP_EINVAL


def _oracle_tents_prefix(w, gpu_tents, n_layers):
    """The oracle pitcher's first n_layers layers, checked bit for bit against the library's
    list (the oracle side never takes its input from the library)."""
    key = ("tents", w.name, n_layers)
    if key not in _ORACLE:
        _ORACLE[key] = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, w.causality, max_rounds=n_layers)
    ot = _ORACLE[key]
    n = len(ot["vertex"])
    assert np.array_equal(ot["layer_ptr"], gpu_tents["layer_ptr"][: n_layers + 1])
    assert np.array_equal(ot["vertex"], gpu_tents["vertex"][:n])
    assert np.array_equal(ot["t_top"].view(np.uint64), gpu_tents["t_top"][:n].view(np.uint64))
    return ot


def _single_layer_check(w, precision, layer_frac, n_sample, seed, variant=0):
    """Full-size workload, the launch configuration of a real evolve: one layer applied to a
    seeded random state on the GPU; the oracle recomputes a sample of that layer's tents."""
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=precision)
    t = m.pitch(w.T, w.causality)
    t.set_variant(variant)
    gpu_tents = t.get()
    L = int(layer_frac * (len(gpu_tents["layer_ptr"]) - 1))
    tents = _oracle_tents_prefix(w, gpu_tents, L + 1)
    vals = np.random.default_rng(seed).standard_normal(m.lattice_shape[1:])
    st = m.state_from_lattice(torch.tensor(vals[None], device=DEV))
    t.evolve_layers(st, L, L + 1)
    out = m.state_to_lattice(st).cpu().numpy()[0]
    lp = tents["layer_ptr"]
    idx = np.arange(lp[L], lp[L + 1])
    sample = np.random.default_rng(seed + 1).choice(idx, size=min(n_sample, len(idx)), replace=False)
    disc = oracle_setup(w)
    ref = oracle_single_tents(w, disc, tents, L, vals, sample)
    errs = []
    for tt, r in ref.items():
        patch = disc.mesh.patch[int(tents["vertex"][tt])]
        errs.append(max(rel_l2(out[patch], r), max_rel(out[patch], r)))
    # elements outside the layer's patches are untouched
    touched = np.zeros(len(w.elems), bool)
    for tt in idx:
        touched[disc.mesh.patch[int(tents["vertex"][tt])]] = True
    assert rel_l2(out[~touched], vals[~touched]) < (1e-14 if precision == mtp.MTP_FP64 else 1e-7)
    return max(errs)


@pytest.mark.parametrize("precision", [mtp.MTP_FP64, mtp.MTP_FP32])
def test_cube16_p3_single_layer_sampled(precision):
    """3D cavity workload at full size (16^3 x 6 perturbed tets, p = 3, T = 1)."""
    w = S.cube_mode(16, 3, 1.0)
    err = _single_layer_check(w, precision, 0.5, 6, 101)
    assert err <= TOL[precision], err


@pytest.mark.parametrize("precision,variant", [(mtp.MTP_FP64, 0), (mtp.MTP_FP32, 0), (mtp.MTP_FP32, 3)])
def test_graded32_p4_single_layer_sampled(precision, variant):
    """Graded 32^3 x 6 tets, p = 4, eps = 4 ball (full size of the mixed-precision workload);
    variant 3 computes the volume term on the tcgen05 tensor cores."""
    w = S.graded_sphere(32, 4, 0.5)
    err = _single_layer_check(w, precision, 0.3, 3, 202, variant)
    assert err <= TOL[precision], err


@pytest.mark.parametrize("precision,variant", [(mtp.MTP_FP64, 0), (mtp.MTP_FP32, 0), (mtp.MTP_FP32_SPLIT, 0),
                                               (mtp.MTP_FP32, 3), (mtp.MTP_FP32, 4)])
def test_cube16_p3_twenty_layers_dag_walk(precision, variant):
    """3D cavity workload at full size (16^3 x 6 perturbed tets, p = 3, T = 1): 20 consecutive
    layers from the middle of the evolve applied by the persistent DAG walk (one launch, the
    bench's launch configuration) to a seeded random state; the oracle applies every tent of
    the same 20 layers.  Compared on every element the layers touch.  Variants 3 and 4 run the
    volume term on the tcgen05 tensor cores."""
    w = S.cube_mode(16, 3, 1.0)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=3, precision=precision)
    t = m.pitch(w.T, w.causality)
    t.set_variant(variant)
    tents = t.get()
    L0 = (len(tents["layer_ptr"]) - 1) // 2
    L1 = L0 + 20
    vals = np.random.default_rng(303).standard_normal(m.lattice_shape[1:])
    st = m.state_from_lattice(torch.tensor(vals[None], device=DEV))
    t.evolve_layers(st, L0, L1)
    out = m.state_to_lattice(st).cpu().numpy()[0]
    tents = _oracle_tents_prefix(w, tents, L1)
    key = ("cube16_layers", L0, L1)
    if key not in _ORACLE:
        _ORACLE[key] = oracle_layers(w, tents, L0, L1, vals)
    ref = _ORACLE[key]
    lp = tents["layer_ptr"]
    disc_patch = oracle_setup(w).mesh.patch
    touched = np.zeros(len(w.elems), bool)
    for tt in range(lp[L0], lp[L1]):
        touched[disc_patch[int(tents["vertex"][tt])]] = True
    err, emax = rel_l2(out[touched], ref[touched]), max_rel(out[touched], ref[touched])
    print(f"20 layers ({lp[L1] - lp[L0]} tents, {touched.sum()} elements): rel l2 {err:.2e}, "
          f"element-wise max {emax:.2e}")
    assert err <= TOL[precision] and emax <= TOL[precision], (err, emax)
    assert np.array_equal(ref[~touched], vals[~touched]) or rel_l2(ref[~touched], vals[~touched]) < 1e-13
    assert rel_l2(out[~touched], vals[~touched]) < (1e-14 if precision != mtp.MTP_FP32 else 1e-7)


def test_pitcher_on_device_box_matches_oracle():
    w = S.cube_mode(8, 2, 0.4)
    ref = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, 0.5)
    got = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2).pitch(w.T).get()
    for k in ("vertex", "layer", "layer_ptr"):
        assert np.array_equal(got[k], ref[k])
    assert np.array_equal(got["t_top"].view(np.uint64), ref["t_top"].view(np.uint64))


@pytest.mark.parametrize("name", ["cube_n2_p3", "te_square_n8_p2"])
def test_persistent_dag_walk_equals_layer_launches(name):
    """The persistent DAG-walking evolve and the per-layer launches apply the same tent maps:
    FP64 results are bit-identical (each tent's arithmetic does not depend on scheduling)."""
    w = _CASES[name]()
    vals0, _, _, _ = _oracle(name)
    outs = []
    for flags in (0, mtp.MTP_FLAG_LAYER_LAUNCHES):
        m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, n_rhs=2, flags=flags)
        t = m.pitch(w.T)
        st = m.state_from_lattice(torch.tensor(np.stack([vals0, 2 * vals0]), device=DEV))
        t.evolve(st)
        outs.append(st.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_fp32_error_against_discretisation_error_cube16():
    """FP32 rounding vs discretisation error on the 3D cavity workload (16^3 x 6 perturbed tets,
    p = 3, T = 1, exact (1,1,1) mode known; lattice l2 norms).  Plain FP32 (measured on GB300:
    FP64 discretisation error 1.83e-5, FP32-vs-FP64 distance 5.1e-6, ratio 0.28) stays inside the
    1e-5 FP32 tolerance but not within a tenth of the discretisation error; the split mode (Taylor
    sum as an FP32 hi + lo pair, FP64 state between tents) must reach that tenth."""
    w = S.cube_mode(16, 3, 1.0)
    pts = S.lattice_points(w.verts, w.elems, w.p)
    E0, H0 = w.exact(pts, 0.0)
    ET, HT = w.exact(pts, w.T)
    exact_T = np.concatenate([ET, HT], -1)
    outs = {}
    for prec in (mtp.MTP_FP64, mtp.MTP_FP32, mtp.MTP_FP32_SPLIT):
        m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=prec)
        t = m.pitch(w.T)
        st = m.state_from_lattice(torch.tensor(np.concatenate([E0, H0], -1)[None], device=DEV))
        t.evolve(st)
        outs[prec] = m.state_to_lattice(st).cpu().numpy()[0]
    e_disc = rel_l2(outs[mtp.MTP_FP64], exact_T)
    e32 = rel_l2(outs[mtp.MTP_FP32], outs[mtp.MTP_FP64])
    esplit = rel_l2(outs[mtp.MTP_FP32_SPLIT], outs[mtp.MTP_FP64])
    print(f"e_disc {e_disc:.3e}  fp32-vs-fp64 {e32:.3e} ({e32 / e_disc:.3f} e_disc)  "
          f"split-vs-fp64 {esplit:.3e} ({esplit / e_disc:.3f} e_disc)")
    assert e_disc < 1e-4
    assert e32 <= 1e-5
    assert e32 <= 0.35 * e_disc
    assert esplit <= 0.1 * e_disc


# Tensor-core modes (3D): TF32 operands have a unit roundoff of 2^-11 ~ 4.9e-4, so a tent
# (m q = 12..40 stages of contractions over up to 3 x 35 products) stays within ~1e-3 relative;
# the 3-term hi + lo split recovers FP32-level products (tolerance as FP32).
TC_TOL = {mtp.MTP_TF32: 3e-3, mtp.MTP_TF32X3: 1e-5}


@pytest.mark.parametrize("precision", [mtp.MTP_TF32, mtp.MTP_TF32X3])
@pytest.mark.parametrize("name", ["cube_n2_p1", "cube_n2_p2", "cube_n2_p3", "cube_n2_p4", "graded_n3_p2"])
def test_tensor_core_modes_match_oracle(name, precision):
    w = _CASES[name]()
    vals0, ref, _, _ = _oracle(name)
    out, e0, e1 = _gpu_full(w, precision, vals0)
    err = rel_l2(out[0], ref)
    print(f"{name} mode {precision}: rel l2 {err:.2e}")
    assert err <= TC_TOL[precision], (name, precision, err)


@pytest.mark.parametrize("precision", [mtp.MTP_TF32, mtp.MTP_TF32X3])
def test_tensor_core_modes_graded32_single_layer(precision):
    w = S.graded_sphere(32, 4, 0.5)
    err = _single_layer_check(w, precision, 0.3, 3, 202)
    print(f"graded32 single layer mode {precision}: {err:.2e}")
    assert err <= TC_TOL[precision], err
