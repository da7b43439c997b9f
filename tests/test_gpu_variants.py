"""Kernel shape variants 1 (one patch element per stage item) and 2 (one element and one row per
item, 512 threads), and 3, 4 (those item shapes with the volume term on the tcgen05 tensor
cores, 3xTF32 with FP32 accumulation in tensor memory) selected with mtp_tents_set_variant,
against the default paired variant and against the oracle, FP32."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from _oracle_bridge import max_rel, oracle_full_run, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(w, vals0, variant, launch=0):
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=mtp.MTP_FP32)
    t = m.pitch(w.T, w.causality)
    t.set_variant(variant)
    t.set_launch(launch)
    st = m.state_from_lattice(torch.tensor(vals0[None], device=DEV))
    t.evolve(st)
    return m.state_to_lattice(st).cpu().numpy()[0]


@pytest.mark.parametrize("name", ["cube_n2_p3", "cube_n2_p4", "graded_n3_p2", "te_square_n4_p3", "cube_n2_p5"])
def test_variants_match_oracle_and_variant0(name):
    w = {"cube_n2_p3": lambda: S.cube_mode(2, 3, 0.1), "cube_n2_p4": lambda: S.cube_mode(2, 4, 0.04),
         "graded_n3_p2": lambda: S.graded_sphere(n=3, p=2, T=0.06, width=0.3),
         "te_square_n4_p3": lambda: S.te_square(4, 3, 0.2), "cube_n2_p5": lambda: S.cube_mode(2, 5, 0.015)}[name]()
    vals0, ref, _, _ = oracle_full_run(w)
    v0 = _run(w, vals0, 0)
    for variant in (1, 2):
        for launch in (0, 2):
            v1 = _run(w, vals0, variant, launch)
            err, emax = rel_l2(v1, ref), max_rel(v1, ref)
            print(f"{name} variant {variant} launch {launch}: rel l2 {err:.2e}, element-wise max {emax:.2e}, "
                  f"vs variant 0 {rel_l2(v1, v0):.2e}")
            assert err <= 1e-5 and emax <= 1e-5, (err, emax)
            assert rel_l2(v1, v0) <= 2e-6


_TC5_CASES = {
    "cube_n2_p2": lambda: S.cube_mode(2, 2, 0.12),
    "cube_n2_p3": lambda: S.cube_mode(2, 3, 0.1),
    "cube_n2_p4": lambda: S.cube_mode(2, 4, 0.04),
    "graded_n3_p2": lambda: S.graded_sphere(n=3, p=2, T=0.06, width=0.3),   # eps jump: impedances differ
    "graded_n3_p4": lambda: S.graded_sphere(n=3, p=4, T=0.03, width=0.3),
}


@pytest.mark.parametrize("name", list(_TC5_CASES))
def test_tcgen05_variants_match_oracle_and_variant0(name):
    """Patches from 1 to 24 tetrahedra: up to 128 (element, field) rows take one MMA chunk, the
    24-tet interior patches (144 rows) two.  Both the persistent DAG walk and per-layer
    launches (each CTA allocates and frees its own tensor memory)."""
    w = _TC5_CASES[name]()
    vals0, ref, _, _ = oracle_full_run(w)
    v0 = _run(w, vals0, 0)
    for variant in (3, 4):
        for launch in (0, 2):
            v1 = _run(w, vals0, variant, launch)
            err, emax = rel_l2(v1, ref), max_rel(v1, ref)
            print(f"{name} variant {variant} launch {launch}: rel l2 {err:.2e}, element-wise max {emax:.2e}, "
                  f"vs variant 0 {rel_l2(v1, v0):.2e}")
            assert err <= 1e-5 and emax <= 1e-5, (err, emax)
            assert rel_l2(v1, v0) <= 5e-6


def test_tcgen05_variant_multi_rhs_equals_single():
    """Several right-hand sides in one DAG-walk CTA (the MMA mbarrier phase carries over from
    one right-hand side and tent to the next) and in per-layer launches (one CTA per tent and
    right-hand side): each equals its own single-RHS evolve."""
    w = S.cube_mode(2, 3, 0.1)
    rng = np.random.default_rng(17)
    m1 = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=3, precision=mtp.MTP_FP32)
    stack = rng.standard_normal((3,) + tuple(m1.lattice_shape[1:]))
    singles = [_run(w, stack[r], 3) for r in range(3)]
    for launch in (0, 2):
        m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=3, precision=mtp.MTP_FP32, n_rhs=3)
        t = m.pitch(w.T, w.causality)
        t.set_variant(3)
        t.set_launch(launch)
        st = m.state_from_lattice(torch.tensor(stack, device=DEV))
        t.evolve(st)
        many = m.state_to_lattice(st).cpu().numpy()
        for r in range(3):
            assert np.array_equal(many[r], singles[r]), (launch, r, rel_l2(many[r], singles[r]))


def test_variants_refused_outside_fp32():
    w = S.cube_mode(2, 2, 0.1)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=2, precision=mtp.MTP_FP64)
    t = m.pitch(w.T)
    for v in (1, 2, 3, 4):
        with pytest.raises(mtp.MtpError) as ex:
            t.set_variant(v)
        assert ex.value.code == mtp.MTP_EUNSUPPORTED
    with pytest.raises(mtp.MtpError) as ex:
        t.set_variant(5)
    assert ex.value.code == mtp.MTP_EINVAL
