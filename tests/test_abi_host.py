"""C-ABI library on the host (no GPU): exported symbols, argument checking, and the
host tent pitcher against the oracle's pitcher, bit for bit (Sec. 2)."""
import ctypes
import os
import re

import numpy as np
import pytest

import mtp_synth as S
import paper_1906_11029_gb300 as mtp
from oracle.pitch import pitch_tents

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "mtp.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(mtp_\w+)\s*\(", header, re.M))
    assert declared, "no declarations parsed"
    lib = ctypes.CDLL(mtp.library_path())
    missing = [s for s in sorted(declared) if not hasattr(lib, s)]
    assert not missing, missing
    assert declared == set(mtp.ABI_SYMBOLS)


def test_mesh_errors():
    v, e = S.square_mesh(2)
    one = np.ones(len(e))
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, e, one, one, p=6)
    assert ex.value.code == mtp.MTP_EUNSUPPORTED
    bad = e.copy()
    bad[0] = [0, 1, 2]                           # collinear vertices (0,0), (.5,0), (1,0)
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, bad, one, one, p=2)
    assert ex.value.code == mtp.MTP_EMESH
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, e, -one, one, p=2)
    assert ex.value.code == mtp.MTP_EINVAL
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, np.vstack([e, e[:1]]), np.ones(len(e) + 1), np.ones(len(e) + 1), p=2)
    assert ex.value.code == mtp.MTP_EMESH       # a facet shared by three elements
    m = mtp.Mesh(2, v, e, one, one, p=2)
    with pytest.raises(mtp.MtpError) as ex:
        m.pitch(0.5, causality_factor=1.5)
    assert ex.value.code == mtp.MTP_EINVAL
    for T, cf in ((0.5, 1.5), (-1.0, 0.5), (float("inf"), 0.5)):   # checked before any device work
        with pytest.raises(mtp.MtpError) as ex:
            m.pitch(T, causality_factor=cf, device=True)
        assert ex.value.code == mtp.MTP_EINVAL
    with pytest.raises(mtp.MtpError) as ex:
        m.pitch(0.5, wavespeed=np.zeros(len(e)), device=True)
    assert ex.value.code == mtp.MTP_EINVAL


def test_mesh_info():
    w = S.cube_mode(3, 3, 0.1)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=3)
    assert m.info == {"dim": 3, "n_fields": 6, "n_basis": 20, "n_elems": 162, "n_verts": 64, "max_patch": 24}


def _compare(w, cf=0.5, wavespeed=None):
    ref = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, cf, wavespeed)
    m = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=1)
    t = m.pitch(w.T, cf, wavespeed)
    got = t.get()
    for k in ("vertex", "layer", "layer_ptr"):
        assert np.array_equal(got[k], ref[k]), k
    for k in ("t_bot", "t_top"):
        assert np.array_equal(got[k].view(np.uint64), ref[k].view(np.uint64)), k   # bit-exact
    return got


@pytest.mark.parametrize("make", [
    lambda: S.te_square(8, 2, 0.5),                               # 2D TE cavity, 128 triangles
    lambda: S.Workload("sq_pert", 2, S.perturb_interior(*[S.square_mesh(6)[0]], 1 / 6, 0.2, 3),
                       S.square_mesh(6)[1], np.ones(72), np.ones(72), 1, 0.3),
    lambda: S.cube_mode(6, 1, 0.3),                               # perturbed Kuhn cube
    lambda: S.graded_sphere(n=6, p=1, T=0.2),                     # graded + eps jump
    lambda: S.adjoint_cube(n=4, p=1, T=0.3),                      # random eps per element
])
def test_pitcher_bit_exact_against_oracle(make):
    _compare(make())


def test_pitcher_bit_exact_with_wavespeed():
    w = S.adjoint_cube(n=3, p=1, T=0.2)
    _compare(w, cf=0.4, wavespeed=np.ones(len(w.elems)))


@pytest.mark.slow
def test_pitcher_bit_exact_cube16():
    _compare(S.cube_mode(16, 3, 1.0))


def test_patch_larger_than_build_limit_is_rejected():
    # a 2D fan of 20 triangles around one vertex: patch 20 > the 2D limit (16)
    k = 20
    ang = np.linspace(0, 2 * np.pi, k, endpoint=False)
    v = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], 1)])
    e = np.array([[0, 1 + i, 1 + (i + 1) % k] for i in range(k)], np.int32)
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, e, np.ones(k), np.ones(k), p=2)
    assert ex.value.code == mtp.MTP_EUNSUPPORTED


def test_tensor_core_precision_is_3d_only():
    v, e = S.square_mesh(2)
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, e, np.ones(len(e)), np.ones(len(e)), p=2, precision=mtp.MTP_TF32)
    assert ex.value.code == mtp.MTP_EUNSUPPORTED


def test_split_precision_accepted_any_dim_and_state_is_double():
    for dim, (v, e) in ((2, S.square_mesh(2)), (3, S.cube_mesh(1))):
        m = mtp.Mesh(dim, v, e, np.ones(len(e)), np.ones(len(e)), p=5, precision=mtp.MTP_FP32_SPLIT)
        import torch
        assert m.torch_dtype() == torch.float64
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(2, v, e, np.ones(len(e)), np.ones(len(e)), p=2, precision=mtp.MTP_FP32_SPLIT + 1)
    assert ex.value.code == mtp.MTP_EINVAL


@pytest.mark.parametrize("dim", [2, 3])
def test_reference_tables_build_for_every_degree(dim):
    """Mesh creation builds the reference tables; it fails if either basis is not in
    ascending degree order or if an entry that the degree structure makes zero is more than
    rounding residue (the tent kernels skip those blocks)."""
    v, e = S.square_mesh(2) if dim == 2 else S.cube_mesh(2)
    one = np.ones(len(e))
    for p in range(1, 6):
        m = mtp.Mesh(dim, v, e, one, one, p=p)
        nb = (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6
        assert m.info["n_basis"] == nb


def test_kernel_variant_and_rk4_flag_validation():
    """Host-side checks of mtp_tents_set_variant and MTP_FLAG_SUBSTITUTED_RK4 (no GPU needed)."""
    v, e = S.cube_mesh(1)
    one = np.ones(len(e))
    t32 = mtp.Mesh(3, v, e, one, one, p=2, precision=mtp.MTP_FP32).pitch(0.1)
    for variant in (0, 1, 2, 3, 4, 0):
        t32.set_variant(variant)
    for bad in (-1, 5):
        with pytest.raises(mtp.MtpError) as ex:
            t32.set_variant(bad)
        assert ex.value.code == mtp.MTP_EINVAL
    # the tcgen05 variants are built for 3D, p = 2..4
    vs, es = S.square_mesh(2)
    cases = [(2, vs, es, 2), (3, v, e, 1), (3, v, e, 5)]
    for dim, vv, ee, p in cases:
        t = mtp.Mesh(dim, vv, ee, np.ones(len(ee)), np.ones(len(ee)), p=p, precision=mtp.MTP_FP32).pitch(0.1)
        t.set_variant(2)
        for tcv in (3, 4):
            with pytest.raises(mtp.MtpError) as ex:
                t.set_variant(tcv)
            assert ex.value.code == mtp.MTP_EUNSUPPORTED, (dim, p, tcv)
    for prec in (mtp.MTP_FP64, mtp.MTP_FP32_SPLIT, mtp.MTP_TF32):
        t = mtp.Mesh(3, v, e, one, one, p=2, precision=prec).pitch(0.1)
        t.set_variant(0)
        with pytest.raises(mtp.MtpError) as ex:
            t.set_variant(1)
        assert ex.value.code == mtp.MTP_EUNSUPPORTED
    # the substituted-RK4 control is built in FP64 only, and only the SAT kernels take variants
    rk = mtp.Mesh(3, v, e, one, one, p=2, precision=mtp.MTP_FP64, flags=mtp.MTP_FLAG_SUBSTITUTED_RK4)
    with pytest.raises(mtp.MtpError) as ex:
        rk.pitch(0.1).set_variant(2)
    assert ex.value.code == mtp.MTP_EUNSUPPORTED
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(3, v, e, one, one, p=2, precision=mtp.MTP_FP32, flags=mtp.MTP_FLAG_SUBSTITUTED_RK4)
    assert ex.value.code == mtp.MTP_EUNSUPPORTED
    with pytest.raises(mtp.MtpError) as ex:
        mtp.Mesh(3, v, e, one, one, p=2, flags=8)
    assert ex.value.code == mtp.MTP_EINVAL


def test_tuner_cache_key_separates_workload_shapes():
    from paper_1906_11029_gb300 import tune
    a = tune._key(3, 4, "fp32", 24, 196608, 892.0)
    assert a != tune._key(3, 4, "fp32", 24, 3072, 892.0)          # element count
    assert a != tune._key(3, 4, "fp32", 24, 196608, 40.0)         # tents-per-layer bucket
    assert a == tune._key(3, 4, "fp32", 24, 196608, 900.0)        # same power-of-two bucket
    assert {c for c in tune.candidates(3, 4, "fp32")} == {
        (mtp.MTP_FP32, 0), (mtp.MTP_FP32, 1), (mtp.MTP_FP32, 2), (mtp.MTP_FP32, 3), (mtp.MTP_FP32, 4),
        (mtp.MTP_TF32X3, 0)}
    assert (mtp.MTP_FP32, 3) not in tune.candidates(3, 5, "fp32")
    assert (mtp.MTP_TF32, 0) in tune.candidates(3, 4, "tf32")
    assert all(c[0] == mtp.MTP_FP32 for c in tune.candidates(2, 3, "fp32"))
