"""mtp_energy_noalloc: the energy reduction for callers that cannot allocate device memory
when they need the result (it keeps its scratch in a static device array).  Checked through
the C ABI against mtp_energy on the same states, on two calls in a row (the second call
reuses the scratch the first one left behind).  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import mtp_synth as S
import paper_1906_11029_gb300 as mtp

pytestmark = pytest.mark.gpu
TOL = {mtp.MTP_FP64: 1e-11, mtp.MTP_FP32: 1e-5, mtp.MTP_TF32: 1e-5, mtp.MTP_TF32X3: 1e-5, mtp.MTP_FP32_SPLIT: 1e-11}
CASES = [(2, mtp.MTP_FP64), (2, mtp.MTP_FP32), (3, mtp.MTP_FP64), (3, mtp.MTP_FP32), (3, mtp.MTP_TF32),
         (3, mtp.MTP_TF32X3), (3, mtp.MTP_FP32_SPLIT)]


@pytest.mark.parametrize("dim,precision", CASES)
def test_energy_noalloc_matches_energy(dim, precision):
    """Tensor-core meshes keep float states like FP32 ones and split meshes double states like
    FP64 ones, so each is reduced the same way as the corresponding plain mesh."""
    w = S.te_square(5, 3, 0.1) if dim == 2 else S.graded_sphere(n=3, p=3, T=0.05)
    n_rhs = 3
    m = mtp.Mesh(dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=precision, n_rhs=n_rhs)
    eps = torch.tensor(w.eps, dtype=torch.float64, device="cuda")
    mu = torch.tensor(w.mu, dtype=torch.float64, device="cuda")
    out = torch.full((n_rhs,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        vals = np.random.default_rng(10 * call + dim).standard_normal(m.lattice_shape)
        st = m.state_from_lattice(torch.tensor(vals, device="cuda"))
        ref = m.energy(st)                               # the existing entry point
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        mtp.mtp_energy_noalloc(st, eps, mu, dim, len(w.elems), w.p, precision, n_rhs, out)
        torch.cuda.synchronize()
        if call == 1:                                    # nothing allocated (and kept) by the call
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL[precision] * np.abs(ref)), (call, got, ref)


def test_energy_noalloc_rejects_too_many_rhs():
    w = S.te_square(2, 1, 0.1)
    m = mtp.Mesh(2, w.verts, w.elems, w.eps, w.mu, p=1, n_rhs=65)
    st = m.new_state()
    eps = torch.ones(len(w.elems), dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(mtp.MtpError) as ex:
        mtp.mtp_energy_noalloc(st, eps, eps, 2, len(w.elems), 1, mtp.MTP_FP64, 65, out)
    assert ex.value.code == mtp.MTP_EINVAL


def test_energy_noalloc_binding_checks_tensor_sizes():
    """The Python binding refuses tensors shorter than the call reads or of the wrong type
    before any pointer reaches the kernel."""
    w = S.te_square(2, 1, 0.1)
    m = mtp.Mesh(2, w.verts, w.elems, w.eps, w.mu, p=1, n_rhs=2)
    st = m.new_state()
    ne = len(w.elems)
    eps = torch.ones(ne, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    bad = [(st[:1], eps, eps, out), (st, eps[:-1], eps, out), (st, eps, eps.float(), out), (st, eps, eps, out[:1])]
    for a, b, c, d in bad:
        with pytest.raises(mtp.MtpError) as ex:
            mtp.mtp_energy_noalloc(a, b, c, 2, ne, 1, mtp.MTP_FP64, 2, d)
        assert ex.value.code == mtp.MTP_EINVAL
