"""GB300 explicit Mapped Tent Pitching (MTP) + SAT time stepping for Maxwell.

Thin ctypes binding of the C ABI declared in ``include/mtp.h``: every function
here only marshals arguments (numpy arrays for host data, torch CUDA tensors for
device state, the current torch stream) and calls the library; all evolution
work runs in the library's CUDA kernels.  There is no CPU fallback: importing
without the built library raises.

Functions keep the ABI's names (``mtp_mesh_create``, ``mtp_pitch_tents``, ...);
``Mesh`` and ``Tents`` wrap the handles for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmtp.so")

MTP_OK, MTP_EINVAL, MTP_EMESH, MTP_ECAUSAL = 0, -1, -2, -3
MTP_ENOMEM, MTP_ECUDA, MTP_ETIMEOUT, MTP_ENUMERIC, MTP_EUNSUPPORTED = -4, -5, -6, -7, -8
MTP_FP64, MTP_FP32, MTP_TF32, MTP_TF32X3, MTP_FP32_SPLIT = 0, 1, 2, 3, 4
MTP_FLAG_LAYER_LAUNCHES, MTP_FLAG_TEST_STALL, MTP_FLAG_SUBSTITUTED_RK4 = 1, 2, 4
_CODES = {0: "MTP_OK", -1: "MTP_EINVAL", -2: "MTP_EMESH", -3: "MTP_ECAUSAL", -4: "MTP_ENOMEM",
          -5: "MTP_ECUDA", -6: "MTP_ETIMEOUT", -7: "MTP_ENUMERIC", -8: "MTP_EUNSUPPORTED"}

ABI_SYMBOLS = ["mtp_mesh_create", "mtp_mesh_destroy", "mtp_mesh_info", "mtp_pitch_tents", "mtp_pitch_tents_device",
               "mtp_tents_destroy", "mtp_tents_info", "mtp_tents_get", "mtp_state_from_lattice",
               "mtp_state_to_lattice", "mtp_evolve", "mtp_evolve_layers", "mtp_evolve_host",
               "mtp_tents_set_launch", "mtp_tents_set_variant", "mtp_tents_autotune", "mtp_batch_create", "mtp_batch_destroy", "mtp_batch_info", "mtp_batch_evolve",
               "mtp_adjoint", "mtp_energy", "mtp_energy_noalloc", "mtp_probe_rates", "mtp_last_error"]


class MtpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class mtp_options(C.Structure):
    _fields_ = [("p", C.c_int), ("q", C.c_int), ("m", C.c_int), ("precision", C.c_int),
                ("n_rhs", C.c_int), ("flags", C.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = C.CDLL(LIB_PATH)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "mtp_mesh_create": (C.c_int, [C.c_int, I64, P, I64, P, P, P, C.POINTER(mtp_options), C.POINTER(P)]),
        "mtp_mesh_destroy": (None, [P]),
        "mtp_mesh_info": (C.c_int, [P, P, P, P, P, P, P]),
        "mtp_pitch_tents": (C.c_int, [P, P, D, D, C.POINTER(P)]),
        "mtp_pitch_tents_device": (C.c_int, [P, P, D, D, C.POINTER(P), P]),
        "mtp_tents_destroy": (None, [P]),
        "mtp_tents_info": (C.c_int, [P, P, P, P]),
        "mtp_tents_get": (C.c_int, [P, P, P, P, P, P]),
        "mtp_state_from_lattice": (C.c_int, [P, P, P, P]),
        "mtp_state_to_lattice": (C.c_int, [P, P, P, P]),
        "mtp_evolve": (C.c_int, [P, P, D, P]),
        "mtp_evolve_layers": (C.c_int, [P, P, I64, I64, P]),
        "mtp_evolve_host": (C.c_int, [P, P, P, D, P]),
        "mtp_tents_set_launch": (C.c_int, [P, C.c_int]),
        "mtp_tents_set_variant": (C.c_int, [P, C.c_int]),
        "mtp_tents_autotune": (C.c_int, [P, P, I64, I64, P, P, P]),
        "mtp_batch_create": (C.c_int, [I64, P, C.POINTER(P)]),
        "mtp_batch_destroy": (None, [P]),
        "mtp_batch_info": (C.c_int, [P, P, P, P]),
        "mtp_batch_evolve": (C.c_int, [P, P, P]),
        "mtp_adjoint": (C.c_int, [P, P, P, P, P, P, I64, P]),
        "mtp_energy": (C.c_int, [P, P, P, P]),
        "mtp_energy_noalloc": (C.c_int, [P, P, P, C.c_int, I64, C.c_int, C.c_int, C.c_int, P, P]),
        "mtp_probe_rates": (C.c_int, [P, P]),
        "mtp_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(rc):
    if rc != MTP_OK:
        raise MtpError(rc, _lib.mtp_last_error().decode())


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _stream(stream=None):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


def library_path():
    return LIB_PATH


# ------------------------------------------------------------------------ raw ABI names
def mtp_mesh_create(dim, vertices, elements, eps, mu, p, precision=MTP_FP64, n_rhs=1, q=0, m=0, flags=0):
    v = np.ascontiguousarray(vertices, np.float64)
    e = np.ascontiguousarray(elements, np.int32)
    ep = np.ascontiguousarray(eps, np.float64)
    mu_ = np.ascontiguousarray(mu, np.float64)
    opts = mtp_options(p, q, m, precision, n_rhs, flags)
    h = C.c_void_p()
    _check(_lib.mtp_mesh_create(dim, len(v), _ptr(v), len(e), _ptr(e), _ptr(ep), _ptr(mu_),
                                C.byref(opts), C.byref(h)))
    return h


def mtp_mesh_destroy(h):
    _lib.mtp_mesh_destroy(h)


def mtp_mesh_info(h):
    dim, nf, nb, mp = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    ne, nv = C.c_int64(), C.c_int64()
    _check(_lib.mtp_mesh_info(h, C.byref(dim), C.byref(nf), C.byref(nb), C.byref(ne), C.byref(nv), C.byref(mp)))
    return {"dim": dim.value, "n_fields": nf.value, "n_basis": nb.value, "n_elems": ne.value,
            "n_verts": nv.value, "max_patch": mp.value}


def mtp_pitch_tents(mesh, T, causality_factor=0.5, wavespeed=None):
    ws = None if wavespeed is None else np.ascontiguousarray(wavespeed, np.float64)
    h = C.c_void_p()
    _check(_lib.mtp_pitch_tents(mesh, _ptr(ws), causality_factor, T, C.byref(h)))
    return h


def mtp_pitch_tents_device(mesh, T, causality_factor=0.5, wavespeed=None, stream=None):
    """Same tent list as mtp_pitch_tents, with the rounds on the current CUDA device."""
    ws = None if wavespeed is None else np.ascontiguousarray(wavespeed, np.float64)
    h = C.c_void_p()
    _check(_lib.mtp_pitch_tents_device(mesh, _ptr(ws), causality_factor, T, C.byref(h), _stream(stream)))
    return h


def mtp_tents_destroy(h):
    _lib.mtp_tents_destroy(h)


def mtp_tents_info(h):
    nt, nl, st = C.c_int64(), C.c_int64(), C.c_double()
    _check(_lib.mtp_tents_info(h, C.byref(nt), C.byref(nl), C.byref(st)))
    return {"n_tents": nt.value, "n_layers": nl.value, "spacetime_dofs": st.value}


def mtp_tents_get(h):
    info = mtp_tents_info(h)
    n, nl = info["n_tents"], info["n_layers"]
    v = np.empty(n, np.int32)
    tb = np.empty(n, np.float64)
    tt = np.empty(n, np.float64)
    lay = np.empty(n, np.int32)
    lp = np.empty(nl + 1, np.int64)
    _check(_lib.mtp_tents_get(h, _ptr(v), _ptr(tb), _ptr(tt), _ptr(lay), _ptr(lp)))
    return {"vertex": v, "t_bot": tb, "t_top": tt, "layer": lay, "layer_ptr": lp}


def mtp_state_from_lattice(mesh, vals_dev, state_dev, stream=None):
    _check(_lib.mtp_state_from_lattice(mesh, _ptr(vals_dev), _ptr(state_dev), _stream(stream)))


def mtp_state_to_lattice(mesh, state_dev, vals_dev, stream=None):
    _check(_lib.mtp_state_to_lattice(mesh, _ptr(state_dev), _ptr(vals_dev), _stream(stream)))


def mtp_evolve(tents, state_dev, T, stream=None):
    _check(_lib.mtp_evolve(tents, _ptr(state_dev), T, _stream(stream)))


def mtp_evolve_layers(tents, state_dev, layer_begin, layer_end, stream=None):
    _check(_lib.mtp_evolve_layers(tents, _ptr(state_dev), layer_begin, layer_end, _stream(stream)))


def mtp_evolve_host(tents, state_in, state_out, T, stream=None):
    _check(_lib.mtp_evolve_host(tents, _ptr(state_in), _ptr(state_out), T, _stream(stream)))


def mtp_tents_set_launch(h, launch):
    _check(_lib.mtp_tents_set_launch(h, launch))


def mtp_tents_set_variant(h, variant):
    _check(_lib.mtp_tents_set_variant(h, variant))


def mtp_tents_autotune(h, scratch_state, layer_begin, layer_end, stream=None):
    best = C.c_int()
    ms = np.zeros(3, np.float64)
    _check(_lib.mtp_tents_autotune(h, _ptr(scratch_state), layer_begin, layer_end, C.byref(best), _ptr(ms),
                                   _stream(stream)))
    return best.value, ms.tolist()


def mtp_batch_create(tents_handles):
    arr = (C.c_void_p * len(tents_handles))(*[t.value if isinstance(t, C.c_void_p) else t for t in tents_handles])
    h = C.c_void_p()
    _check(_lib.mtp_batch_create(len(tents_handles), arr, C.byref(h)))
    return h


def mtp_batch_destroy(h):
    _lib.mtp_batch_destroy(h)


def mtp_batch_info(h):
    ni, nt, st = C.c_int64(), C.c_int64(), C.c_double()
    _check(_lib.mtp_batch_info(h, C.byref(ni), C.byref(nt), C.byref(st)))
    return {"n_instances": ni.value, "n_tents": nt.value, "spacetime_dofs": st.value}


def mtp_batch_evolve(h, states, stream=None):
    arr = (C.c_void_p * len(states))(*[_ptr(s) for s in states])
    _check(_lib.mtp_batch_evolve(h, arr, _stream(stream)))


class Batch:
    """Owns an mtp_batch_t over several Tents (kept alive here)."""

    def __init__(self, tents_list):
        self.tents = list(tents_list)
        self.h = mtp_batch_create([t.h for t in self.tents])
        self.info = mtp_batch_info(self.h)

    def evolve(self, states, stream=None):
        mtp_batch_evolve(self.h, states, stream)

    def __del__(self):
        if getattr(self, "h", None):
            mtp_batch_destroy(self.h)
            self.h = None


def mtp_adjoint(tents, state0_dev, lam_T_dev, lam_0_dev, geps_dev, gmu_dev, checkpoint_every=0, stream=None):
    _check(_lib.mtp_adjoint(tents, _ptr(state0_dev), _ptr(lam_T_dev), _ptr(lam_0_dev), _ptr(geps_dev),
                            _ptr(gmu_dev), checkpoint_every, _stream(stream)))


def mtp_energy(mesh, state_dev, n_rhs=1, stream=None):
    out = np.zeros(n_rhs, np.float64)
    _check(_lib.mtp_energy(mesh, _ptr(state_dev), _ptr(out), _stream(stream)))
    return out


def mtp_energy_noalloc(state_dev, eps_dev, mu_dev, dim, n_elems, p, precision, n_rhs, out_dev, stream=None):
    """Energies into the caller's device buffer out_dev[n_rhs]; allocates nothing (see mtp.h).
    Torch tensors are checked against the sizes and types the call reads and writes before the
    pointers cross the ABI (a wrong size would make the kernel access memory out of bounds)."""
    _check_noalloc_args(state_dev, eps_dev, mu_dev, dim, n_elems, p, precision, n_rhs, out_dev)
    _check(_lib.mtp_energy_noalloc(_ptr(state_dev), _ptr(eps_dev), _ptr(mu_dev), dim, n_elems, p, precision,
                                   n_rhs, _ptr(out_dev), _stream(stream)))


def _check_noalloc_args(state, eps, mu, dim, n_elems, p, precision, n_rhs, out):
    import torch
    if dim not in (2, 3) or not 1 <= p <= 5 or n_elems < 1 or n_rhs < 1:
        return                                   # the library reports these itself
    nf = 3 if dim == 2 else 6
    nb = (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6
    want = torch.float64 if precision in (MTP_FP64, MTP_FP32_SPLIT) else torch.float32
    checks = [(state, want, n_rhs * n_elems * nf * nb, "state"), (eps, torch.float64, n_elems, "eps"),
              (mu, torch.float64, n_elems, "mu"), (out, torch.float64, n_rhs, "out")]
    for t, dtype, n, name in checks:
        if not isinstance(t, torch.Tensor):
            continue
        if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype or t.numel() < n:
            raise MtpError(MTP_EINVAL, f"mtp_energy_noalloc: {name} must be a contiguous CUDA {dtype} "
                                       f"tensor of at least {n} elements (got {t.dtype}, {t.numel()}, "
                                       f"cuda={t.is_cuda})")


def mtp_probe_rates(stream=None):
    """{"fp32_fma", "fp64_fma", "mma_tf32", "mma_bf16"} in TFLOP/s, measured on the current device."""
    out = np.zeros(4, np.float64)
    _check(_lib.mtp_probe_rates(_ptr(out), _stream(stream)))
    return dict(zip(["fp32_fma", "fp64_fma", "mma_tf32", "mma_bf16"], out.tolist()))


# ------------------------------------------------------------------------ convenience wrappers
class Mesh:
    """Owns an mtp_mesh_t.  Arrays are host (numpy) data; see include/mtp.h."""

    def __init__(self, dim, vertices, elements, eps, mu, p, precision=MTP_FP64, n_rhs=1, q=0, m=0, flags=0):
        self.h = mtp_mesh_create(dim, vertices, elements, eps, mu, p, precision, n_rhs, q, m, flags)
        self.info = mtp_mesh_info(self.h)
        self.p, self.precision, self.n_rhs = p, precision, n_rhs
        self.q = q or p + 1
        self.m = m or 2 * p

    @property
    def state_shape(self):
        i = self.info
        return (self.n_rhs, i["n_elems"], i["n_fields"], i["n_basis"])

    @property
    def lattice_shape(self):
        i = self.info
        return (self.n_rhs, i["n_elems"], i["n_basis"], i["n_fields"])

    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision in (MTP_FP64, MTP_FP32_SPLIT) else torch.float32

    def new_state(self, device="cuda"):
        import torch
        return torch.zeros(self.state_shape, dtype=self.torch_dtype(), device=device)

    def state_from_lattice(self, vals_dev, state_dev=None, stream=None):
        state_dev = self.new_state(vals_dev.device) if state_dev is None else state_dev
        mtp_state_from_lattice(self.h, vals_dev, state_dev, stream)
        return state_dev

    def state_to_lattice(self, state_dev, vals_dev=None, stream=None):
        import torch
        if vals_dev is None:
            vals_dev = torch.empty(self.lattice_shape, dtype=torch.float64, device=state_dev.device)
        mtp_state_to_lattice(self.h, state_dev, vals_dev, stream)
        return vals_dev

    def energy(self, state_dev, stream=None):
        return mtp_energy(self.h, state_dev, self.n_rhs, stream)

    def pitch(self, T, causality_factor=0.5, wavespeed=None, device=False):
        """Tents to time T; ``device=True`` runs the pitcher's rounds on the GPU (same list)."""
        return Tents(self, T, causality_factor, wavespeed, device)

    def __del__(self):
        if getattr(self, "h", None):
            mtp_mesh_destroy(self.h)
            self.h = None


class Tents:
    def __init__(self, mesh: Mesh, T, causality_factor=0.5, wavespeed=None, device=False):
        self.mesh = mesh                       # keeps the mesh alive
        self.T = T
        pitch = mtp_pitch_tents_device if device else mtp_pitch_tents
        self.h = pitch(mesh.h, T, causality_factor, wavespeed)
        self.info = mtp_tents_info(self.h)

    def get(self):
        return mtp_tents_get(self.h)

    def evolve(self, state_dev, stream=None):
        mtp_evolve(self.h, state_dev, self.T, stream)

    def evolve_layers(self, state_dev, layer_begin, layer_end, stream=None):
        mtp_evolve_layers(self.h, state_dev, layer_begin, layer_end, stream)

    def set_launch(self, launch):
        mtp_tents_set_launch(self.h, launch)

    def set_variant(self, variant):
        mtp_tents_set_variant(self.h, variant)

    def autotune(self, scratch_state, layer_begin, layer_end, stream=None):
        return mtp_tents_autotune(self.h, scratch_state, layer_begin, layer_end, stream)

    def evolve_host(self, state_in, state_out, stream=None):
        mtp_evolve_host(self.h, state_in, state_out, self.T, stream)

    def __del__(self):
        if getattr(self, "h", None):
            mtp_tents_destroy(self.h)
            self.h = None


def _torch_function():
    import torch

    class MtpEvolveFunction(torch.autograd.Function):
        """Y_T = evolve(Y_0) with gradients w.r.t. Y_0 and the per-element eps, mu of the tents'
        mesh, computed by the reverse sweep mtp_adjoint (tent-layer checkpointing with
        recomputation).  ``eps``/``mu`` must hold the mesh's values; they are inputs only so
        that autograd routes their gradients."""

        @staticmethod
        def forward(ctx, Y0, eps, mu, tents, checkpoint_every=0):
            YT = Y0.detach().clone().contiguous()
            tents.evolve(YT)
            ctx.save_for_backward(Y0.detach().contiguous())
            ctx.tents = tents
            ctx.k = checkpoint_every
            return YT

        @staticmethod
        def backward(ctx, gYT):
            (Y0,) = ctx.saved_tensors
            t = ctx.tents
            lam0 = torch.empty_like(Y0)
            ne = t.mesh.info["n_elems"]
            geps = torch.empty(ne, dtype=torch.float64, device=Y0.device)
            gmu = torch.empty(ne, dtype=torch.float64, device=Y0.device)
            mtp_adjoint(t.h, Y0, gYT.contiguous().to(Y0.dtype), lam0, geps, gmu, ctx.k)
            return lam0, geps, gmu, None, None

    return MtpEvolveFunction


def mtp_evolve_autograd(Y0, eps, mu, tents, checkpoint_every=0):
    """Differentiable evolve (see MtpEvolveFunction)."""
    return _torch_function().apply(Y0, eps, mu, tents, checkpoint_every)
