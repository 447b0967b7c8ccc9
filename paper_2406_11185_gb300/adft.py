"""Thin Python binding of the C ABI in include/adft.h (argument marshalling only).

Every computation runs in the CUDA library ``lib/libadft.so``; PyTorch only
provides device memory and the current stream.  There is no CPU fallback: if
the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libadft.so")

ADFT_OK = 0
ADFT_ERR_ARG = -1
ADFT_ERR_UNSUPPORTED = -2
ADFT_ERR_ASYM_D = -3
ADFT_ERR_NONFINITE = -4
ADFT_ERR_OOM = -5
ADFT_ERR_CUDA = -6
ADFT_ERR_TIMEOUT = -7
ADFT_ERR_ABORTED = -8
ADFT_PREC_FP64 = 0
ADFT_PREC_MIXED = 1
ADFT_LMAX = 3
ADFT_MAX_NPRIM = 16
ADFT_STATIC_MAX_NBF = 16384

EXPORTED = [
    "adft_basis_create", "adft_basis_nbf", "adft_basis_dims", "adft_basis_schwarz", "adft_jk_build",
    "adft_jk_energy", "adft_jk_grad", "adft_jk_last_stats", "adft_jk_last_timings", "adft_basis_set_abort", "adft_jk_status",
    "adft_basis_destroy", "adft_batch_create", "adft_batch_offsets", "adft_batch_grad_offsets", "adft_batch_jk",
    "adft_batch_destroy", "adft_status_string", "adft_last_error_message", "adft_version", "adft_autotune",
    "adft_set_tuning", "adft_jk_plan", "adft_energy_static", "adft_batch_last_stats", "adft_batch_last_timings", "adft_batch_autotune",
    "adft_batch_set_tuning", "adft_alu_peak", "adft_jk_last_class_stats", "adft_one_electron", "adft_one_electron_grad",
]


class AdftError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {detail}".strip())


class adft_shell(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("l", ctypes.c_int), ("nprim", ctypes.c_int),
                ("exps", ctypes.POINTER(ctypes.c_double)), ("coefs", ctypes.POINTER(ctypes.c_double))]


class adft_opts(ctypes.Structure):
    _fields_ = [("thresh", ctypes.c_double), ("split", ctypes.c_double), ("precision", ctypes.c_int),
                ("check", ctypes.c_int), ("stream", ctypes.c_void_p), ("pair_mask", ctypes.c_void_p),
                ("omega", ctypes.c_double)]


class adft_stats(ctypes.Structure):
    _fields_ = [("quartets_fp64", ctypes.c_int64), ("quartets_fp32", ctypes.c_int64),
                ("quartets_total", ctypes.c_int64), ("prim_quartets_fp64", ctypes.c_int64),
                ("prim_quartets_fp32", ctypes.c_int64), ("flops_fp64", ctypes.c_double),
                ("flops_fp32", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libadft.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_2406_11185_gb300/build.py)")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.adft_basis_create.argtypes = [dp, ip, ctypes.POINTER(adft_shell), ip, ip, ctypes.POINTER(vp)]
    L.adft_basis_nbf.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.adft_basis_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int)] * 1 + [ctypes.POINTER(ctypes.c_int)] * 3
    L.adft_basis_schwarz.argtypes = [vp, dp]
    L.adft_jk_build.argtypes = [vp, vp, ctypes.POINTER(adft_opts), vp, vp]
    L.adft_jk_energy.argtypes = [vp, vp, ctypes.POINTER(adft_opts), vp, ip]
    L.adft_jk_grad.argtypes = [vp, vp, ctypes.POINTER(adft_opts), vp]
    L.adft_jk_last_stats.argtypes = [vp, ctypes.POINTER(adft_stats)]
    L.adft_jk_last_timings.argtypes = [vp, dp]
    L.adft_basis_set_abort.argtypes = [vp, ip]
    L.adft_jk_status.argtypes = [vp]
    L.adft_basis_destroy.argtypes = [vp]
    L.adft_basis_destroy.restype = None
    L.adft_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
    L.adft_batch_offsets.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.adft_batch_grad_offsets.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.adft_batch_jk.argtypes = [vp, vp, ctypes.POINTER(adft_opts), vp, vp, vp, vp]
    L.adft_batch_destroy.argtypes = [vp]
    L.adft_batch_destroy.restype = None
    L.adft_autotune.argtypes = [vp, vp, ctypes.POINTER(adft_opts), ctypes.POINTER(ctypes.c_int), dp]
    L.adft_set_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.adft_jk_plan.argtypes = [vp, vp, ctypes.POINTER(adft_opts), ctypes.POINTER(adft_stats),
                               ctypes.POINTER(ctypes.c_int64)]
    L.adft_batch_last_stats.argtypes = [vp, ctypes.POINTER(adft_stats)]
    L.adft_batch_last_timings.argtypes = [vp, dp]
    L.adft_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(adft_opts), ctypes.POINTER(ctypes.c_int), dp]
    L.adft_batch_set_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.adft_energy_static.argtypes = [vp, vp, vp, ip, vp, vp]
    L.adft_alu_peak.argtypes = [ip, ip, dp, dp]
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.adft_jk_last_class_stats.argtypes = [vp, i64p, i64p, i64p, dp]
    L.adft_one_electron.argtypes = [vp, dp, vp, vp, vp, vp]
    L.adft_one_electron_grad.argtypes = [vp, dp, vp, vp, vp, vp]
    L.adft_status_string.argtypes = [ip]
    L.adft_status_string.restype = ctypes.c_char_p
    L.adft_last_error_message.restype = ctypes.c_char_p
    L.adft_version.restype = ctypes.c_char_p
    _lib = L
    return L


def status_string(st: int) -> str:
    return load().adft_status_string(int(st)).decode()


def last_error() -> str:
    return load().adft_last_error_message().decode()


def _check(st: int, where: str):
    if st != ADFT_OK:
        raise AdftError(st, where, last_error())


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_opts(thresh=1e-12, split=1e-5, precision="fp64", check=True, stream=None, pair_mask=None,
              omega=0.0) -> adft_opts:
    """adft_opts; pair_mask: None or [2, 55] of 0/1 (band, class pair) owned by
    this call (the array is kept alive by the returned structure); omega > 0:
    the long-range operator erf(omega r)/r."""
    prec = {"fp64": ADFT_PREC_FP64, "mixed": ADFT_PREC_MIXED}[precision] if isinstance(precision, str) \
        else int(precision)
    o = adft_opts(float(thresh), float(split), prec, 1 if check else 0, _stream_ptr(stream), None, float(omega))
    if pair_mask is not None:
        m = np.ascontiguousarray(np.asarray(pair_mask, dtype=np.uint8).reshape(-1))
        if m.size != 2 * NCP:
            raise ValueError("pair_mask must hold 2 x 55 entries")
        o.pair_mask = m.ctypes.data
        o._mask = m
    return o


class Basis:
    """Owns one adft_basis handle (adft_basis_create / adft_basis_destroy)."""

    def __init__(self, atoms, shells, spherical=True):
        L = load()
        self._keep = []
        xyz = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64).reshape(-1, 3))
        arr = (adft_shell * len(shells))()
        for i, (atom, l, exps, coefs) in enumerate(shells):
            e = np.ascontiguousarray(exps, dtype=np.float64)
            c = np.ascontiguousarray(coefs, dtype=np.float64)
            self._keep += [e, c]
            arr[i] = adft_shell(int(atom), int(l), len(e), e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = ctypes.c_void_p()
        _check(L.adft_basis_create(xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), xyz.shape[0], arr,
                                   len(shells), 1 if spherical else 0, ctypes.byref(h)), "adft_basis_create")
        self.handle = h
        self.natom = xyz.shape[0]
        self.nshell = len(shells)
        n = ctypes.c_int()
        _check(L.adft_basis_nbf(h, ctypes.byref(n)), "adft_basis_nbf")
        self.nbf = n.value
        self._keep = None

    @classmethod
    def from_molecule(cls, mol):
        return cls(mol.atoms, mol.shells, mol.spherical)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().adft_basis_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def schwarz(self) -> np.ndarray:
        Q = np.zeros(self.nshell * (self.nshell + 1) // 2)
        _check(load().adft_basis_schwarz(self.handle, Q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "adft_basis_schwarz")
        return Q


def adft_basis_create(atoms, shells, spherical=True) -> Basis:
    return Basis(atoms, shells, spherical)


def _check_matrix(D, n):
    import torch
    if not (isinstance(D, torch.Tensor) and D.is_cuda and D.dtype == torch.float64 and D.is_contiguous()
            and tuple(D.shape) == (n, n)):
        raise ValueError(f"D must be a contiguous CUDA float64 tensor of shape ({n}, {n})")


def adft_jk_build(basis: Basis, D, thresh=1e-12, split=1e-5, precision="fp64", check=True, stream=None, out=None,
                  pair_mask=None, omega=0.0):
    """J, K (torch CUDA float64) of Eq. 1 for density D (partial sums over the
    class pairs of pair_mask, if given); omega > 0: J and K of the long-range
    operator erf(omega r)/r."""
    import torch
    _check_matrix(D, basis.nbf)
    J, K = out if out is not None else (torch.empty_like(D), torch.empty_like(D))
    o = make_opts(thresh, split, precision, check, stream, pair_mask, omega)
    _check(load().adft_jk_build(basis.handle, ctypes.c_void_p(D.data_ptr()), ctypes.byref(o),
                                ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(K.data_ptr())), "adft_jk_build")
    return J, K


def adft_jk_energy(basis: Basis, D, thresh=1e-12, split=1e-5, precision="fp64", check=True, stream=None,
                   on_device=False, pair_mask=None, omega=0.0):
    """E_JK = 1/2 tr(DJ) - 1/4 tr(DK); a float, or a 1-element CUDA tensor
    (a partial sum over the class pairs of pair_mask, if given); omega > 0:
    with J and K of erf(omega r)/r."""
    import torch
    _check_matrix(D, basis.nbf)
    o = make_opts(thresh, split, precision, check, stream, pair_mask, omega)
    if on_device:
        E = torch.empty(1, dtype=torch.float64, device=D.device)
        _check(load().adft_jk_energy(basis.handle, ctypes.c_void_p(D.data_ptr()), ctypes.byref(o),
                                     ctypes.c_void_p(E.data_ptr()), 1), "adft_jk_energy")
        return E
    e = ctypes.c_double()
    _check(load().adft_jk_energy(basis.handle, ctypes.c_void_p(D.data_ptr()), ctypes.byref(o),
                                 ctypes.cast(ctypes.byref(e), ctypes.c_void_p), 0), "adft_jk_energy")
    return e.value


def adft_jk_grad(basis: Basis, D, thresh=1e-12, split=1e-5, precision="fp64", check=True, stream=None,
                 pair_mask=None, omega=0.0):
    """dE_JK/dR [natom, 3] (torch CUDA float64) at fixed D (a partial sum over
    the class pairs of pair_mask, if given).  omega > 0 is not supported
    (ADFT_ERR_UNSUPPORTED)."""
    import torch
    _check_matrix(D, basis.nbf)
    g = torch.empty((basis.natom, 3), dtype=torch.float64, device=D.device)
    o = make_opts(thresh, split, precision, check, stream, pair_mask, omega)
    _check(load().adft_jk_grad(basis.handle, ctypes.c_void_p(D.data_ptr()), ctypes.byref(o),
                               ctypes.c_void_p(g.data_ptr())), "adft_jk_grad")
    return g


_JK_ENERGY_FN = None


def _jk_energy_function():
    """The torch.autograd.Function of jk_energy (created on first use, so that
    importing this module does not import torch)."""
    global _JK_ENERGY_FN
    if _JK_ENERGY_FN is not None:
        return _JK_ENERGY_FN
    import torch

    class JKEnergy(torch.autograd.Function):
        """E_JK(D, R) = 1/2 tr(DJ) - 1/4 tr(DK) as a function of the nuclear
        coordinates R.  Forward: adft_jk_energy on a basis built at R.
        Backward: grad_output times adft_jk_grad, the derivative integrals
        contracted with D (x) D on the GPU, recomputed rather than stored.
        D receives no gradient."""

        @staticmethod
        def forward(ctx, D, coords, shells, spherical, thresh, split, precision):
            xyz = coords.detach().to("cpu", torch.float64).numpy()
            basis = Basis(xyz, shells, spherical)
            E = adft_jk_energy(basis, D, thresh=thresh, split=split, precision=precision, check=False,
                               on_device=True)
            ctx.basis = basis
            ctx.opts = (thresh, split, precision)
            ctx.coords_meta = (coords.device, coords.dtype)
            ctx.save_for_backward(D)
            return E.reshape(())

        @staticmethod
        def backward(ctx, grad_E):
            (D,) = ctx.saved_tensors
            thresh, split, precision = ctx.opts
            g = adft_jk_grad(ctx.basis, D, thresh=thresh, split=split, precision=precision, check=False)
            device, dtype = ctx.coords_meta
            return None, (grad_E.to(g.device) * g).to(device, dtype), None, None, None, None, None

    _JK_ENERGY_FN = JKEnergy
    return JKEnergy


def jk_energy(D, coords, shells, spherical=True, thresh=1e-12, split=1e-5, precision="fp64"):
    """Differentiable E_JK (torch scalar on D's device) of density D (CUDA,
    float64, nbf x nbf) at nuclear coordinates coords (natom x 3, bohr; any
    device), basis shells [(atom, l, exps, coefs)].  E.backward() fills
    coords.grad with dE/dR from the GPU gradient kernels."""
    return _jk_energy_function().apply(D, coords, shells, spherical, thresh, split, precision)


def __getattr__(name):
    if name == "JKEnergy":
        return _jk_energy_function()
    raise AttributeError(name)


def adft_jk_last_stats(basis: Basis) -> dict:
    st = adft_stats()
    _check(load().adft_jk_last_stats(basis.handle, ctypes.byref(st)), "adft_jk_last_stats")
    return {k: getattr(st, k) for k, _ in adft_stats._fields_}


def adft_one_electron(basis: Basis, charges, stream=None, device=None):
    """Overlap S, kinetic T and nuclear attraction V (CUDA tensors [nbf, nbf])
    for nuclear charges `charges` (one per atom)."""
    import torch
    q = np.ascontiguousarray(np.asarray(charges, dtype=np.float64))
    if q.shape != (basis.natom,):
        raise ValueError(f"charges must hold {basis.natom} values")
    dev = torch.device("cuda") if device is None else device
    out = [torch.empty((basis.nbf, basis.nbf), dtype=torch.float64, device=dev) for _ in range(3)]
    vp = ctypes.c_void_p
    _check(load().adft_one_electron(basis.handle, q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    _stream_ptr(stream), *[vp(t.data_ptr()) for t in out]), "adft_one_electron")
    return tuple(out)


def adft_one_electron_grad(basis: Basis, charges, D, W, stream=None):
    """sum D dH/dR - sum W dS/dR [natom, 3] (CUDA float64) for the density D
    and the energy-weighted density W (CUDA [nbf, nbf] on the current device):
    the one-electron part of the closed-shell SCF nuclear gradient."""
    import torch
    q = np.ascontiguousarray(np.asarray(charges, dtype=np.float64))
    if q.shape != (basis.natom,):
        raise ValueError(f"charges must hold {basis.natom} values")
    _check_matrix(D, basis.nbf)
    _check_matrix(W, basis.nbf)
    g = torch.empty((basis.natom, 3), dtype=torch.float64, device=D.device)
    vp = ctypes.c_void_p
    _check(load().adft_one_electron_grad(basis.handle, q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         vp(D.data_ptr()), vp(W.data_ptr()), _stream_ptr(stream),
                                         vp(g.data_ptr())), "adft_one_electron_grad")
    return g


def adft_jk_last_class_stats(basis: Basis) -> dict:
    """Per (band, class pair) arrays [2, 55]: quartets, prim_quartets,
    bra_prims (int64) and flops (counted) of the last build."""
    out = {k: np.zeros(2 * NCP, dtype=np.int64) for k in ("quartets", "prim_quartets", "bra_prims")}
    fl = np.zeros(2 * NCP, dtype=np.float64)
    i64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(load().adft_jk_last_class_stats(basis.handle, i64(out["quartets"]), i64(out["prim_quartets"]),
                                           i64(out["bra_prims"]), fl.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "adft_jk_last_class_stats")
    res = {k: v.reshape(2, NCP) for k, v in out.items()}
    res["flops"] = fl.reshape(2, NCP)
    return res


def adft_jk_last_timings(basis: Basis) -> dict:
    """Device milliseconds of the phases of the last call (CUDA events)."""
    ms = (ctypes.c_double * 4)()
    _check(load().adft_jk_last_timings(basis.handle, ms), "adft_jk_last_timings")
    return {"setup_screen_ms": ms[0], "eri_fp64_ms": ms[1], "eri_fp32_ms": ms[2], "transform_ms": ms[3]}


def adft_basis_set_abort(basis: Basis, flag: bool):
    _check(load().adft_basis_set_abort(basis.handle, 1 if flag else 0), "adft_basis_set_abort")


def adft_jk_status(basis: Basis) -> int:
    return int(load().adft_jk_status(basis.handle))


NCP = 55  # class pairs up to f shells


def adft_autotune(basis: Basis, D, thresh=1e-12, split=1e-5, precision="mixed", stream=None,
                  return_times=False, omega=0.0):
    """Run the launch-shape autotuner on density D; returns the [2, 55] table
    (FP64 band, FP32 band) now installed in the handle, each entry
    blocks_per_SM + TUNE_VARIANT_STRIDE * kernel_variant (and the best kernel
    time of every class pair in ms with return_times)."""
    _check_matrix(D, basis.nbf)
    tab = (ctypes.c_int * (2 * NCP))()
    ms = (ctypes.c_double * (2 * NCP))()
    o = make_opts(thresh, split, precision, False, stream, omega=omega)
    _check(load().adft_autotune(basis.handle, ctypes.c_void_p(D.data_ptr()), ctypes.byref(o), tab, ms),
           "adft_autotune")
    t = np.array(tab[:], dtype=np.int32).reshape(2, NCP)
    return (t, np.array(ms[:]).reshape(2, NCP)) if return_times else t


def adft_jk_plan(basis: Basis, D, thresh=1e-12, split=1e-5, precision="mixed", stream=None):
    """Screening only: (stats dict, [2, 55] shell quartets per band and class pair)."""
    _check_matrix(D, basis.nbf)
    st = adft_stats()
    q = (ctypes.c_int64 * (2 * NCP))()
    o = make_opts(thresh, split, precision, False, stream)
    _check(load().adft_jk_plan(basis.handle, ctypes.c_void_p(D.data_ptr()), ctypes.byref(o), ctypes.byref(st), q),
           "adft_jk_plan")
    return {k: getattr(st, k) for k, _ in adft_stats._fields_}, np.array(q[:], dtype=np.int64).reshape(2, NCP)


TUNE_VARIANT_STRIDE = 256


def adft_set_tuning(basis: Basis, table) -> None:
    """Install a [2, 55] launch-shape table (adft_autotune's encoding)."""
    t = np.ascontiguousarray(np.asarray(table, dtype=np.int32).reshape(-1))
    if t.size != 2 * NCP:
        raise ValueError("table must hold 2 x 55 entries")
    _check(load().adft_set_tuning(basis.handle, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "adft_set_tuning")


class Batch:
    """Owns an adft_batch of several bases (adft_batch_create / destroy)."""

    def __init__(self, bases):
        L = load()
        self.bases = list(bases)
        arr = (ctypes.c_void_p * len(self.bases))(*[b.handle.value for b in self.bases])
        h = ctypes.c_void_p()
        _check(L.adft_batch_create(arr, len(self.bases), ctypes.byref(h)), "adft_batch_create")
        self.handle = h
        self.nmol = len(self.bases)
        off = (ctypes.c_int64 * (self.nmol + 1))()
        _check(L.adft_batch_offsets(h, off), "adft_batch_offsets")
        self.offsets = np.array(off[:], dtype=np.int64)
        goff = (ctypes.c_int64 * (self.nmol + 1))()
        _check(L.adft_batch_grad_offsets(h, goff), "adft_batch_grad_offsets")
        self.grad_offsets = np.array(goff[:], dtype=np.int64)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().adft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, mats):
        import torch
        return torch.cat([m.reshape(-1) for m in mats]).contiguous()

    def unpack(self, flat):
        out = []
        for i, b in enumerate(self.bases):
            out.append(flat[self.offsets[i]:self.offsets[i + 1]].reshape(b.nbf, b.nbf))
        return out


def adft_batch_jk(batch: Batch, D_packed, thresh=1e-10, split=1e-5, precision="mixed", check=False, stream=None,
                  energy=True, grad=False, out=None):
    """Packed J, K (and per-molecule E, packed gradient) of every molecule."""
    import torch
    if not (isinstance(D_packed, torch.Tensor) and D_packed.is_cuda and D_packed.dtype == torch.float64
            and D_packed.is_contiguous() and D_packed.numel() == int(batch.offsets[-1])):
        raise ValueError("D_packed must be a contiguous CUDA float64 tensor of the packed size")
    if out is None:
        J, K = torch.empty_like(D_packed), torch.empty_like(D_packed)
        E = torch.empty(batch.nmol, dtype=torch.float64, device=D_packed.device) if energy else None
        G = torch.empty(int(batch.grad_offsets[-1]), dtype=torch.float64, device=D_packed.device) if grad else None
    else:
        J, K, E, G = out
    o = make_opts(thresh, split, precision, check, stream)
    vp = ctypes.c_void_p
    _check(load().adft_batch_jk(batch.handle, vp(D_packed.data_ptr()), ctypes.byref(o), vp(J.data_ptr()),
                                vp(K.data_ptr()), vp(E.data_ptr()) if E is not None else None,
                                vp(G.data_ptr()) if G is not None else None), "adft_batch_jk")
    return J, K, E, G


def adft_batch_last_stats(batch: Batch) -> dict:
    st = adft_stats()
    _check(load().adft_batch_last_stats(batch.handle, ctypes.byref(st)), "adft_batch_last_stats")
    return {k: getattr(st, k) for k, _ in adft_stats._fields_}


def adft_batch_last_timings(batch: Batch) -> dict:
    ms = (ctypes.c_double * 4)()
    _check(load().adft_batch_last_timings(batch.handle, ms), "adft_batch_last_timings")
    return {"setup_screen_ms": ms[0], "eri_fp64_ms": ms[1], "eri_fp32_ms": ms[2], "transform_ms": ms[3]}


def adft_batch_autotune(batch: Batch, D_packed, thresh=1e-10, split=1e-5, precision="mixed",
                        stream=None) -> np.ndarray:
    tab = (ctypes.c_int * (2 * NCP))()
    o = make_opts(thresh, split, precision, False, stream)
    _check(load().adft_batch_autotune(batch.handle, ctypes.c_void_p(D_packed.data_ptr()), ctypes.byref(o), tab,
                                      None), "adft_batch_autotune")
    return np.array(tab[:], dtype=np.int32).reshape(2, NCP)


def adft_batch_set_tuning(batch: Batch, table) -> None:
    """Install a [2, 55] launch-shape table in a batch (adft_autotune's encoding)."""
    t = np.ascontiguousarray(np.asarray(table, dtype=np.int32).reshape(-1))
    if t.size != 2 * NCP:
        raise ValueError("table must hold 2 x 55 entries")
    _check(load().adft_batch_set_tuning(batch.handle, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
           "adft_batch_set_tuning")


def adft_alu_peak(fp64: bool, iters: int = 20000) -> dict:
    """Measured FMA peak of the current device: {"tflops", "ms"} (FP64 or FP32)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().adft_alu_peak(1 if fp64 else 0, int(iters), ctypes.byref(tf), ctypes.byref(ms)), "adft_alu_peak")
    return {"tflops": tf.value, "ms": ms.value}


def adft_energy_static(D, J, K, stream=None):
    """E = 1/2 tr(DJ) - 1/4 tr(DK) with no device allocation inside the call
    (scratch is a fixed array in the library); returns a 1-element CUDA
    tensor.  The output tensor is allocated here by PyTorch, before the call."""
    import torch
    n = D.shape[0]
    for M in (D, J, K):
        _check_matrix(M, n)
        if M.device != D.device:
            raise ValueError("D, J and K must be on the same CUDA device")
    if stream is not None and getattr(stream, "device", D.device) != D.device:
        raise ValueError("the stream must belong to D's device")
    with torch.cuda.device(D.device):
        E = torch.empty(1, dtype=torch.float64, device=D.device)
        vp = ctypes.c_void_p
        _check(load().adft_energy_static(vp(D.data_ptr()), vp(J.data_ptr()), vp(K.data_ptr()), n,
                                         vp(E.data_ptr()), _stream_ptr(stream)), "adft_energy_static")
    return E
