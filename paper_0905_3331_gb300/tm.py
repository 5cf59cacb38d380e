"""Python binding of the C ABI in include/tm.h (ctypes; argument marshalling only).

Every operation runs in the CUDA library libtmqcd.so built from csrc/ for sm_103a.
There is no fallback: if the library is missing or no GPU is present the calls
raise.  Buffers may be torch tensors (CUDA or CPU), numpy arrays or raw integer
addresses; streams default to torch's current CUDA stream.

Canonical arrays (complex128, order t, z, y, x, spin, colour):
  spinor (T, L, L, L, 4, 3)   gauge (T, L, L, L, 4, 3, 3)   half field (h, 4, 3), h = V / 2
Device half fields of a given precision are opaque byte buffers of
``half_field_bytes(prec)`` bytes each (layout documented in include/tm.h).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

F64, F32, F16, DF64 = 0, 1, 2, 3
LINK18, LINK12, LINK8 = 18, 12, 8
CG_FP64, CG_SQRT_EPS, CG_RELIABLE = 0, 1, 2
HOP_PIPELINED = 3  # hopping-kernel choice: one thread per site, software-pipelined loads
HOP_PAIRED = 5     # hopping-kernel choice: two sites per thread, packed FP32 pairs

STATUS = {0: "TM_OK", 1: "TM_ERR_ARG", 2: "TM_ERR_ODD_EXTENT", 3: "TM_ERR_NO_GAUGE",
          4: "TM_ERR_NOT_SU3", 5: "TM_ERR_NONFINITE", 6: "TM_ERR_CUDA",
          7: "TM_ERR_NOT_CONVERGED", 8: "TM_ERR_TIMEOUT", 9: "TM_ERR_OOM",
          10: "TM_ERR_UNSUPPORTED"}

_lib = None


class TMError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.status_name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.status_name}: {message}")


class CGParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mode", ctypes.c_int),
                ("sloppy_prec", ctypes.c_int), ("sloppy_link", ctypes.c_int),
                ("delta", ctypes.c_double), ("use_x0", ctypes.c_int), ("flavour", ctypes.c_int),
                ("update_prec", ctypes.c_int)]


class TmSystem(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_void_p), ("mu", ctypes.c_double), ("flavour", ctypes.c_int),
                ("x", ctypes.c_void_p), ("b", ctypes.c_void_p)]


class CGInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("schur_rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libtmqcd.so (it must have been built: ``paper_0905_3331_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is not built; run "
                           "paper_0905_3331_gb300.build.build() (or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "tm_lattice_create": ([I, I, D, D, ctypes.POINTER(P)], I),
        "tm_lattice_destroy": ([P], I),
        "tm_lattice_set_params": ([P, D, D], I),
        "tm_volume": ([P], S),
        "tm_half_field_bytes": ([P, I], S),
        "tm_set_hop_threads": ([P, I, I, I], I),
        "tm_get_hop_threads": ([P, I, I], I),
        "tm_set_gauge": ([P, P, P], I),
        "tm_pack_half": ([P, I, P, P, I, P], I),
        "tm_unpack_half": ([P, I, P, P, I, P], I),
        "tm_apply_D": ([P, P, P, I, I, I, P], I),
        "tm_apply_hopping_eo": ([P, I, P, P, I, I, I, P], I),
        "tm_apply_Mee_inv": ([P, P, P, I, I, I, P], I),
        "tm_solve_cg": ([P, P, P, I, ctypes.POINTER(CGParams), ctypes.POINTER(CGInfo), P], I),
        "tm_cg_params_default": ([ctypes.POINTER(CGParams)], None),
        "tm_solve_cg_batch": ([ctypes.POINTER(TmSystem), I, ctypes.POINTER(CGParams),
                               ctypes.POINTER(CGInfo), P], I),
        "tm_meson_contract": ([P, P, P, P], I),
        "tm_correlator": ([P, P, P, I, P, P], I),
        "tm_solve_bicgstab": ([P, P, P, I, ctypes.POINTER(CGParams), ctypes.POINTER(CGInfo), P], I),
        "tm_solve_mr": ([P, P, P, I, ctypes.POINTER(CGParams), ctypes.POINTER(CGInfo), P], I),
        "tm_apply_Dh": ([P, P, P, D, D, I, P], I),
        "tm_solve_doublet": ([P, P, P, D, D, ctypes.POINTER(CGParams), ctypes.POINTER(CGInfo), P], I),
        "tm_solve_normal": ([P, P, P, ctypes.POINTER(CGParams), ctypes.POINTER(CGInfo), P], I),
        "tm_chrono_guess": ([P, P, ctypes.POINTER(P), I, P, I, P], I),
        "tm_last_error": ([], ctypes.c_char_p),
        "tm_launch_count": ([], ctypes.c_ulonglong),
        "tm_reset_launch_count": ([], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    """Names of the ABI functions this binding binds (all must exist in the library)."""
    return ["tm_lattice_create", "tm_lattice_destroy", "tm_lattice_set_params", "tm_volume",
            "tm_half_field_bytes", "tm_set_hop_threads", "tm_get_hop_threads", "tm_set_gauge", "tm_pack_half", "tm_unpack_half", "tm_apply_D",
            "tm_apply_hopping_eo", "tm_apply_Mee_inv", "tm_solve_cg", "tm_solve_cg_batch",
            "tm_cg_params_default", "tm_meson_contract", "tm_correlator", "tm_solve_bicgstab", "tm_solve_mr", "tm_solve_normal", "tm_chrono_guess", "tm_apply_Dh",
            "tm_solve_doublet",
            "tm_last_error", "tm_launch_count", "tm_reset_launch_count"]


def _check(status: int, where: str):
    if status != 0:
        msg = load().tm_last_error()
        raise TMError(status, where, msg.decode() if msg else "")


def _addr(buf) -> int:
    """Address of a torch tensor, numpy array or integer address."""
    if buf is None:
        return 0
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _sync():
    """Wait for the device (after a call that wrote a host buffer on a stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            torch.cuda.synchronize()
    except ImportError:
        pass


def _stream(stream) -> int:
    if stream is not None:
        return int(stream if isinstance(stream, int) else stream.cuda_stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def launch_count() -> int:
    return int(load().tm_launch_count())


def reset_launch_count():
    load().tm_reset_launch_count()


@dataclass
class SolveInfo:
    iters: int
    reliable_updates: int
    true_rel_residual: float
    schur_rel_residual: float
    seconds: float
    status: int


class Lattice:
    """A T x L^3 lattice with hopping parameter kappa and bare twisted mass mu (mu~ = 2 kappa mu)."""

    def __init__(self, T: int, L: int, kappa: float, mu: float):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.tm_lattice_create(T, L, kappa, mu, ctypes.byref(h)), "tm_lattice_create")
        self._h = h
        self.T, self.L, self.kappa, self.mu = T, L, kappa, mu
        self.V = T * L ** 3
        self.h = self.V // 2

    def close(self):
        if getattr(self, "_h", None):
            load().tm_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, kappa: float, mu: float):
        _check(load().tm_lattice_set_params(self._h, kappa, mu), "tm_lattice_set_params")
        self.kappa, self.mu = kappa, mu

    def half_field_bytes(self, prec: int) -> int:
        return int(load().tm_half_field_bytes(self._h, prec))

    def set_hop_threads(self, prec: int, link: int, threads_per_site: int):
        """Fix the hopping kernel for one form: threads per site 1, 2 or 4, HOP_PIPELINED (3,
        one thread per site with software-pipelined loads) or HOP_PAIRED (5, two sites per thread
        with packed FP32 pairs) -- the last two for FP32 / FP16 storage; 0 re-tunes."""
        _check(load().tm_set_hop_threads(self._h, prec, link, threads_per_site),
               "tm_set_hop_threads")

    def hop_threads(self, prec: int, link: int) -> int:
        return int(load().tm_get_hop_threads(self._h, prec, link))

    def set_gauge(self, U, stream=None):
        _check(load().tm_set_gauge(self._h, _addr(U), _stream(stream)), "tm_set_gauge")

    def pack_half(self, prec: int, dst, src, nrhs: int = 1, stream=None):
        _check(load().tm_pack_half(self._h, prec, _addr(dst), _addr(src), nrhs, _stream(stream)),
               "tm_pack_half")

    def unpack_half(self, prec: int, dst, src, nrhs: int = 1, stream=None):
        _check(load().tm_unpack_half(self._h, prec, _addr(dst), _addr(src), nrhs, _stream(stream)),
               "tm_unpack_half")

    def apply_D(self, out, inp, flavour: int = 1, dagger: bool = False, nrhs: int = 1, stream=None):
        _check(load().tm_apply_D(self._h, _addr(out), _addr(inp), flavour, int(dagger), nrhs,
                                 _stream(stream)), "tm_apply_D")

    def apply_hopping_eo(self, out_parity: int, out, inp, prec: int = F64, link: int = LINK18,
                         nrhs: int = 1, stream=None):
        _check(load().tm_apply_hopping_eo(self._h, out_parity, _addr(out), _addr(inp), prec, link,
                                          nrhs, _stream(stream)), "tm_apply_hopping_eo")

    def apply_Mee_inv(self, out, inp, flavour: int = 1, prec: int = F64, nrhs: int = 1,
                      stream=None):
        _check(load().tm_apply_Mee_inv(self._h, _addr(out), _addr(inp), flavour, prec, nrhs,
                                       _stream(stream)), "tm_apply_Mee_inv")

    def meson_contract(self, props, out=None, stream=None):
        """Timeslice Gram matrices of a 12-column point-source propagator (tm_meson_contract).
        props: (12, T, L, L, L, 4, 3) complex128 (device or host).  Returns (T, 12, 12)."""
        if out is None:
            out = np.zeros((self.T, 12, 12), dtype=np.complex128)
        _check(load().tm_meson_contract(self._h, _addr(props), _addr(out), _stream(stream)),
               "tm_meson_contract")
        if isinstance(out, np.ndarray):
            _sync()
        return out

    def solve_cg(self, x, b, nrhs: int = 1, tol: float = 1e-10, max_iter: int = 100000,
                 mode: int = CG_FP64, sloppy_prec: int = F32, sloppy_link: int = LINK12,
                 delta: float = 0.1, use_x0: bool = False, flavour: int = 1,
                 update_prec: int = F64, stream=None, check: bool = True) -> SolveInfo:
        """tm_solve_cg: M(flavour) x = b to the relative residual tol (modes CG_FP64,
        CG_SQRT_EPS, CG_RELIABLE).  update_prec is the arithmetic of the residual recomputations
        inside the loop: F64, DF64, or F32 (FP32 recomputations relative to the last FP64 one,
        for FP16 storage); convergence is always confirmed in FP64."""
        p = CGParams(tol, max_iter, mode, sloppy_prec, sloppy_link, delta, int(use_x0), flavour,
                     update_prec)
        info = CGInfo()
        st = load().tm_solve_cg(self._h, _addr(x), _addr(b), nrhs, ctypes.byref(p),
                                ctypes.byref(info), _stream(stream))
        if check:
            _check(st, "tm_solve_cg")
        d = info.as_dict()
        d["status"] = st
        return SolveInfo(**d)

    def solve_bicgstab(self, x, b, nrhs: int = 1, tol: float = 1e-10, max_iter: int = 100000,
                       mode: int = CG_FP64, sloppy_prec: int = F32, sloppy_link: int = LINK12,
                       delta: float = 0.1, use_x0: bool = False, flavour: int = 1, stream=None,
                       check: bool = True) -> SolveInfo:
        """Solve M^f x = b with BiCGstab on the even/odd Schur system (iters = BiCGstab
        iterations, two Schur applications each)."""
        p = CGParams(tol, max_iter, mode, sloppy_prec, sloppy_link, delta, int(use_x0), flavour, F64)
        info = CGInfo()
        st = load().tm_solve_bicgstab(self._h, _addr(x), _addr(b), nrhs, ctypes.byref(p),
                                      ctypes.byref(info), _stream(stream))
        if check:
            _check(st, "tm_solve_bicgstab")
        d = info.as_dict()
        d["status"] = st
        return SolveInfo(**d)

    def apply_Dh(self, out, inp, mubar: float, epsbar: float, nrhs: int = 1, stream=None):
        """out = M_h inp for the non-degenerate doublet (fields (2, T, L, L, L, 4, 3) per rhs)."""
        _check(load().tm_apply_Dh(self._h, _addr(out), _addr(inp), mubar, epsbar, nrhs,
                                  _stream(stream)), "tm_apply_Dh")
        if isinstance(out, np.ndarray):
            _sync()
        return out

    def solve_doublet(self, x, b, mubar: float, epsbar: float, tol: float = 1e-10,
                      max_iter: int = 100000, mode: int = CG_FP64, sloppy_link: int = LINK12,
                      delta: float = 0.1, stream=None, check: bool = True) -> SolveInfo:
        """Solve M_h x = b for the doublet (even/odd CG; mode CG_FP64 or CG_RELIABLE with FP32
        sloppy storage)."""
        p = CGParams(tol, max_iter, mode, F32, sloppy_link, delta, 0, 1, F64)
        info = CGInfo()
        st = load().tm_solve_doublet(self._h, _addr(x), _addr(b), mubar, epsbar, ctypes.byref(p),
                                     ctypes.byref(info), _stream(stream))
        if check:
            _check(st, "tm_solve_doublet")
        d = info.as_dict()
        d["status"] = st
        return SolveInfo(**d)

    def solve_mr(self, x, b, nrhs: int = 1, tol: float = 1e-10, max_iter: int = 100000,
                 mode: int = CG_FP64, sloppy_link: int = LINK12, delta: float = 0.1,
                 use_x0: bool = False, flavour: int = 1, stream=None, check: bool = True) -> SolveInfo:
        """Solve M^f x = b with the minimal residual iteration on the even/odd Schur system
        (FP64, or FP32 sloppy storage with reliable updates)."""
        p = CGParams(tol, max_iter, mode, F32, sloppy_link, delta, int(use_x0), flavour, F64)
        info = CGInfo()
        st = load().tm_solve_mr(self._h, _addr(x), _addr(b), nrhs, ctypes.byref(p), ctypes.byref(info),
                                _stream(stream))
        if check:
            _check(st, "tm_solve_mr")
        d = info.as_dict()
        d["status"] = st
        return SolveInfo(**d)

    def solve_normal(self, X, phi, tol: float = 1e-10, max_iter: int = 100000,
                     mode: int = CG_FP64, sloppy_prec: int = F32, sloppy_link: int = LINK12,
                     delta: float = 0.1, use_x0: bool = False, flavour: int = 1,
                     update_prec: int = F64, stream=None, check: bool = True) -> SolveInfo:
        """Solve Qhat^f Qhat^-f X = phi (FP64 odd half fields on the device); with use_x0 the
        content of X is the initial guess."""
        p = CGParams(tol, max_iter, mode, sloppy_prec, sloppy_link, delta, int(use_x0), flavour,
                     update_prec)
        info = CGInfo()
        st = load().tm_solve_normal(self._h, _addr(X), _addr(phi), ctypes.byref(p),
                                    ctypes.byref(info), _stream(stream))
        if check:
            _check(st, "tm_solve_normal")
        d = info.as_dict()
        d["status"] = st
        return SolveInfo(**d)

    def chrono_guess(self, X0, chi, phi, flavour: int = 1, stream=None):
        """X0 = sum_i c_i chi_i with the c_i of the chronological guess (Galerkin condition on
        Qhat^f Qhat^-f); chi is a list of FP64 odd half fields on the device."""
        n = len(chi)
        arr = (ctypes.c_void_p * max(n, 1))(*[_addr(c) for c in chi])
        _check(load().tm_chrono_guess(self._h, _addr(X0), arr, n, _addr(phi), flavour,
                                      _stream(stream)), "tm_chrono_guess")


def solve_cg_batch(systems, tol: float = 1e-10, max_iter: int = 100000, sloppy_prec: int = F32,
                   sloppy_link: int = LINK12, delta: float = 0.1, stream=None, check: bool = True):
    """Solve many systems together.  `systems` is a list of (lattice, mu, x, b) or
    (lattice, mu, x, b, flavour) with x, b device buffers (canonical full fields).
    Returns one SolveInfo per system."""
    n = len(systems)
    arr = (TmSystem * n)()
    for k, sysk in enumerate(systems):
        lat, mu, x, b = sysk[:4]
        flavour = sysk[4] if len(sysk) > 4 else 1
        arr[k] = TmSystem(lat._h, mu, flavour, _addr(x), _addr(b))
    p = CGParams(tol, max_iter, CG_RELIABLE, sloppy_prec, sloppy_link, delta, 0, 1, F64)
    infos = (CGInfo * n)()
    st = load().tm_solve_cg_batch(arr, n, ctypes.byref(p), infos, _stream(stream))
    if check:
        _check(st, "tm_solve_cg_batch")
    out = []
    for k in range(n):
        d = infos[k].as_dict()
        out.append(SolveInfo(**d))
    return out


def correlator(lat, A, X, stream=None):
    """C(t) = tr[A_t (X (x) 1_colour)] for X = Gamma gamma5 (4 x 4, or a stack (n, 4, 4)) on
    source spin (tm_correlator); A from Lattice.meson_contract (host or device).  C_PP uses
    X = identity.  Returns (T,) or (n, T) complex128 (numpy for host A, else on A's device)."""
    if hasattr(X, "data_ptr"):  # a torch tensor (host or device)
        import torch
        Xa = X.contiguous()
        if Xa.dtype != torch.complex128:
            raise TypeError("X must be complex128")
        single = Xa.dim() == 2
        n = 1 if single else Xa.shape[0]
    else:
        Xa = np.ascontiguousarray(np.asarray(X, dtype=np.complex128))
        single = Xa.ndim == 2
        Xa = Xa.reshape(-1, 4, 4)
        n = Xa.shape[0]
    if isinstance(A, np.ndarray):
        A = np.ascontiguousarray(A, dtype=np.complex128)
        C = np.zeros((n, lat.T), dtype=np.complex128)
    else:
        import torch
        A = A.contiguous()
        C = torch.zeros((n, lat.T), dtype=torch.complex128, device=A.device)
    _check(load().tm_correlator(lat._h, _addr(A), _addr(Xa), n, _addr(C), _stream(stream)),
           "tm_correlator")
    if isinstance(C, np.ndarray):
        _sync()
    return C[0] if single else C
