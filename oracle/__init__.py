"""Plain FP64 CPU oracle for the Wilson twisted-mass operator and its even/odd CG.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the library under
``paper_0905_3331_gb300`` never imports it and it never imports that library.

The arithmetic lives in ``tm_oracle.c`` (C99 complex, FP64), written from the
paper's definitions: eq. eo0 for M, App. A for the gamma matrices, Sec. 2.4 for
the fermion boundary phases, eq. eo2-eo4 for the even/odd blocks, App. B.2 for
the two inversion steps and Sec. 4.4 for the stopping rule.  This module only
compiles it (gcc) and marshals numpy arrays.

Array conventions (canonical order t, z, y, x, spin, colour; Sec. 4.7.2):
  spinor field  complex128, shape (T, Lz, Ly, Lx, 4, 3)
  gauge field   complex128, shape (T, Lz, Ly, Lx, 4, 3, 3), direction mu = t, x, y, z
Half-lattice vectors are full-lattice arrays that are zero on the other parity.

Parity pins: every function here is pinned by the CPU tests in
tests/test_oracle_pins.py (closed forms, invariants, dense brute force and a
hand-derived worked example).  Agreement with the original tmLQCD program's own
outputs is "parity unpinned": no code or data of that program exist here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtm_oracle.so")
_lock = threading.Lock()
_lib = None

# Plain IEEE arithmetic on every host: no FMA contraction, textbook complex multiply.
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fcx-limited-range"]


def build(force: bool = False) -> str:
    """Compile tm_oracle.c into _build/libtm_oracle.so (gcc); returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_variant(src_text: str, path: str) -> str:
    """Compile C source text with the oracle's flags into `path` (for tests that plant a
    mistake in a copy of the oracle and check that the pins catch it)."""
    csrc = path[:-3] + ".c"
    with open(csrc, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", *CFLAGS, csrc, "-o", path, "-lm"], check=True)
    return path


def load_library(path: str):
    """Load and configure a compiled oracle library (the default one is loaded lazily)."""
    return _configure(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    """Set the ctypes signatures of every oracle entry point."""
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    L = ctypes.c_long
    lib.orc_gamma.argtypes = [I, P]
    lib.orc_hopping.argtypes = [P, P, I, P, P, P, I]
    lib.orc_apply_M.argtypes = [P, P, I, D, D, I, P, P, P]
    lib.orc_apply_M_sites.argtypes = [P, P, I, D, D, I, P, P, P, L, P]
    lib.orc_hopping_sites.argtypes = [P, P, I, P, P, P, L, P]
    lib.orc_apply_Mdiag.argtypes = [P, D, I, I, P, P]
    lib.orc_apply_Mdiag_inv.argtypes = [P, D, I, I, P, P]
    lib.orc_apply_Moff.argtypes = [P, P, I, D, P, I, P, P]
    lib.orc_schur.argtypes = [P, P, I, D, D, I, P, P, P, I]
    lib.orc_normal_op.argtypes = [P, P, I, D, D, I, P, P, P]
    lib.orc_cg.argtypes = [P, P, I, D, D, I, P, P, P, D, I,
                           ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.orc_cg.restype = I
    lib.orc_bicgstab.argtypes = [P, P, I, D, D, I, P, P, P, D, I,
                                 ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.orc_bicgstab.restype = I
    lib.orc_mr.argtypes = [P, P, I, D, D, I, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.orc_mr.restype = I
    lib.orc_eo_prepare.argtypes = [P, P, I, D, D, I, P, P, P]
    lib.orc_eo_reconstruct.argtypes = [P, P, I, D, D, I, P, P, P]
    lib.orc_solve.argtypes = [P, P, I, D, D, I, P, P, P, D, I, ctypes.POINTER(I),
                              ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.orc_solve.restype = I
    lib.orc_num_threads.restype = I
    lib.orc_pauli.argtypes = [I, P]
    lib.orc_apply_Mh.argtypes = [P, P, I, D, D, D, P, P, P]
    lib.orc_apply_Mh_dag.argtypes = [P, P, I, D, D, D, P, P, P]
    lib.orc_solve_Mh.argtypes = [P, P, I, D, D, D, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.orc_solve_Mh.restype = I
    return lib


# ------------------------------------------------------------------ helpers ---
@dataclass(frozen=True)
class Lattice:
    """Extents and boundary phases.  dims are in direction order (T, Lx, Ly, Lz)."""
    T: int
    Lx: int
    Ly: int
    Lz: int
    theta: tuple = (1.0, 0.0, 0.0, 0.0)  # antiperiodic in time (Sec. 2.4, theta = 1)
    spread: bool = False                  # phase on every hop (Sec. 4.1.2) instead

    @classmethod
    def cubic(cls, T: int, L: int, **kw) -> "Lattice":
        return cls(T, L, L, L, **kw)

    @property
    def V(self) -> int:
        return self.T * self.Lx * self.Ly * self.Lz

    @property
    def spinor_shape(self):
        return (self.T, self.Lz, self.Ly, self.Lx, 4, 3)

    @property
    def gauge_shape(self):
        return (self.T, self.Lz, self.Ly, self.Lx, 4, 3, 3)

    def _dims(self):
        return np.array([self.T, self.Lx, self.Ly, self.Lz], dtype=np.int32)

    def _theta(self):
        return np.array(self.theta, dtype=np.float64)

    def parity_mask(self) -> np.ndarray:
        """Boolean array (T, Lz, Ly, Lx): True on odd sites."""
        t, z, y, x = np.indices((self.T, self.Lz, self.Ly, self.Lx))
        return ((t + z + y + x) & 1).astype(bool)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a: np.ndarray, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def num_threads() -> int:
    """OpenMP threads used by the operator's site loops."""
    return int(_load().orc_num_threads())


def gamma(k: int) -> np.ndarray:
    """gamma_k (k = 0..3) or gamma_5 (k = 4) as typed from App. A."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().orc_gamma(k, _ptr(out))
    return out


# ---------------------------------------------------------------- operator ---
def hopping(lat: Lattice, U, psi, out_parity: int = -1) -> np.ndarray:
    """Pure hopping sum H (eq. eo0 bracket, no -kappa); out_parity 0/1 gives H_eo/H_oe."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_hopping(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), _ptr(U),
                        _ptr(psi), _ptr(out), int(out_parity))
    return out


def apply_M(lat: Lattice, U, psi, kappa: float, mu: float, f: int = 1) -> np.ndarray:
    """M psi of eq. eo0 on the full lattice (mu~ = 2 kappa mu, flavour sign f)."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_apply_M(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                        int(f), _ptr(U), _ptr(psi), _ptr(out))
    return out


def apply_M_sites(lat: Lattice, U, psi, kappa: float, mu: float, sites, f: int = 1):
    """(M psi) at the given lexicographic site indices: array (len(sites), 4, 3)."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, lat.spinor_shape)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    _load().orc_apply_M_sites(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa,
                              mu, int(f), _ptr(U), _ptr(psi), _ptr(sites), len(sites),
                              _ptr(out))
    return out


def hopping_sites(lat: Lattice, U, psi, sites) -> np.ndarray:
    """(H psi) at the given lexicographic site indices: array (len(sites), 4, 3)."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, lat.spinor_shape)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    _load().orc_hopping_sites(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), _ptr(U),
                              _ptr(psi), _ptr(sites), len(sites), _ptr(out))
    return out


def apply_Mdiag(lat: Lattice, psi, mut: float, f: int, parity: int) -> np.ndarray:
    """(1 + i f mu~ gamma5) psi on the sites of one parity (eq. eo2)."""
    psi = _c(psi, lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_apply_Mdiag(_ptr(lat._dims()), mut, int(f), int(parity), _ptr(psi), _ptr(out))
    return out


def apply_Mdiag_inv(lat: Lattice, psi, mut: float, f: int, parity: int) -> np.ndarray:
    """(1 - i f mu~ gamma5)/(1 + mu~^2) psi on the sites of one parity (eq. eo3)."""
    psi = _c(psi, lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_apply_Mdiag_inv(_ptr(lat._dims()), mut, int(f), int(parity), _ptr(psi),
                                _ptr(out))
    return out


def apply_Moff(lat: Lattice, U, psi, kappa: float, out_parity: int) -> np.ndarray:
    """M_eo (out_parity 0) or M_oe (out_parity 1) = -kappa H restricted (eq. eo2)."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_apply_Moff(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa,
                           _ptr(U), int(out_parity), _ptr(psi), _ptr(out))
    return out


def schur(lat: Lattice, U, v, kappa: float, mu: float, f: int = 1, gamma5: bool = False):
    """Mhat^f v (or Qhat^f v = gamma5 Mhat^f v) on odd sites, eq. eo2/eo4."""
    U = _c(U, lat.gauge_shape)
    v = _c(v, lat.spinor_shape)
    out = np.empty_like(v)
    _load().orc_schur(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                      int(f), _ptr(U), _ptr(v), _ptr(out), int(gamma5))
    return out


def normal_op(lat: Lattice, U, v, kappa: float, mu: float, f: int = 1) -> np.ndarray:
    """Qhat^f Qhat^-f v on odd sites (eq. eo6)."""
    U = _c(U, lat.gauge_shape)
    v = _c(v, lat.spinor_shape)
    out = np.empty_like(v)
    _load().orc_normal_op(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                          int(f), _ptr(U), _ptr(v), _ptr(out))
    return out


@dataclass
class CGResult:
    x: np.ndarray
    converged: bool
    iters: int
    relres: float


def cg(lat: Lattice, U, b, kappa: float, mu: float, f: int = 1, tol: float = 1e-10,
       max_iter: int = 10000, x0=None) -> CGResult:
    """CG on Qhat^f Qhat^-f X = b (odd-site vectors), relative stop ||r||/||b|| < tol."""
    U = _c(U, lat.gauge_shape)
    b = _c(b, lat.spinor_shape)
    x = np.zeros_like(b) if x0 is None else _c(x0, lat.spinor_shape).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = _load().orc_cg(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                        int(f), _ptr(U), _ptr(b), _ptr(x), tol, int(max_iter),
                        ctypes.byref(it), ctypes.byref(rr))
    return CGResult(x, st == 0, it.value, rr.value)


def bicgstab(lat: Lattice, U, b, kappa: float, mu: float, f: int = 1, tol: float = 1e-10,
             max_iter: int = 10000, x0=None) -> CGResult:
    """BiCGstab on the Schur operator Mhat^f X = b (odd-site vectors, eq. eo4; Sec. 4.4),
    relative stop ||r||/||b|| < tol confirmed on the recomputed residual.  iters counts
    BiCGstab iterations (two applications of Mhat each)."""
    U = _c(U, lat.gauge_shape)
    b = _c(b, lat.spinor_shape)
    x = np.zeros_like(b) if x0 is None else _c(x0, lat.spinor_shape).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = _load().orc_bicgstab(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                              int(f), _ptr(U), _ptr(b), _ptr(x), tol, int(max_iter),
                              ctypes.byref(it), ctypes.byref(rr))
    return CGResult(x, st == 0, it.value, rr.value)


def mr(lat: Lattice, U, b, kappa: float, mu: float, f: int = 1, tol: float = 1e-10,
       max_iter: int = 10000, x0=None) -> CGResult:
    """Minimal residual iteration on Mhat^f X = b (odd-site vectors, eq. eo4; Sec. 4.4)."""
    U = _c(U, lat.gauge_shape)
    b = _c(b, lat.spinor_shape)
    x = np.zeros_like(b) if x0 is None else _c(x0, lat.spinor_shape).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = _load().orc_mr(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu, int(f),
                        _ptr(U), _ptr(b), _ptr(x), tol, int(max_iter), ctypes.byref(it),
                        ctypes.byref(rr))
    return CGResult(x, st == 0, it.value, rr.value)


def eo_prepare(lat: Lattice, U, phi, kappa: float, mu: float, f: int = 1) -> np.ndarray:
    """varphi_e = (M_ee)^-1 phi_e, varphi_o = phi_o - M_oe varphi_e (App. B.2)."""
    U = _c(U, lat.gauge_shape)
    phi = _c(phi, lat.spinor_shape)
    out = np.empty_like(phi)
    _load().orc_eo_prepare(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                           int(f), _ptr(U), _ptr(phi), _ptr(out))
    return out


def eo_reconstruct(lat: Lattice, U, varphi, psi_o, kappa: float, mu: float,
                   f: int = 1) -> np.ndarray:
    """psi_e = varphi_e - (M_ee)^-1 M_eo psi_o (App. B.2); returns psi with both parities."""
    U = _c(U, lat.gauge_shape)
    varphi = _c(varphi, lat.spinor_shape)
    psi = _c(psi_o, lat.spinor_shape).copy()
    _load().orc_eo_reconstruct(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa,
                               mu, int(f), _ptr(U), _ptr(varphi), _ptr(psi))
    return psi


@dataclass
class SolveResult:
    psi: np.ndarray
    converged: bool
    iters: int
    relres_normal: float
    relres_full: float


def solve(lat: Lattice, U, phi, kappa: float, mu: float, f: int = 1, tol: float = 1e-10,
          max_iter: int = 10000) -> SolveResult:
    """M^f psi = phi by even/odd preconditioning + CG (App. B.2, eq. eo6)."""
    U = _c(U, lat.gauge_shape)
    phi = _c(phi, lat.spinor_shape)
    psi = np.zeros_like(phi)
    it = ctypes.c_int(0)
    rn = ctypes.c_double(0)
    rf = ctypes.c_double(0)
    st = _load().orc_solve(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mu,
                           int(f), _ptr(U), _ptr(phi), _ptr(psi), tol, int(max_iter),
                           ctypes.byref(it), ctypes.byref(rn), ctypes.byref(rf))
    return SolveResult(psi, st == 0, it.value, rn.value, rf.value)


def solve_bicgstab(lat: Lattice, U, phi, kappa: float, mu: float, f: int = 1,
                   tol: float = 1e-10, max_iter: int = 10000) -> SolveResult:
    """M^f psi = phi by even/odd preconditioning (App. B.2) with BiCGstab on the Schur system
    Mhat^f psi_o = varphi_o (eq. eo4) instead of CG on the normal equations."""
    U = _c(U, lat.gauge_shape)
    phi = _c(phi, lat.spinor_shape)
    varphi = eo_prepare(lat, U, phi, kappa, mu, f)
    odd = lat.parity_mask()[..., None, None]
    b = np.where(odd, varphi, 0)
    res = bicgstab(lat, U, b, kappa, mu, f, tol, max_iter)
    psi = eo_reconstruct(lat, U, varphi, res.x, kappa, mu, f)
    full = np.linalg.norm(phi - apply_M(lat, U, psi, kappa, mu, f)) / np.linalg.norm(phi)
    return SolveResult(psi, res.converged, res.iters, res.relres, full)


def solve_mr(lat: Lattice, U, phi, kappa: float, mu: float, f: int = 1, tol: float = 1e-10,
             max_iter: int = 10000) -> SolveResult:
    """M^f psi = phi by even/odd preconditioning (App. B.2) with MR on Mhat^f psi_o = varphi_o."""
    U = _c(U, lat.gauge_shape)
    phi = _c(phi, lat.spinor_shape)
    varphi = eo_prepare(lat, U, phi, kappa, mu, f)
    b = np.where(lat.parity_mask()[..., None, None], varphi, 0)
    res = mr(lat, U, b, kappa, mu, f, tol, max_iter)
    psi = eo_reconstruct(lat, U, varphi, res.x, kappa, mu, f)
    full = np.linalg.norm(phi - apply_M(lat, U, psi, kappa, mu, f)) / np.linalg.norm(phi)
    return SolveResult(psi, res.converged, res.iters, res.relres, full)


# ------------------------------------------------------------- contractions ---
def meson_contract(props) -> np.ndarray:
    """Timeslice sums of the Gram matrix of a 12-column point-source propagator:
    A[t][j][k] = sum_{x, x_t = t} <psi_j(x), psi_k(x)> (conjugate on psi_j), the building
    block of the correlators C_PG(t) = sum_x tr[G^dag G Gamma gamma5] of Sec. 4.3.
    props: (12, T, L, L, L, 4, 3).  Plain numpy definition."""
    P = np.asarray(props, dtype=np.complex128)
    return np.einsum("jtzyxsc,ktzyxsc->tjk", P.conj(), P)


def correlator(A, G) -> np.ndarray:
    """C(t) = tr[A_t (G (x) 1_colour)] with G = Gamma gamma5 acting on source spin."""
    A = np.asarray(A)
    T = A.shape[0]
    big = np.kron(np.asarray(G, dtype=np.complex128), np.eye(3))
    return np.array([np.trace(A[t] @ big) for t in range(T)])


# ------------------------------------------------------- chronological guess ---
def chrono_guess(lat: Lattice, U, chis, phi, kappa: float, mu: float, f: int = 1):
    """Chronological solver guess (Sec. 4.2, eq. chrono) for A X = phi, A = Qhat^f Qhat^-f
    (eq. eo6): the coefficients c solve sum_i <chi_j, A chi_i> c_i = <chi_j, phi> and the
    guess is X0 = sum_i c_i chi_i.  chis: list of odd-site vectors.  Returns (X0, c).
    Plain numpy: the matrix by its definition, numpy.linalg.solve for the n x n system."""
    phi = _c(phi, lat.spinor_shape)
    n = len(chis)
    if n == 0:
        return np.zeros_like(phi), np.zeros(0, dtype=np.complex128)
    chis = [_c(c, lat.spinor_shape) for c in chis]
    Achi = [normal_op(lat, U, chi, kappa, mu, f) for chi in chis]
    G = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        for i in range(n):
            G[j, i] = np.vdot(chis[j], Achi[i])
    rhs = np.array([np.vdot(chis[j], phi) for j in range(n)])
    c = np.linalg.solve(G, rhs)
    X0 = np.zeros_like(phi)
    for i in range(n):
        X0 += c[i] * chis[i]
    return X0, c


# ------------------------------------------------------ non-degenerate doublet ---
def pauli(k: int) -> np.ndarray:
    """tau_k (k = 1, 2, 3; 0 is the flavour identity) as typed from App. A."""
    out = np.zeros((2, 2), dtype=np.complex128)
    _load().orc_pauli(int(k), _ptr(out))
    return out


def apply_Mh(lat: Lattice, U, psi, kappa: float, mubar: float, epsbar: float) -> np.ndarray:
    """M_h psi for the doublet of eq. Dh, hopping-parameter form (psi: (2,) + spinor shape)."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, (2,) + lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_apply_Mh(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mubar, epsbar,
                         _ptr(U), _ptr(psi), _ptr(out))
    return out


def apply_Mh_dag(lat: Lattice, U, psi, kappa: float, mubar: float, epsbar: float) -> np.ndarray:
    """M_h^dag psi = tau1 gamma5 M_h gamma5 tau1 psi."""
    U = _c(U, lat.gauge_shape)
    psi = _c(psi, (2,) + lat.spinor_shape)
    out = np.empty_like(psi)
    _load().orc_apply_Mh_dag(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mubar,
                             epsbar, _ptr(U), _ptr(psi), _ptr(out))
    return out


def solve_Mh(lat: Lattice, U, phi, kappa: float, mubar: float, epsbar: float, tol: float = 1e-10,
             max_iter: int = 20000) -> CGResult:
    """M_h psi = phi on the full lattice by CG on the normal equations (CGNR)."""
    U = _c(U, lat.gauge_shape)
    phi = _c(phi, (2,) + lat.spinor_shape)
    psi = np.zeros_like(phi)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = _load().orc_solve_Mh(_ptr(lat._dims()), _ptr(lat._theta()), int(lat.spread), kappa, mubar,
                              epsbar, _ptr(U), _ptr(phi), _ptr(psi), tol, int(max_iter),
                              ctypes.byref(it), ctypes.byref(rr))
    return CGResult(psi, st == 0, it.value, rr.value)
