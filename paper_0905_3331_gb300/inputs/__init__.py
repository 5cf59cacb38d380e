"""Seeded synthetic inputs: random SU(3) gauge fields and spinor sources.

This module holds none of the Dirac operator's or the solver's arithmetic; it
draws inputs only, and both the CUDA path and the CPU oracle are fed from it.
The drawing is done by ``synth.c`` (compiled with gcc on first use); see its
header for the exact recipe.

The paper's own inputs are HMC gauge ensembles (Sec. 3.1), which do not exist
here; random SU(3) links U = exp(i eps H) stand in for them, at the paper's
lattice shapes, with the roughness controlled by eps.

Arrays use the canonical order t, z, y, x, spin, colour (Sec. 4.7.2):
  gauge   complex128 (T, L, L, L, 4, 3, 3), direction mu = t, x, y, z
  spinor  complex128 (T, L, L, L, 4, 3)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtm_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into _build/libtm_synth.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-fcx-limited-range", _SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            U64, L, D, P = ctypes.c_uint64, ctypes.c_long, ctypes.c_double, ctypes.c_void_p
            lib.syn_splitmix64.argtypes = [U64, U64]
            lib.syn_splitmix64.restype = U64
            lib.syn_uniform.argtypes = [U64, U64]
            lib.syn_uniform.restype = D
            lib.syn_normal.argtypes = [U64, U64]
            lib.syn_normal.restype = D
            lib.syn_normals.argtypes = [U64, U64, L, P]
            lib.syn_su3.argtypes = [U64, D, L, P]
            lib.syn_hermitian.argtypes = [U64, L, P]
            lib.syn_gaussian.argtypes = [U64, L, P]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------ random draws ---
def splitmix64(seed: int, i: int) -> int:
    """Draw i (0-based) of the SplitMix64 stream started at state `seed`."""
    return int(_load().syn_splitmix64(seed, i))


def normals(seed: int, start: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().syn_normals(seed, start, n, _ptr(out))
    return out


def random_su3(n: int, eps: float, seed: int) -> np.ndarray:
    """n matrices exp(i eps H) in SU(3), shape (n, 3, 3)."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    _load().syn_su3(seed, float(eps), n, _ptr(out))
    return out


def hermitian_generators(n: int, seed: int) -> np.ndarray:
    """The traceless Hermitian H of the first n links of stream `seed`, (n, 3, 3)."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    _load().syn_hermitian(seed, n, _ptr(out))
    return out


def random_gauge(T: int, L: int, eps: float, seed: int) -> np.ndarray:
    """Gauge field U_mu(x) = exp(i eps H), shape (T, L, L, L, 4, 3, 3)."""
    V = T * L * L * L
    return random_su3(4 * V, eps, seed).reshape(T, L, L, L, 4, 3, 3)


def unit_gauge(T: int, L: int) -> np.ndarray:
    """Free field: every link is the identity."""
    U = np.zeros((T, L, L, L, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_spinor(T: int, L: int, seed: int, shape_prefix=()) -> np.ndarray:
    """Complex Gaussian spinor field, E|component|^2 = 1, shape (*prefix, T, L, L, L, 4, 3)."""
    shape = tuple(shape_prefix) + (T, L, L, L, 4, 3)
    out = np.empty(shape, dtype=np.complex128)
    _load().syn_gaussian(seed, int(np.prod(shape)), _ptr(out))
    return out


def point_source(T: int, L: int, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """Unit point source at site (t, z, y, x), one spin and colour component."""
    out = np.zeros((T, L, L, L, 4, 3), dtype=np.complex128)
    t, z, y, x = site
    out[t, z, y, x, spin, colour] = 1.0
    return out


# -------------------------------------------------------------- workloads ---
@dataclass(frozen=True)
class Workload:
    """One lattice problem: extents, gauge roughness, kappa, bare twisted mass mu."""
    name: str
    T: int
    L: int
    eps: float
    kappa: float
    mu: float
    gauge_seed: int = 1
    source_seed: int = 2

    @property
    def V(self) -> int:
        return self.T * self.L ** 3

    @property
    def mut(self) -> float:
        """mu~ = 2 kappa mu (App. B.1)."""
        return 2.0 * self.kappa * self.mu

    def gauge(self) -> np.ndarray:
        return random_gauge(self.T, self.L, self.eps, self.gauge_seed)

    def source(self, index: int = 0) -> np.ndarray:
        return gaussian_spinor(self.T, self.L, self.source_seed + index)


# The lattice problems the library is exercised on, named by their shapes.
WORKLOADS = {
    "4^4": Workload("4^4", 4, 4, 0.3, 0.160, 0.01),
    "16^3x32": Workload("16^3x32", 32, 16, 0.5, 0.1632, 0.004),
    "32^3x64": Workload("32^3x64", 64, 32, 0.6, 0.1615, 0.003),
    "48^3x96": Workload("48^3x96", 96, 48, 0.6, 0.1615, 0.0015),
    "24^3x48": Workload("24^3x48", 48, 24, 0.6, 0.1615, 0.003),
    "8^4": Workload("8^4", 8, 8, 0.5, 0.1632, 0.002),
    "12^3x24": Workload("12^3x24", 24, 12, 0.5, 0.1632, 0.002),
}


@dataclass(frozen=True)
class BatchedSystem:
    """One system of the batched workload: its lattice problem (gauge field and kappa from the
    workload), its own bare twisted mass, and its source (a unit point source at the origin with
    spin-colour index 3 s + c, or the workload's Gaussian source number `index`)."""
    workload: Workload
    mu: float
    kind: str   # "point" or "gaussian"
    index: int

    def source(self) -> np.ndarray:
        w = self.workload
        if self.kind == "point":
            return point_source(w.T, w.L, self.index // 3, self.index % 3)
        return w.source(self.index)


BATCHED_MU = (0.002, 0.005, 0.01)


def batched_workload():
    """The batched workload: the 12 spin-colour point sources of one propagator on 24^3 x 48
    (eps 0.6, kappa 0.1615, mu 0.003), then the 8^4, 12^3 x 24 and 16^3 x 32 lattices (eps 0.5,
    kappa 0.1632) with 4 Gaussian sources each for every mu in {0.002, 0.005, 0.01}: 48 systems
    on 4 gauge fields."""
    big = WORKLOADS["24^3x48"]
    out = [BatchedSystem(big, big.mu, "point", j) for j in range(12)]
    for name in ("8^4", "12^3x24", "16^3x32"):
        for mu in BATCHED_MU:
            out += [BatchedSystem(WORKLOADS[name], mu, "gaussian", k) for k in range(4)]
    return out
