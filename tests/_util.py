"""Test helpers: checkerboard bookkeeping between canonical full fields and half fields.

A half field of parity p lists the sites of that parity in lexicographic order
(cb = lex / 2), which is the order numpy's boolean indexing of the flattened
(T, Lz, Ly, Lx) site array produces.
"""
import numpy as np


def parity_of_sites(T, L):
    t, z, y, x = np.indices((T, L, L, L))
    return ((t + z + y + x) & 1).reshape(-1)


def to_half(field, parity):
    """canonical full (T, L, L, L, 4, 3) -> half (h, 4, 3) of the given parity."""
    T, L = field.shape[0], field.shape[1]
    flat = field.reshape(-1, 4, 3)
    return np.ascontiguousarray(flat[parity_of_sites(T, L) == parity])


def from_half(half, parity, T, L):
    """half (h, 4, 3) -> canonical full field, zero on the other parity."""
    out = np.zeros((T * L ** 3, 4, 3), dtype=np.complex128)
    out[parity_of_sites(T, L) == parity] = half
    return out.reshape(T, L, L, L, 4, 3)


def lex_of_half(T, L, parity):
    """Lexicographic site index of each half-field entry."""
    return np.flatnonzero(parity_of_sites(T, L) == parity)


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def site_rel_max(a, b):
    """Largest per-site relative error: max over sites of ||a_x - b_x|| / ||b_x|| (the 12 complex
    components of each site; arrays shaped (..., 4, 3)).  A wrong site or a wrong boundary slab
    shows here even where the global 2-norm would hide it."""
    a = np.asarray(a).reshape(-1, 12)
    b = np.asarray(b).reshape(-1, 12)
    return float((np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)).max())
