"""The seeded input generators: published RNG outputs and the properties of the draws."""
import numpy as np
import pytest

from paper_0905_3331_gb300 import inputs

scipy_linalg = pytest.importorskip("scipy.linalg")


def test_splitmix64_published_outputs():
    """First outputs of SplitMix64 from state 1234567, as printed by the published
    reference implementation (Vigna, splitmix64.c)."""
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    assert [inputs.splitmix64(1234567, i) for i in range(5)] == expect


def test_normals_moments():
    z = inputs.normals(7, 0, 1 << 20)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs((z ** 4).mean() - 3) < 0.05
    # counter-based: any window equals the same slice of a longer draw
    assert np.array_equal(inputs.normals(7, 1000, 10), z[1000:1010])


def test_generators_are_traceless_hermitian_and_normalised():
    """H = sum_a h_a lambda_a / 2: tr H = 0, H = H^dag, tr H^2 = sum h_a^2 / 2, and the map
    h -> H has rank 8 (the 8 Gell-Mann matrices are independent)."""
    n = 2000
    H = inputs.hermitian_generators(n, seed=3)
    h = inputs.normals(3, 0, 8 * n).reshape(n, 8)
    assert np.abs(np.trace(H, axis1=1, axis2=2)).max() < 1e-15
    assert np.abs(H - np.conj(np.swapaxes(H, 1, 2))).max() == 0
    tr2 = np.einsum("nij,nji->n", H, H).real
    assert np.allclose(tr2, (h ** 2).sum(1) / 2, rtol=1e-13)
    flat = np.concatenate([H.real.reshape(n, 9), H.imag.reshape(n, 9)], axis=1)
    coef, *_ = np.linalg.lstsq(h, flat, rcond=None)
    assert np.linalg.matrix_rank(coef) == 8
    assert np.allclose(h @ coef, flat, atol=1e-13)


def test_links_are_su3_and_equal_expm():
    eps = 0.6
    U = inputs.random_su3(500, eps, seed=5)
    H = inputs.hermitian_generators(500, seed=5)
    eye = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, 1, 2)) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    E = np.stack([scipy_linalg.expm(1j * eps * h) for h in H])
    assert np.abs(E - U).max() < 1e-13


def test_gauge_field_layout_and_seed():
    U = inputs.random_gauge(4, 2, 0.3, seed=1)
    assert U.shape == (4, 2, 2, 2, 4, 3, 3)
    flat = inputs.random_su3(4 * 4 * 8, 0.3, seed=1)
    assert np.array_equal(U.reshape(-1, 3, 3), flat)  # link i = lex * 4 + mu
    assert not np.array_equal(inputs.random_gauge(4, 2, 0.3, seed=2), U)


def test_gaussian_source_normalisation():
    s = inputs.gaussian_spinor(8, 8, seed=2)
    assert s.shape == (8, 8, 8, 8, 4, 3)
    m2 = (np.abs(s) ** 2).mean()
    assert abs(m2 - 1) < 0.02
    assert abs(s.real.var() - 0.5) < 0.02 and abs(s.imag.var() - 0.5) < 0.02
