"""GPU meson contraction (tm_meson_contract) and the pion correlator from 12 point sources."""
import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import F32, LINK12, Lattice, correlator, inputs, solve_cg_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T,L", [(4, 4), (6, 2), (8, 8)])
def test_contraction_matches_oracle(T, L):
    lat = Lattice(T, L, 0.16, 0.01)
    props = inputs.gaussian_spinor(T, L, 31, shape_prefix=(12,))
    ref = oracle.meson_contract(props)
    got_dev = torch.zeros((T, 12, 12), dtype=torch.complex128, device="cuda:0")
    lat.meson_contract(torch.from_numpy(props).cuda(), out=got_dev)
    got = got_dev.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-13
    got_host = lat.meson_contract(props)  # host buffers
    assert np.array_equal(got_host, got)
    # Gram matrices are Hermitian, C_PP is real and positive
    assert np.abs(got - np.conj(np.swapaxes(got, 1, 2))).max() < 1e-10 * np.abs(got).max()
    c = correlator(got, np.eye(4))
    assert np.all(c.real > 0) and np.abs(c.imag).max() < 1e-9 * c.real.max()
    lat.close()


def test_pion_correlator_from_batched_point_sources():
    """d-quark propagator on 8^4 from 12 point sources (one batched solve), contracted on the
    GPU; compared with the oracle's contraction of the oracle's own solves."""
    w = inputs.WORKLOADS["8^4"]
    U = w.gauge()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    srcs = [inputs.point_source(w.T, w.L, s, c) for s in range(4) for c in range(3)]
    props = torch.zeros((12,) + srcs[0].shape, dtype=torch.complex128, device="cuda:0")
    bs = [torch.from_numpy(b).cuda() for b in srcs]
    systems = [(lat, w.mu, props[k], bs[k], -1) for k in range(12)]
    solve_cg_batch(systems, sloppy_prec=F32, sloppy_link=LINK12, delta=1e-3, tol=1e-12)
    A = lat.meson_contract(props)
    C = correlator(A, np.eye(4)).real
    olat = oracle.Lattice.cubic(w.T, w.L)
    ref_props = np.stack([oracle.solve(olat, U, b, w.kappa, w.mu, f=-1, tol=1e-12).psi for b in srcs])
    C_ref = oracle.correlator(oracle.meson_contract(ref_props), np.eye(4)).real
    assert np.allclose(C, C_ref, rtol=1e-8, atol=0)
    # the correlator falls off from the source and is symmetric about T/2 on average
    assert C[0] > C[1] > C[w.T // 2]
    lat.close()
