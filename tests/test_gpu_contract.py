"""GPU meson contraction (tm_meson_contract), correlators (tm_correlator) and the point-source
propagators they are built from (Sec. 4.3)."""
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
    c = correlator(lat, got, np.eye(4))
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
    X = _gammas()
    C = correlator(lat, A, X)  # C_PP, C_PA, C_PV on the device
    olat = oracle.Lattice.cubic(w.T, w.L)
    ref_props = np.stack([oracle.solve(olat, U, b, w.kappa, w.mu, f=-1, tol=1e-12).psi for b in srcs])
    A_ref = oracle.meson_contract(ref_props)
    # both propagators are solutions to 1e-12: the correlators agree to about that
    for g in range(len(X)):
        C_ref = oracle.correlator(A_ref, X[g])
        assert np.linalg.norm(C[g] - C_ref) / np.linalg.norm(C_ref) < 1e-8, g
    # the pion correlator falls off from the source
    Cpp = C[0].real
    assert Cpp[0] > Cpp[1] > Cpp[w.T // 2]
    lat.close()


def _gammas():
    """X = Gamma gamma5 for C_PP (Gamma = gamma5), C_PA (Gamma = gamma0 gamma5) and C_PV
    (Gamma = gamma0), and a random complex X, gamma matrices of App. A."""
    g = [oracle.gamma(k) for k in range(5)]
    rng = np.random.default_rng(41)
    return np.stack([np.eye(4), g[0], g[0] @ g[4],
                     rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))]).astype(np.complex128)


@pytest.mark.parametrize("T,L", [(4, 4), (6, 2), (16, 8)])
def test_correlators_match_the_oracle(T, L):
    """tm_correlator against the oracle's trace, on the same Gram matrices (host and device)."""
    lat = Lattice(T, L, 0.16, 0.01)
    A = oracle.meson_contract(inputs.gaussian_spinor(T, L, 33, shape_prefix=(12,)))
    X = _gammas()
    ref = np.stack([oracle.correlator(A, x) for x in X])
    got_host = correlator(lat, A, X)
    assert np.abs(got_host - ref).max() < 1e-13 * np.abs(ref).max()
    got_dev = correlator(lat, torch.from_numpy(A).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(got_dev, got_host)
    assert np.array_equal(correlator(lat, A, X[1]), got_host[1])  # one matrix alone
    lat.close()


def _point_props(lat, mu, sites, flavour, T, L):
    """Solutions of M(flavour) x = b for the 12 point sources at each lexicographic site in
    `sites` (one batched solve, FP64 true residual 1e-12): (len(sites), 12, T, L, L, L, 4, 3)."""
    shape = (T, L, L, L, 4, 3)
    bs, xs, systems = [], [], []
    for y in sites:
        for s in range(4):
            for c in range(3):
                b = torch.zeros(shape, dtype=torch.complex128, device="cuda:0")
                b.view(-1, 4, 3)[y, s, c] = 1.0
                x = torch.zeros_like(b)
                bs.append(b)
                xs.append(x)
                systems.append((lat, mu, x, b, flavour))
    infos = solve_cg_batch(systems, sloppy_prec=F32, sloppy_link=LINK12, delta=1e-3, tol=1e-12)
    assert max(i.true_rel_residual for i in infos) < 1e-12
    return torch.stack(xs).reshape((len(sites), 12) + shape).cpu().numpy()


@pytest.mark.parametrize("T,L,nsites", [(2, 2, 16), (4, 4, 16)])
def test_u_and_d_propagators_are_related_by_gamma5_hermiticity(T, L, nsites):
    """G_u(x, 0) = gamma5 G_d(0, x)^dag gamma5 (Sec. 4.3; M(mu)^dag = gamma5 M(-mu) gamma5), site by
    site: the u propagator (flavour +1) from the 12 point sources at the origin, read at x, against
    the d propagator (flavour -1) from the 12 point sources at x, read at the origin.  On 2^4 x runs
    over every site; on 4^4 over 16 sites of both parities, including the origin and sites on the
    boundaries."""
    w = inputs.WORKLOADS["4^4"]
    U = inputs.random_gauge(T, L, w.eps, 7)
    lat = Lattice(T, L, w.kappa, w.mu)
    lat.set_gauge(U)
    V = T * L ** 3
    if nsites >= V:
        sites = np.arange(V)
    else:
        rng = np.random.default_rng(43)
        sites = np.unique(np.concatenate([[0, 1, L - 1, V - 1, V // 2], rng.choice(V, nsites, replace=False)]))[:nsites]
    Gu = _point_props(lat, w.mu, [0], +1, T, L)[0]          # [j][x][s][c]: column j of G_u(x, 0)
    Gd = _point_props(lat, w.mu, list(sites), -1, T, L)     # [y][j][x][s][c]: column j of G_d(x, y)
    g5 = np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3))       # on the 12 spin-colour indices
    Gu_sites = Gu.reshape(12, V, 12)
    worst = 0.0
    for k, y in enumerate(sites):
        u_block = Gu_sites[:, y, :].T                              # G_u(y, 0)[sink][source]
        d_block = Gd[k].reshape(12, V, 12)[:, 0, :].T              # G_d(0, y)[sink][source]
        expect = g5 @ d_block.conj().T @ g5
        worst = max(worst, np.abs(u_block - expect).max() / np.abs(expect).max())
    assert worst < 1e-10
    lat.close()
