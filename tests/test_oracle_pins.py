"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself or with a retyped copy of its own
formulas.  Each pin is one of: a closed form (free-field spectrum), an algebraic
identity (Clifford algebra, gauge covariance, gamma5-hermiticity, Schur
complement), a library routine on a special case (dense inverse, dense solve,
dense Schur complement) or a worked example derived by hand from the paper
(tests/golden/point_source_unit_gauge.txt).  Together they are chosen so that a
dropped term, a wrong sign, a wrong link orientation, a transposed operand or a
misplaced boundary phase in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import Lattice
from paper_0905_3331_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "point_source_unit_gauge.txt")


# ------------------------------------------------------------------ helpers ---
def dense_from(apply, lat: Lattice, rows_mask=None, cols_mask=None):
    """Dense matrix of a linear map on spinor fields, built column by column."""
    n = 12 * lat.V
    cols = np.arange(n) if cols_mask is None else np.flatnonzero(cols_mask)
    rows = np.arange(n) if rows_mask is None else np.flatnonzero(rows_mask)
    A = np.empty((len(rows), len(cols)), dtype=np.complex128)
    e = np.zeros(lat.spinor_shape, dtype=np.complex128)
    flat = e.reshape(-1)
    for k, j in enumerate(cols):
        flat[j] = 1.0
        A[:, k] = apply(e).reshape(-1)[rows]
        flat[j] = 0.0
    return A


def component_mask(lat: Lattice, parity: int) -> np.ndarray:
    """Boolean mask over the 12 V spinor components: True on sites of the parity."""
    odd = lat.parity_mask()
    m = odd if parity == 1 else ~odd
    return np.broadcast_to(m[..., None, None], lat.spinor_shape).reshape(-1)


def free_field_momenta(lat: Lattice):
    """Allowed momenta p_nu = (2 n + theta_nu) pi / L_nu (boundary phase of Sec. 2.4)."""
    ext = (lat.T, lat.Lx, lat.Ly, lat.Lz)
    grids = [(2 * np.arange(n) + th) * np.pi / n for n, th in zip(ext, lat.theta)]
    P = np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1).reshape(-1, 4)
    return P


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def rand_spinor(lat, seed):
    return inputs.gaussian_spinor(lat.T, lat.Lx, seed)


# ------------------------------------------------------------- App. A ---
def test_gamma_matrices_clifford_algebra():
    """{gamma_mu, gamma_nu} = 2 delta, each Hermitian, gamma0 gamma1 gamma2 gamma3 = gamma5 = diag(1,1,-1,-1)."""
    g = [oracle.gamma(k) for k in range(5)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            ac = g[m] @ g[n] + g[n] @ g[m]
            assert np.array_equal(ac, 2.0 * (m == n) * np.eye(4))
    assert np.array_equal(g[0] @ g[1] @ g[2] @ g[3], g[4])
    assert np.array_equal(g[4], np.diag([1.0, 1.0, -1.0, -1.0]).astype(complex))
    for m in range(4):
        assert np.array_equal(g[4] @ g[m], -g[m] @ g[4])


# --------------------------------------------------- hand-derived example ---
def _read_golden():
    hops, diag = [], {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "diag":
                diag[int(tok[1])] = complex(float(tok[2]), float(tok[3]))
            else:
                s0, mu, side = int(tok[0]), int(tok[1]), tok[2]
                v = np.array([complex(float(tok[3 + 2 * k]), float(tok[4 + 2 * k]))
                              for k in range(4)])
                hops.append((s0, mu, side, v))
    return hops, diag


def test_point_source_worked_example():
    """H and M on a point source over a unit gauge field match the hand-derived values."""
    lat = Lattice.cubic(4, 4)
    U = inputs.unit_gauge(4, 4)
    x0 = (0, 1, 2, 3)  # (t, z, y, x)
    hops, diag = _read_golden()
    kappa, mu = 0.125, 0.2
    c0 = 1
    for s0 in (0, 2):
        src = inputs.point_source(4, 4, s0, c0, x0)
        H = oracle.hopping(lat, U, src)
        M = oracle.apply_M(lat, U, src, kappa, mu)
        expect = np.zeros(lat.spinor_shape, dtype=complex)
        for (s, mu_dir, side, v) in hops:
            if s != s0:
                continue
            # axis of the array for direction mu: t -> 0, x -> 3, y -> 2, z -> 1
            axis = {0: 0, 1: 3, 2: 2, 3: 1}[mu_dir]
            site = list(x0)
            site[axis] = (site[axis] + (-1 if side == "fwd" else 1)) % 4
            expect[tuple(site)][:, c0] = v
        assert np.array_equal(H, expect), f"s0={s0}"
        expect_M = -kappa * expect
        for s in range(4):
            if s == s0:
                expect_M[x0][s, c0] = diag[s0]
        assert np.allclose(M, expect_M, rtol=0, atol=1e-15)


# ------------------------------------------------------ free-field closed form ---
@pytest.mark.parametrize("T,L", [(2, 2), (4, 2)])
def test_free_field_eigenvalues_of_M(T, L):
    """Unit gauge: eigenvalues of M are 1 - 2k sum cos p +- i sqrt(mu~^2 + 4k^2 sum sin^2 p), 6-fold."""
    lat = Lattice.cubic(T, L)
    kappa, mu = 0.13, 0.35
    mut = 2 * kappa * mu
    U = inputs.unit_gauge(T, L)
    M = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, mu), lat)
    ev = np.linalg.eigvals(M)
    P = free_field_momenta(lat)
    a = 1 - 2 * kappa * np.cos(P).sum(1)
    w = np.sqrt(mut ** 2 + 4 * kappa ** 2 * (np.sin(P) ** 2).sum(1))
    expect = np.concatenate([np.repeat(a + 1j * w, 6), np.repeat(a - 1j * w, 6)])
    key = lambda z: np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))
    assert np.allclose(ev[key(ev)], expect[key(expect)], atol=1e-10)


@pytest.mark.parametrize("T,L,theta", [(4, 4, (1.0, 0.0, 0.0, 0.0)), (4, 2, (0.0, 0.0, 0.0, 0.0)),
                                       (2, 4, (1.0, 0.5, 0.0, 0.25))])
def test_free_field_spectrum_of_MdagM(T, L, theta):
    """Unit gauge: eigenvalues of M^dag M are (1 - 2k sum cos p)^2 + 4k^2 sum sin^2 p + mu~^2, 12-fold."""
    lat = Lattice(T, L, L, L, theta=theta)
    kappa, mu = 0.16, 0.01
    mut = 2 * kappa * mu
    U = inputs.unit_gauge(T, L)
    M = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, mu), lat)
    ev = np.linalg.eigvalsh(M.conj().T @ M)
    P = free_field_momenta(lat)
    lam = (1 - 2 * kappa * np.cos(P).sum(1)) ** 2 + 4 * kappa ** 2 * (np.sin(P) ** 2).sum(1) + mut ** 2
    assert np.allclose(np.sort(ev), np.sort(np.repeat(lam, 12)), rtol=0, atol=1e-12)


# ----------------------------------------------------------- link dependence ---
def test_gauge_covariance():
    """U_mu(x) -> G(x) U_mu(x) G(x+mu)^dag, psi -> G psi  implies  M psi -> G M psi."""
    T, L = 4, 4
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.7, seed=11)
    G = inputs.random_su3(lat.V, 2.0, seed=12).reshape(T, L, L, L, 3, 3)
    axis = {0: 0, 1: 3, 2: 2, 3: 1}
    Ug = np.empty_like(U)
    for mu in range(4):
        Gfwd = np.roll(G, -1, axis=axis[mu])  # G(x + mu^)
        Ug[..., mu, :, :] = G @ U[..., mu, :, :] @ np.conj(np.swapaxes(Gfwd, -1, -2))
    psi = rand_spinor(lat, 13)
    psig = np.einsum("tzyxab,tzyxsb->tzyxsa", G, psi)
    kappa, mu = 0.16, 0.05
    lhs = oracle.apply_M(lat, Ug, psig, kappa, mu)
    rhs = np.einsum("tzyxab,tzyxsb->tzyxsa", G, oracle.apply_M(lat, U, psi, kappa, mu))
    assert rel(lhs, rhs) < 1e-13


# ------------------------------------------------------- adjoint structure ---
def test_gamma5_hermiticity_with_twisted_mass():
    """<chi, g5 M(mu) g5 psi> = <M(-mu) chi, psi>, i.e. g5 M(mu) g5 = M(-mu)^dag."""
    T, L = 4, 4
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.6, seed=21)
    psi, chi = rand_spinor(lat, 22), rand_spinor(lat, 23)
    g5 = np.array([1, 1, -1, -1])[:, None]
    kappa, mu = 0.16, 0.07
    lhs = np.vdot(chi, g5 * oracle.apply_M(lat, U, g5 * psi, kappa, mu))
    rhs = np.vdot(oracle.apply_M(lat, U, chi, kappa, -mu), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # and the plain identity at mu = 0; f = -1 is mu -> -mu
    lhs0 = np.vdot(chi, g5 * oracle.apply_M(lat, U, g5 * psi, kappa, 0.0))
    rhs0 = np.vdot(oracle.apply_M(lat, U, chi, kappa, 0.0), psi)
    assert abs(lhs0 - rhs0) < 1e-12 * abs(rhs0)
    assert np.allclose(oracle.apply_M(lat, U, psi, kappa, mu, f=-1),
                       oracle.apply_M(lat, U, psi, kappa, -mu), rtol=0, atol=1e-15)


# ------------------------------------------------------- boundary phases ---
@pytest.mark.parametrize("theta", [(1.0, 0.0, 0.0, 0.0), (1.0, 0.3, 0.0, 0.7)])
def test_boundary_phase_placement_equivalence(theta):
    """Spread phases (Sec. 4.1.2) = W^dag M W with boundary phases (Sec. 2.4), W = exp(i pi sum theta x/L)."""
    T, L = 4, 4
    lb = Lattice(T, L, L, L, theta=theta)
    ls = Lattice(T, L, L, L, theta=theta, spread=True)
    U = inputs.random_gauge(T, L, 0.5, seed=31)
    psi = rand_spinor(lb, 32)
    t, z, y, x = np.indices((T, L, L, L))
    ph = np.exp(1j * np.pi * (theta[0] * t / T + theta[1] * x / L + theta[2] * y / L
                              + theta[3] * z / L))[..., None, None]
    lhs = oracle.apply_M(ls, U, psi, 0.15, 0.02)
    rhs = np.conj(ph) * oracle.apply_M(lb, U, ph * psi, 0.15, 0.02)
    assert rel(lhs, rhs) < 1e-13
    # and the phase is really there: the periodic operator differs
    lp = Lattice(T, L, L, L, theta=(0.0, 0.0, 0.0, 0.0))
    assert rel(oracle.apply_M(lp, U, psi, 0.15, 0.02), oracle.apply_M(lb, U, psi, 0.15, 0.02)) > 1e-3


# --------------------------------------------------- even/odd blocks (B.1) ---
def test_site_diagonal_inverse_is_the_inverse():
    """(M_ee)^-1 of eq. eo3 equals numpy's inverse of the 12x12 site block and inverts M_ee."""
    lat = Lattice.cubic(2, 2)
    mut = 0.37
    even_site = (0, 0, 0, 0)
    for f in (+1, -1):
        blk = np.zeros((12, 12), complex)
        blk_inv = np.zeros((12, 12), complex)
        for j in range(12):
            e = np.zeros(lat.spinor_shape, complex)
            e[even_site].reshape(-1)[j] = 1.0
            blk[:, j] = oracle.apply_Mdiag(lat, e, mut, f, 0)[even_site].reshape(-1)
            blk_inv[:, j] = oracle.apply_Mdiag_inv(lat, e, mut, f, 0)[even_site].reshape(-1)
        assert np.allclose(blk_inv, np.linalg.inv(blk), rtol=0, atol=1e-15)
        # M_ee = 1 + i f mu~ gamma5 (x) 1_colour
        g5 = np.diag([1, 1, -1, -1]).astype(complex)
        assert np.allclose(blk, np.kron(np.eye(4) + 1j * f * mut * g5, np.eye(3)), atol=1e-16)
    psi = rand_spinor(lat, 41)
    back = oracle.apply_Mdiag(lat, oracle.apply_Mdiag_inv(lat, psi, mut, 1, 1), mut, 1, 1)
    odd = lat.parity_mask()[..., None, None]
    assert rel(back, np.where(odd, psi, 0)) < 1e-15


def test_even_odd_blocks_tile_the_operator():
    """M = diag - kappa (H_eo + H_oe): the parity-restricted hoppings add up to the full one."""
    T, L = 4, 4
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.5, seed=51)
    psi = rand_spinor(lat, 52)
    H = oracle.hopping(lat, U, psi)
    He = oracle.hopping(lat, U, psi, out_parity=0)
    Ho = oracle.hopping(lat, U, psi, out_parity=1)
    assert np.array_equal(He + Ho, H)
    odd = lat.parity_mask()[..., None, None]
    # H_eo reads only odd sites: zeroing the even input changes nothing
    assert np.array_equal(oracle.hopping(lat, U, np.where(odd, psi, 0), out_parity=0), He)
    kappa, mu = 0.15, 0.03
    M = oracle.apply_M(lat, U, psi, kappa, mu)
    D = oracle.apply_Mdiag(lat, psi, 2 * kappa * mu, 1, 0) + oracle.apply_Mdiag(lat, psi, 2 * kappa * mu, 1, 1)
    assert rel(M, D - kappa * H) < 1e-15
    assert np.allclose(oracle.apply_Moff(lat, U, psi, kappa, 1), -kappa * Ho, atol=0)


@pytest.mark.parametrize("T,L", [(2, 2), (4, 4)])
def test_schur_operator_is_the_dense_schur_complement(T, L):
    """Mhat = M_oo - M_oe M_ee^-1 M_eo, computed with numpy from dense blocks of M (eq. eo2/eo4),
    and det M = det M_ee det Mhat."""
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.6, seed=61)
    kappa, mu = 0.16, 0.04
    for f in (+1, -1):
        M = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, mu, f), lat)
        e, o = component_mask(lat, 0), component_mask(lat, 1)
        Mee, Meo = M[np.ix_(e, e)], M[np.ix_(e, o)]
        Moe, Moo = M[np.ix_(o, e)], M[np.ix_(o, o)]
        S = Moo - Moe @ np.linalg.solve(Mee, Meo)
        Mhat = dense_from(lambda v: oracle.schur(lat, U, v, kappa, mu, f), lat,
                          rows_mask=o, cols_mask=o)
        assert np.abs(Mhat - S).max() < 1e-13
        s1, l1 = np.linalg.slogdet(M)
        s2, l2 = np.linalg.slogdet(Mee)
        s3, l3 = np.linalg.slogdet(Mhat)
        assert abs(l1 - (l2 + l3)) < 1e-9 and abs(s1 - s2 * s3) < 1e-9
        # Qhat = gamma5 Mhat and (Qhat^f)^dag = Qhat^-f (eq. eo6)
        Q = dense_from(lambda v: oracle.schur(lat, U, v, kappa, mu, f, gamma5=True), lat,
                       rows_mask=o, cols_mask=o)
        Qm = dense_from(lambda v: oracle.schur(lat, U, v, kappa, mu, -f, gamma5=True), lat,
                        rows_mask=o, cols_mask=o)
        g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), lat.V // 2)
        assert np.abs(Q - g5[:, None] * Mhat).max() == 0
        assert np.abs(Q.conj().T - Qm).max() < 1e-14


@pytest.mark.parametrize("T,L", [(2, 2), (4, 4)])
def test_even_odd_solve_equals_dense_solve(T, L):
    """The even/odd Schur + CG solve (App. B.2) equals numpy's dense solve of M psi = phi."""
    lat = Lattice.cubic(T, L)
    w = inputs.WORKLOADS["4^4"]
    U = inputs.random_gauge(T, L, w.eps, seed=w.gauge_seed)
    phi = inputs.gaussian_spinor(T, L, w.source_seed)
    M = dense_from(lambda v: oracle.apply_M(lat, U, v, w.kappa, w.mu), lat)
    psi_dense = np.linalg.solve(M, phi.reshape(-1)).reshape(lat.spinor_shape)
    res = oracle.solve(lat, U, phi, w.kappa, w.mu, tol=1e-13, max_iter=5000)
    assert res.converged
    assert rel(res.psi, psi_dense) < 1e-10
    # residual identities: even part of phi - M psi vanishes, full = normal residual
    r = phi - oracle.apply_M(lat, U, res.psi, w.kappa, w.mu)
    odd = lat.parity_mask()[..., None, None]
    assert np.linalg.norm(np.where(odd, 0, r)) < 1e-14 * np.linalg.norm(phi)
    varphi = oracle.eo_prepare(lat, U, phi, w.kappa, w.mu)
    bnorm = np.linalg.norm(np.where(odd, varphi, 0))
    assert abs(res.relres_full * np.linalg.norm(phi) - res.relres_normal * bnorm) < 1e-13 * bnorm


def test_reconstruction_residual_is_the_normal_residual_for_any_X():
    """For any X on the odd sites, not only a solution: with x_o = Qhat^-f X and x_e reconstructed
    as in App. B.2, the full residual phi - M x vanishes on the even sites (up to rounding), and
    its odd part is gamma5 (b - Qhat^f Qhat^-f X) with b = gamma5 varphi_o (eq. eo6), for both
    flavours.  A mixed solve relies on this when it confirms convergence through the
    reconstruction's residual."""
    T, L = 4, 4
    lat = Lattice.cubic(T, L)
    w = inputs.WORKLOADS["4^4"]
    U = inputs.random_gauge(T, L, w.eps, seed=w.gauge_seed)
    phi = inputs.gaussian_spinor(T, L, w.source_seed)
    g5 = oracle.gamma(4)
    odd = lat.parity_mask()[..., None, None]

    def gamma5(v):
        return np.einsum("ab,...bc->...ac", g5, v)

    for f in (1, -1):
        X = _odd(lat, 17 + f)
        varphi = oracle.eo_prepare(lat, U, phi, w.kappa, w.mu, f)
        b = np.where(odd, gamma5(varphi), 0)
        xo = np.where(odd, oracle.schur(lat, U, X, w.kappa, w.mu, -f, gamma5=True), 0)
        psi = oracle.eo_reconstruct(lat, U, varphi, xo, w.kappa, w.mu, f)
        r = phi - oracle.apply_M(lat, U, psi, w.kappa, w.mu, f)
        rn = b - oracle.normal_op(lat, U, X, w.kappa, w.mu, f)
        assert np.linalg.norm(np.where(odd, 0, r)) < 1e-13 * np.linalg.norm(phi)
        assert rel(np.where(odd, r, 0), np.where(odd, gamma5(rn), 0)) < 1e-12


def test_cg_reaches_tolerance_on_4x4x4x4():
    """4^4 workload (kappa 0.160, mu 0.01, eps 0.3): CG stops with a true relative residual below 1e-10."""
    w = inputs.WORKLOADS["4^4"]
    lat = Lattice.cubic(w.T, w.L)
    U = w.gauge()
    phi = w.source()
    res = oracle.solve(lat, U, phi, w.kappa, w.mu, tol=1e-10)
    assert res.converged and res.relres_normal < 1e-10
    r = phi - oracle.apply_M(lat, U, res.psi, w.kappa, w.mu)
    assert np.linalg.norm(r) / np.linalg.norm(phi) < 1e-10
    # flavour -1 solves M(-mu)
    res_m = oracle.solve(lat, U, phi, w.kappa, w.mu, f=-1, tol=1e-10)
    r = phi - oracle.apply_M(lat, U, res_m.psi, w.kappa, -w.mu)
    assert np.linalg.norm(r) / np.linalg.norm(phi) < 1e-10


def test_cg_on_normal_equations_matches_dense():
    """orc_cg solves Qhat+ Qhat- X = b: compare X with numpy's solve of the dense normal operator."""
    lat = Lattice.cubic(2, 2)
    U = inputs.random_gauge(2, 2, 0.5, seed=71)
    kappa, mu = 0.16, 0.05
    o = component_mask(lat, 1)
    A = dense_from(lambda v: oracle.normal_op(lat, U, v, kappa, mu), lat, rows_mask=o, cols_mask=o)
    assert np.abs(A - A.conj().T).max() < 1e-14
    b = np.where(lat.parity_mask()[..., None, None], inputs.gaussian_spinor(2, 2, 72), 0)
    res = oracle.cg(lat, U, b, kappa, mu, tol=1e-13)
    X = np.linalg.solve(A, b.reshape(-1)[o])
    assert res.converged and rel(res.x.reshape(-1)[o], X) < 1e-10
    # conjugate gradients end within the dimension of the system (here 12 V / 2 = 96)
    assert res.iters <= A.shape[0]


def test_lambda_min_bound():
    """M^dag M = W^dag W + mu~^2 >= mu~^2 on a rough random gauge field."""
    lat = Lattice.cubic(4, 4)
    U = inputs.random_gauge(4, 4, 0.9, seed=81)
    kappa, mu = 0.17, 0.05
    mut = 2 * kappa * mu
    M = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, mu), lat)
    lam = np.linalg.eigvalsh(M.conj().T @ M)
    assert lam.min() >= mut ** 2 * (1 - 1e-9)
    M0 = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, 0.0), lat)
    lam0 = np.linalg.eigvalsh(M0.conj().T @ M0)
    assert np.allclose(lam, lam0 + mut ** 2, atol=1e-11)


def test_sampled_sites_match_full_application():
    lat = Lattice.cubic(4, 4)
    U = inputs.random_gauge(4, 4, 0.5, seed=91)
    psi = rand_spinor(lat, 92)
    full = oracle.apply_M(lat, U, psi, 0.16, 0.01).reshape(lat.V, 4, 3)
    sites = np.array([0, 5, 77, 255, 128])
    part = oracle.apply_M_sites(lat, U, psi, 0.16, 0.01, sites)
    assert np.array_equal(part, full[sites])


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 4)])
def test_sampled_hopping_sites_match_full_hopping(dims):
    """orc_hopping_sites (the checker of the sampled-site hopping parity on large lattices)
    gives, at scattered sites of both parities, the rows of the full hopping sum H psi and of
    its even/odd restrictions H_eo, H_oe: bit for bit, on a random gauge field and spinor."""
    T, Lx, Ly, Lz = dims
    lat = Lattice(T, Lx, Ly, Lz)
    U = np.empty(lat.gauge_shape, dtype=np.complex128)
    Uc = inputs.random_gauge(T, Lx, 0.5, seed=95) if Lx == Ly == Lz else None
    if Uc is not None:
        U[...] = Uc
    else:  # random SU(3) links of a non-cubic lattice: QR of complex Gaussians, det fixed
        rng = np.random.default_rng(95)
        Z = rng.normal(size=lat.gauge_shape) + 1j * rng.normal(size=lat.gauge_shape)
        Q, R = np.linalg.qr(Z)
        d = np.diagonal(R, axis1=-2, axis2=-1)
        Q = Q * (d / np.abs(d))[..., None, :]
        U[...] = Q / np.linalg.det(Q)[..., None, None] ** (1 / 3)
    rng = np.random.default_rng(96)
    psi = rng.normal(size=lat.spinor_shape) + 1j * rng.normal(size=lat.spinor_shape)
    full = oracle.hopping(lat, U, psi).reshape(lat.V, 4, 3)
    sites = np.unique(np.concatenate([rng.integers(0, lat.V, 40), [0, 1, lat.V - 2, lat.V - 1]]))
    odd = lat.parity_mask().reshape(-1)
    assert odd[sites].any() and (~odd[sites]).any()
    part = oracle.hopping_sites(lat, U, psi, sites)
    assert np.array_equal(part, full[sites])
    for p in (0, 1):  # H_{p,1-p}: the input on the other parity only
        other = np.where(lat.parity_mask()[..., None, None] == (1 - p), psi, 0)
        restricted = oracle.hopping(lat, U, other, out_parity=p).reshape(lat.V, 4, 3)
        mine = sites[odd[sites] == p]
        assert np.array_equal(oracle.hopping_sites(lat, U, other, mine), restricted[mine])


# ------------------------------------------------------ correlators (Sec. 4.3) ---
def _free_field_point_propagators(T, L, kappa, mu):
    """The oracle's 12 point-source solves on a unit gauge field, and the closed form of the
    same propagator from momentum space: G(x,0) = (1/V) sum_p e^{ipx} M(p)^-1 with
    M(p) = (1 - 2k sum cos p) + i mu~ g5 - 2ik sum g_mu sin p_mu (antiperiodic p_t), as a
    (T, L, L, L, 4, 4) array [..., sink spin, source spin] (the colour part is the identity)."""
    lat = Lattice.cubic(T, L)
    U = inputs.unit_gauge(T, L)
    mut = 2 * kappa * mu
    props = []
    for s in range(4):
        for c in range(3):
            res = oracle.solve(lat, U, inputs.point_source(T, L, s, c), kappa, mu, tol=1e-13)
            assert res.converged
            props.append(res.psi)
    g = [oracle.gamma(k) for k in range(5)]
    P = free_field_momenta(lat)  # (p_t, p_x, p_y, p_z)
    t, z, y, x = np.indices((T, L, L, L))
    G = np.zeros((T, L, L, L, 4, 4), dtype=complex)
    for p in P:
        Mp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 1j * mut * g[4] \
            - 2j * kappa * sum(g[m] * np.sin(p[m]) for m in range(4))
        phase = np.exp(1j * (p[0] * t + p[1] * x + p[2] * y + p[3] * z))
        G += phase[..., None, None] * np.linalg.inv(Mp)
    G /= lat.V
    return np.stack(props), G


def test_free_field_pion_correlator_from_momentum_space():
    """C_PP(t) = sum_x ||G(x,0)||^2 of the oracle's 12 point-source solves on a unit gauge field
    equals the closed form of the propagator from momentum space, summed over each timeslice."""
    T, L = 4, 4
    props, G = _free_field_point_propagators(T, L, 0.12, 0.05)
    A = oracle.meson_contract(props)
    C = oracle.correlator(A, np.eye(4)).real
    C_closed = 3 * (np.abs(G) ** 2).sum(axis=(1, 2, 3, 4, 5))  # colour identity: 3 copies
    assert np.allclose(C, C_closed, rtol=1e-9, atol=0)
    # the point-source propagator itself, spin block of colour 0, at every site
    Gsolve = props.reshape(4, 3, T, L, L, L, 4, 3)[:, 0, ..., 0]  # [s_src, ..., s_sink]
    assert np.allclose(np.moveaxis(Gsolve, 0, -1), G, rtol=0, atol=1e-10)


def test_free_field_correlators_with_gamma_from_momentum_space():
    """C_PG(t) = sum_x tr[G(x,0)^dag G(x,0) Gamma gamma5] (Sec. 4.3) for Gamma != 1: the
    axial (Gamma = gamma0 gamma5, C_PA), vector (Gamma = gamma0, C_PV) and a random complex
    Gamma, against the closed-form propagator with the trace written out index by index:
    tr[G^dag G X] = sum_{a,b,c} conj(G[a,b]) G[a,c] X[c,b] (a the sink spin; colour: 3 copies).
    The random Gamma fails a transposed or conjugated Gamma, which gamma0 (real symmetric in
    the basis of App. A) would not."""
    T, L = 4, 4
    props, G = _free_field_point_propagators(T, L, 0.12, 0.05)
    A = oracle.meson_contract(props)
    g = [oracle.gamma(k) for k in range(5)]
    rng = np.random.default_rng(5)
    gammas = {"PA": g[0] @ g[4], "PV": g[0],
              "random": rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))}
    for name, Gam in gammas.items():
        X = Gam @ g[4]
        C = oracle.correlator(A, X)
        C_closed = 3 * np.einsum("tzyxab,tzyxac,cb->t", G.conj(), G, X)
        assert np.abs(C_closed).max() > 1e-6, name  # the pin has something to compare
        assert np.allclose(C, C_closed, rtol=1e-9, atol=1e-13 * np.abs(C_closed).max()), name


# ------------------------------------------- chronological guess (Sec. 4.2) ---
def _odd(lat, seed):
    return np.where(lat.parity_mask()[..., None, None], rand_spinor(lat, seed), 0)


def test_chrono_guess_is_exact_on_its_span():
    """phi = A X* with X* = sum_i a_i chi_i: the Galerkin system has the unique solution a,
    so the guess reproduces X* and the coefficients a."""
    lat = Lattice.cubic(4, 2)
    U = inputs.random_gauge(4, 2, 0.5, seed=91)
    kappa, mu = 0.16, 0.04
    chis = [_odd(lat, 92 + i) for i in range(4)]
    a = np.array([0.7 - 0.2j, -1.1 + 0.4j, 0.05j, 2.0])
    Xs = sum(ai * c for ai, c in zip(a, chis))
    phi = oracle.normal_op(lat, U, Xs, kappa, mu, f=-1)
    X0, c = oracle.chrono_guess(lat, U, chis, phi, kappa, mu, f=-1)
    assert np.allclose(c, a, rtol=0, atol=1e-11)
    assert rel(X0, Xs) < 1e-11


def test_chrono_guess_with_a_krylov_history_is_the_cg_iterate():
    """CG from X = 0 minimises the A-norm of the error over the Krylov space
    span{phi, A phi, ..., A^(k-1) phi}; the guess minimises the same functional over the span
    of its history, so with that Krylov basis as history it equals the k-th CG iterate."""
    lat = Lattice.cubic(4, 2)
    U = inputs.random_gauge(4, 2, 0.6, seed=93)
    kappa, mu = 0.15, 0.03
    phi = _odd(lat, 94)
    for k in (1, 3):
        basis = [phi]
        for _ in range(k - 1):
            v = oracle.normal_op(lat, U, basis[-1], kappa, mu)
            basis.append(v / np.linalg.norm(v))
        X0, _ = oracle.chrono_guess(lat, U, basis, phi, kappa, mu)
        res = oracle.cg(lat, U, phi, kappa, mu, tol=1e-30, max_iter=k)
        assert res.iters == k
        assert rel(X0, res.x) < 1e-9


def test_chrono_guess_minimises_the_error_functional():
    """Galerkin orthogonality <chi_j, phi - A X0> = 0 for every j, and every other
    combination of the history has a larger A-norm error than X0 (dense solve for X*)."""
    lat = Lattice.cubic(2, 2)
    U = inputs.random_gauge(2, 2, 0.5, seed=95)
    kappa, mu = 0.16, 0.05
    o = component_mask(lat, 1)
    A = dense_from(lambda v: oracle.normal_op(lat, U, v, kappa, mu), lat, rows_mask=o, cols_mask=o)
    phi = _odd(lat, 96)
    chis = [_odd(lat, 97 + i) for i in range(3)]
    X0, c = oracle.chrono_guess(lat, U, chis, phi, kappa, mu)
    r = phi.reshape(-1)[o] - A @ X0.reshape(-1)[o]
    for chi in chis:
        assert abs(np.vdot(chi.reshape(-1)[o], r)) < 1e-11 * np.linalg.norm(phi)
    Xs = np.linalg.solve(A, phi.reshape(-1)[o])
    B = np.stack([chi.reshape(-1)[o] for chi in chis], axis=1)

    def err(cc):
        e = B @ cc - Xs
        return np.vdot(e, A @ e).real

    e0 = err(c)
    rng = np.random.default_rng(98)
    for _ in range(20):
        d = 1e-3 * (rng.standard_normal(3) + 1j * rng.standard_normal(3))
        assert err(c + d) > e0


# ------------------------------------------------- BiCGstab on Mhat (Sec. 4.4) ---
def test_bicgstab_iterates_match_scipy():
    """The oracle's BiCGstab on the Schur operator produces the same iterates as SciPy's
    bicgstab (a library routine) on the dense Schur matrix, iteration by iteration."""
    from scipy.sparse.linalg import bicgstab as scipy_bicgstab
    lat = Lattice.cubic(4, 2)
    U = inputs.random_gauge(4, 2, 0.5, seed=101)
    kappa, mu = 0.15, 0.05
    o = component_mask(lat, 1)
    Mh = dense_from(lambda v: oracle.schur(lat, U, v, kappa, mu, f=-1), lat, rows_mask=o, cols_mask=o)
    b = _odd(lat, 102)
    iterates = []
    scipy_bicgstab(Mh, b.reshape(-1)[o], rtol=1e-30, atol=0.0, maxiter=6,
                   callback=lambda xk: iterates.append(np.array(xk)))
    assert len(iterates) == 6
    for k in (1, 2, 3, 6):
        res = oracle.bicgstab(lat, U, b, kappa, mu, f=-1, tol=1e-30, max_iter=k)
        assert res.iters == k
        assert rel(res.x.reshape(-1)[o], iterates[k - 1]) < 1e-12, k


@pytest.mark.parametrize("T,L", [(2, 2), (4, 2)])
def test_bicgstab_solve_equals_dense_solve(T, L):
    """Even/odd + BiCGstab on Mhat gives the solution of the dense full system M psi = phi,
    for both flavours, and the same solution as the CG path."""
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.5, seed=103)
    kappa, mu = 0.16, 0.04
    phi = rand_spinor(lat, 104)
    for f in (1, -1):
        M = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, mu, f), lat)
        psi = np.linalg.solve(M, phi.reshape(-1))
        res = oracle.solve_bicgstab(lat, U, phi, kappa, mu, f, tol=1e-12)
        assert res.converged and res.relres_full < 1e-11
        assert rel(res.psi.reshape(-1), psi) < 1e-10
        cg = oracle.solve(lat, U, phi, kappa, mu, f, tol=1e-12)
        assert rel(res.psi, cg.psi) < 1e-10


def test_bicgstab_reaches_tolerance_on_4x4x4x4():
    w = inputs.WORKLOADS["4^4"]
    lat = Lattice.cubic(w.T, w.L)
    U, phi = w.gauge(), w.source()
    res = oracle.solve_bicgstab(lat, U, phi, w.kappa, w.mu, tol=1e-10)
    assert res.converged and res.relres_full < 1e-10
    resid = phi - oracle.apply_M(lat, U, res.psi, w.kappa, w.mu)
    assert np.linalg.norm(resid) / np.linalg.norm(phi) < 1e-10


# ------------------------------------- non-degenerate doublet (eq. Dh, Sec. 2.3) ---
def _doublet(lat, seed):
    return np.stack([rand_spinor(lat, seed), rand_spinor(lat, seed + 1)])


def dense_doublet(apply, lat):
    n = 24 * lat.V
    A = np.empty((n, n), dtype=np.complex128)
    e = np.zeros((2,) + lat.spinor_shape, dtype=np.complex128)
    flat = e.reshape(-1)
    for j in range(n):
        flat[j] = 1.0
        A[:, j] = apply(e).reshape(-1)
        flat[j] = 0.0
    return A


def test_doublet_reconstruction_residual_is_the_normal_residual_for_any_Y():
    """The doublet's even/odd form (the block elimination of App. B.1 with the site term
    D = 1 + i mb g5 tau3 + eb tau1, Schur operator Mhat_h = D - kappa^2 H_oe D^-1 H_eo,
    Qhat_h = G Mhat_h with G = g5 tau1): for ANY odd-site Y, x_o = Qhat_h Y and
    x_e = D^-1 (b_e + kappa H_eo x_o) leave a full residual b - M_h x (the oracle's M_h of
    eq. Dh, applied by its definition) that vanishes on the even sites, and whose odd part is
    G (G varphi_o - Qhat_h^2 Y) with varphi_o = b_o + kappa H_oe D^-1 b_e.  A mixed doublet
    solve relies on this when it confirms convergence through the reconstruction's residual.
    D, D^-1 and G are built here as 8 x 8 matrices on (flavour, spin) from App. A's matrices."""
    T, L = 4, 2
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.5, seed=111)
    kappa, mubar, epsbar = 0.16, 0.15, 0.19
    mb, eb = 2 * kappa * mubar, 2 * kappa * epsbar
    g5 = oracle.gamma(4)
    tau = [oracle.pauli(k) for k in range(4)]
    D = np.eye(8) + 1j * mb * np.kron(tau[3], g5) + eb * np.kron(tau[1], np.eye(4))
    Dinv = np.linalg.inv(D)
    G = np.kron(tau[1], g5)

    def site(Mat, v):  # Mat on the (flavour, spin) index of a doublet field
        w = np.moveaxis(v, 0, -3)                       # (T, Lz, Ly, Lx, 2, 4, 3)
        w = w.reshape(w.shape[:4] + (8, 3))
        out = np.einsum("ab,...bc->...ac", Mat, w).reshape(w.shape[:4] + (2, 4, 3))
        return np.moveaxis(out, -3, 0)

    def hop(v, p):  # H_{p,1-p} on both flavours
        return np.stack([oracle.hopping(lat, U, v[f], out_parity=p) for f in (0, 1)])

    oddm = lat.parity_mask()[None, ..., None, None]
    even = lambda v: np.where(oddm, 0, v)  # noqa: E731
    odd = lambda v: np.where(oddm, v, 0)   # noqa: E731

    def mhat(v):
        return odd(site(D, v)) - kappa ** 2 * hop(even(site(Dinv, hop(v, 0))), 1)

    def qhat(v):
        return site(G, mhat(v))

    b = _doublet(lat, 112)
    varphi = odd(b) + kappa * hop(even(site(Dinv, even(b))), 1)
    Y = odd(_doublet(lat, 114))
    xo = qhat(Y)
    xe = even(site(Dinv, even(b) + kappa * hop(xo, 0)))
    r = b - oracle.apply_Mh(lat, U, xe + xo, kappa, mubar, epsbar)
    assert np.linalg.norm(even(r)) < 1e-13 * np.linalg.norm(b)
    expect = site(G, site(G, varphi) - qhat(qhat(Y)))
    assert rel(odd(r), expect) < 1e-12
    # and with Y the solution of Qhat_h^2 Y = G varphi_o, x solves M_h x = b
    o = np.flatnonzero(np.broadcast_to(oddm, b.shape).reshape(-1))
    n = len(o)
    Q2 = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(b.shape, dtype=np.complex128)
    for k, j in enumerate(o):
        e.reshape(-1)[j] = 1.0
        Q2[:, k] = qhat(qhat(e)).reshape(-1)[o]
        e.reshape(-1)[j] = 0.0
    Ys = np.zeros(b.shape, dtype=np.complex128)
    Ys.reshape(-1)[o] = np.linalg.solve(Q2, site(G, varphi).reshape(-1)[o])
    xo = qhat(Ys)
    xe = even(site(Dinv, even(b) + kappa * hop(xo, 0)))
    assert rel(oracle.apply_Mh(lat, U, xe + xo, kappa, mubar, epsbar), b) < 1e-12


def test_pauli_matrices_algebra():
    """tau_a tau_b = delta_ab + i eps_abc tau_c for the App. A matrices (exact)."""
    t = [oracle.pauli(k) for k in range(4)]
    assert np.array_equal(t[0], np.eye(2))
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    for a in range(3):
        for b in range(3):
            rhs = (a == b) * np.eye(2) + 1j * sum(eps[a, b, c] * t[c + 1] for c in range(3))
            assert np.array_equal(t[a + 1] @ t[b + 1], rhs)


def test_doublet_without_splitting_is_two_twisted_flavours():
    """epsbar = 0: M_h = diag(M(+mubar), M(-mubar)), the pinned one-flavour operator."""
    lat = Lattice.cubic(4, 2)
    U = inputs.random_gauge(4, 2, 0.5, seed=111)
    kappa, mubar = 0.15, 0.07
    psi = _doublet(lat, 112)
    out = oracle.apply_Mh(lat, U, psi, kappa, mubar, 0.0)
    assert rel(out[0], oracle.apply_M(lat, U, psi[0], kappa, mubar, 1)) < 1e-15
    assert rel(out[1], oracle.apply_M(lat, U, psi[1], kappa, mubar, -1)) < 1e-15


def test_doublet_free_field_spectrum():
    """Unit gauge: per momentum, M_h^dag M_h = c0 + 2 eb (w0 tau1 + mb gamma5 tau2) with
    c0 = w0^2 + sum s^2 + mb^2 + eb^2, so its eigenvalues are c0 +- 2 eb sqrt(w0^2 + mb^2),
    twelve of each, w0 = 1 - 2 kappa sum cos p, s = 2 kappa sin p (antiperiodic p_t)."""
    T, L = 4, 2
    lat = Lattice.cubic(T, L)
    U = inputs.unit_gauge(T, L)
    kappa, mubar, epsbar = 0.13, 0.4, 0.3
    mb, eb = 2 * kappa * mubar, 2 * kappa * epsbar
    M = dense_doublet(lambda v: oracle.apply_Mh(lat, U, v, kappa, mubar, epsbar), lat)
    lam = np.sort(np.linalg.eigvalsh(M.conj().T @ M))
    expect = []
    for p in free_field_momenta(lat):
        w0 = 1 - 2 * kappa * np.cos(p).sum()
        c0 = w0 ** 2 + (2 * kappa * np.sin(p)) @ (2 * kappa * np.sin(p)) + mb ** 2 + eb ** 2
        d = 2 * eb * np.sqrt(w0 ** 2 + mb ** 2)
        expect += [c0 + d] * 12 + [c0 - d] * 12
    assert np.allclose(lam, np.sort(expect), rtol=0, atol=1e-12)


def test_doublet_adjoint_relation():
    """<chi, M_h psi> = <M_h^dag chi, psi> with M_h^dag = tau1 gamma5 M_h gamma5 tau1."""
    lat = Lattice.cubic(4, 4)
    U = inputs.random_gauge(4, 4, 0.7, seed=113)
    kappa, mubar, epsbar = 0.16, 0.02, 0.03
    psi, chi = _doublet(lat, 114), _doublet(lat, 116)
    lhs = np.vdot(chi, oracle.apply_Mh(lat, U, psi, kappa, mubar, epsbar))
    rhs = np.vdot(oracle.apply_Mh_dag(lat, U, chi, kappa, mubar, epsbar), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("T,L", [(2, 2), (4, 2)])
def test_doublet_solve_equals_dense_solve(T, L):
    lat = Lattice.cubic(T, L)
    U = inputs.random_gauge(T, L, 0.5, seed=117)
    kappa, mubar, epsbar = 0.16, 0.05, 0.07
    phi = _doublet(lat, 118)
    M = dense_doublet(lambda v: oracle.apply_Mh(lat, U, v, kappa, mubar, epsbar), lat)
    psi = np.linalg.solve(M, phi.reshape(-1))
    res = oracle.solve_Mh(lat, U, phi, kappa, mubar, epsbar, tol=1e-12)
    assert res.converged and rel(res.x.reshape(-1), psi) < 1e-10


# ------------------------------------------------------ MR on Mhat (Sec. 4.4) ---
def test_mr_is_exact_in_one_step_for_the_identity():
    """kappa = 0, mu = 0: Mhat = 1, so the first MR step (alpha = <b, b>/<b, b> = 1) is exact."""
    lat = Lattice.cubic(4, 2)
    U = inputs.random_gauge(4, 2, 0.5, seed=121)
    b = _odd(lat, 122)
    res = oracle.mr(lat, U, b, 0.0, 0.0, tol=1e-14, max_iter=1)
    assert res.iters == 1 and rel(res.x, b) < 1e-15 and res.converged


def test_mr_residual_never_grows_and_solves_the_dense_system():
    """Each MR step minimises ||r - alpha q|| over alpha, so the residual norm cannot grow; with
    the spectrum of Mhat in Re > 0 (kappa 0.13) the iteration converges to the dense solution."""
    lat = Lattice.cubic(4, 2)
    U = inputs.random_gauge(4, 2, 0.5, seed=123)
    kappa, mu = 0.13, 0.05
    b = _odd(lat, 124)
    last = np.inf
    for k in range(1, 12):
        res = oracle.mr(lat, U, b, kappa, mu, tol=1e-30, max_iter=k)
        assert res.iters == k and res.relres <= last * (1 + 1e-12)
        last = res.relres
    assert last < 0.9
    o = component_mask(lat, 1)
    Mh = dense_from(lambda v: oracle.schur(lat, U, v, kappa, mu), lat, rows_mask=o, cols_mask=o)
    res = oracle.mr(lat, U, b, kappa, mu, tol=1e-12, max_iter=5000)
    assert res.converged and rel(res.x.reshape(-1)[o], np.linalg.solve(Mh, b.reshape(-1)[o])) < 1e-10


def test_mr_solve_equals_dense_solve():
    lat = Lattice.cubic(2, 2)
    U = inputs.random_gauge(2, 2, 0.5, seed=125)
    kappa, mu = 0.12, 0.05
    phi = rand_spinor(lat, 126)
    for f in (1, -1):
        M = dense_from(lambda v: oracle.apply_M(lat, U, v, kappa, mu, f), lat)
        res = oracle.solve_mr(lat, U, phi, kappa, mu, f, tol=1e-12, max_iter=5000)
        assert res.converged and rel(res.psi.reshape(-1), np.linalg.solve(M, phi.reshape(-1))) < 1e-10
