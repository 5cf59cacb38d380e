"""GPU solve of the normal equations and the chronological guess against the CPU oracle.

tm_solve_normal solves Qhat^f Qhat^-f X = phi on the odd sites (eq. eo6); the bar is the
ORACLE's operator applied to the GPU solution: ||phi - A X|| / ||phi|| < 1e-10.
tm_chrono_guess (Sec. 4.2, eq. chrono) is compared with the oracle's Galerkin combination
element by element.
"""
import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import (CG_FP64, CG_RELIABLE, CG_SQRT_EPS, F16, F32, F64, LINK8, LINK12,
                                   LINK18, Lattice, TMError, inputs)

from _util import from_half, rel, to_half

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [
    ("fp64", dict(mode=CG_FP64)),
    ("sqrt_eps_f32_12", dict(mode=CG_SQRT_EPS, sloppy_prec=F32, sloppy_link=LINK12)),
    ("reliable_f32_18", dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK18)),
    ("reliable_f16_12", dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK12)),
    ("reliable_f16_8", dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK8)),
]


def dev():
    return torch.device("cuda:0")


class Setup:
    def __init__(self, name, mu=None):
        w = inputs.WORKLOADS[name]
        self.w = w
        self.mu = w.mu if mu is None else mu
        self.U = w.gauge()
        self.olat = oracle.Lattice.cubic(w.T, w.L)
        self.lat = Lattice(w.T, w.L, w.kappa, self.mu)
        self.lat.set_gauge(torch.from_numpy(self.U).to(dev()))
        self.hbytes = self.lat.half_field_bytes(F64)

    def odd_full(self, seed):
        """A Gaussian odd-site vector as a canonical full field (zero on even sites)."""
        psi = inputs.gaussian_spinor(self.w.T, self.w.L, seed)
        return from_half(to_half(psi, 1), 1, self.w.T, self.w.L)

    def to_dev(self, full):
        h = torch.from_numpy(np.ascontiguousarray(to_half(full, 1)).view(np.float64).reshape(-1)).to(dev())
        out = torch.empty(self.hbytes // 8, dtype=torch.float64, device=dev())
        self.lat.pack_half(F64, out, h)
        return out

    def to_host(self, d):
        h = torch.empty(self.hbytes // 8, dtype=torch.float64, device=dev())
        self.lat.unpack_half(F64, h, d)
        torch.cuda.synchronize()
        half = h.cpu().numpy().view(np.complex128).reshape(-1, 4, 3)
        return from_half(half, 1, self.w.T, self.w.L)

    def A(self, full, f=1):
        return oracle.normal_op(self.olat, self.U, full, self.w.kappa, self.mu, f)

    def resid(self, X, phi, f=1):
        return np.linalg.norm(phi - self.A(X, f)) / np.linalg.norm(phi)


@pytest.mark.parametrize("name,kw", MODES)
@pytest.mark.parametrize("flavour", [1, -1])
def test_solve_normal_8x8x8x8(name, kw, flavour):
    S = Setup("8^4")
    phi = S.odd_full(11)
    X = torch.zeros(S.hbytes // 8, dtype=torch.float64, device=dev())
    info = S.lat.solve_normal(X, S.to_dev(phi), tol=1e-10, flavour=flavour, **kw)
    Xh = S.to_host(X)
    assert S.resid(Xh, phi, flavour) < 1e-10
    assert info.schur_rel_residual < 1e-10 and info.iters > 0
    # agreement with the oracle's own CG, both at 1e-12
    S.lat.solve_normal(X, S.to_dev(phi), tol=1e-12, flavour=flavour, **kw)
    ref = oracle.cg(S.olat, S.U, phi, S.w.kappa, S.mu, flavour, tol=1e-12)
    assert ref.converged and rel(S.to_host(X), ref.x) < 1e-9
    S.lat.close()


def test_solve_normal_12x12x12x24_ragged_blocks():
    """h = 20736 odd sites: not a multiple of the 256-thread blocks."""
    S = Setup("12^3x24")
    phi = S.odd_full(12)
    X = torch.zeros(S.hbytes // 8, dtype=torch.float64, device=dev())
    S.lat.solve_normal(X, S.to_dev(phi), tol=1e-10, mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK12)
    assert S.resid(S.to_host(X), phi) < 1e-10
    S.lat.close()


def test_solve_normal_initial_guess():
    S = Setup("8^4")
    phi = S.odd_full(13)
    pd = S.to_dev(phi)
    X = torch.zeros(S.hbytes // 8, dtype=torch.float64, device=dev())
    cold = S.lat.solve_normal(X, pd, tol=1e-10)
    # restarting from the converged solution needs no iteration
    again = S.lat.solve_normal(X, pd, tol=1e-10, use_x0=True)
    assert again.iters == 0 and S.resid(S.to_host(X), phi) < 1e-10
    # a guess near the solution: fewer iterations, same bar
    Xs = S.to_host(X)
    X.copy_(S.to_dev(Xs + 1e-6 * S.odd_full(14)))
    warm = S.lat.solve_normal(X, pd, tol=1e-10, use_x0=True, mode=CG_RELIABLE, sloppy_prec=F32,
                              sloppy_link=LINK12)
    assert S.resid(S.to_host(X), phi) < 1e-10
    assert warm.iters < cold.iters
    S.lat.close()


def test_solve_normal_zero_source_and_arguments():
    S = Setup("4^4")
    X = torch.ones(S.hbytes // 8, dtype=torch.float64, device=dev())
    phi = torch.zeros_like(X)
    info = S.lat.solve_normal(X, phi)
    assert info.iters == 0 and float(X.abs().max()) == 0.0
    with pytest.raises(TMError):
        S.lat.solve_normal(X, X)
    with pytest.raises(TMError):
        S.lat.solve_normal(X, phi.cpu().numpy())
    S.lat.close()


@pytest.mark.parametrize("n", [1, 4, 7])
@pytest.mark.parametrize("flavour", [1, -1])
def test_chrono_guess_matches_oracle(n, flavour):
    S = Setup("8^4")
    phi = S.odd_full(21)
    chis = [S.odd_full(30 + i) for i in range(n)]
    X0 = torch.empty(S.hbytes // 8, dtype=torch.float64, device=dev())
    S.lat.chrono_guess(X0, [S.to_dev(c) for c in chis], S.to_dev(phi), flavour=flavour)
    ref, _ = oracle.chrono_guess(S.olat, S.U, chis, phi, S.w.kappa, S.mu, flavour)
    assert rel(S.to_host(X0), ref) < 1e-11
    S.lat.close()


def test_chrono_guess_exact_on_span_and_degenerate_history():
    """phi = A X* with X* in the span of the history: the guess is X*; a history holding the
    same vector twice (a singular Galerkin matrix) still gives X*; n = 0 gives zero."""
    S = Setup("4^4")
    chis = [S.odd_full(40 + i) for i in range(3)]
    Xs = 0.3 * chis[0] - (1.2 + 0.5j) * chis[1] + 2j * chis[2]
    phi = S.A(Xs)
    dchis = [S.to_dev(c) for c in chis]
    X0 = torch.empty(S.hbytes // 8, dtype=torch.float64, device=dev())
    S.lat.chrono_guess(X0, dchis, S.to_dev(phi))
    assert rel(S.to_host(X0), Xs) < 1e-11
    S.lat.chrono_guess(X0, dchis + [dchis[1].clone()], S.to_dev(phi))
    assert rel(S.to_host(X0), Xs) < 1e-10
    S.lat.chrono_guess(X0, [], S.to_dev(phi))
    assert float(X0.abs().max()) == 0.0
    with pytest.raises(TMError):
        S.lat.chrono_guess(X0, [X0], S.to_dev(phi))
    S.lat.close()


def test_chrono_guess_cuts_iterations_along_a_trajectory():
    """Slowly varying sources, as along a molecular-dynamics trajectory: each solve starts from
    the guess built from the previous N_CSG = 4 solutions and needs fewer iterations than a
    cold start; every solution still meets the oracle-checked bar."""
    S = Setup("8^4")
    base, drift = S.odd_full(51), S.odd_full(52)
    history = []
    cold_total = warm_total = 0
    X = torch.zeros(S.hbytes // 8, dtype=torch.float64, device=dev())
    for k in range(8):
        phi = base + 0.02 * k * drift + 0.0005 * k * k * S.odd_full(53)
        pd = S.to_dev(phi)
        X.zero_()
        cold_total += S.lat.solve_normal(X, pd, tol=1e-10).iters
        S.lat.chrono_guess(X, history[-4:], pd)
        info = S.lat.solve_normal(X, pd, tol=1e-10, use_x0=True)
        warm_total += info.iters
        assert S.resid(S.to_host(X), phi) < 1e-10
        history.append(X.clone())
    assert warm_total < 0.8 * cold_total, (warm_total, cold_total)
    S.lat.close()
