"""GPU non-degenerate doublet (eq. Dh): operator and even/odd CG solve against the CPU oracle.

The operator is compared element by element with the oracle's M_h; every solve meets the bar
||phi - M_h x|| / ||phi|| < 1e-10 with the ORACLE's M_h applied to the GPU solution, and on 4^4
the solution matches the oracle's own solve (CG on the normal equations of the full operator).
"""
import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import (CG_FP64, CG_RELIABLE, CG_SQRT_EPS, LINK8, LINK12, LINK18, Lattice,
                                   TMError, inputs)

from _util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (mubar, epsbar): mubar > epsbar, the 2+1+1 heavy-doublet regime epsbar > mubar, and light masses
PARAMS = [(0.1, 0.05), (0.15, 0.19), (0.02, 0.01)]


def dev():
    return torch.device("cuda:0")


def setup(name):
    w = inputs.WORKLOADS[name]
    U = w.gauge()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev()))
    return w, U, lat


def doublet_source(w, seed=0):
    return np.stack([w.source(seed), w.source(seed + 1)])


def oracle_residual(w, U, phi, x, mubar, epsbar):
    olat = oracle.Lattice.cubic(w.T, w.L)
    r = phi - oracle.apply_Mh(olat, U, x, w.kappa, mubar, epsbar)
    return np.linalg.norm(r) / np.linalg.norm(phi)


@pytest.mark.parametrize("name", ["4^4", "8^4", "12^3x24"])
@pytest.mark.parametrize("mubar,epsbar", PARAMS)
def test_apply_Dh_matches_oracle(name, mubar, epsbar):
    w, U, lat = setup(name)
    psi = doublet_source(w, 3)
    out = torch.empty((2,) + psi.shape[1:], dtype=torch.complex128, device=dev())
    lat.apply_Dh(out, torch.from_numpy(psi).to(dev()), mubar, epsbar)
    ref = oracle.apply_Mh(oracle.Lattice.cubic(w.T, w.L), U, psi, w.kappa, mubar, epsbar)
    got = out.cpu().numpy()
    assert rel(got, ref) < 1e-13
    # host buffers give the identical result
    outh = np.zeros_like(psi)
    lat.apply_Dh(outh, psi, mubar, epsbar)
    assert np.array_equal(outh, got)
    lat.close()


def test_apply_Dh_two_rhs_and_reduction_to_one_flavour():
    """nrhs = 2 equals two single calls; at epsbar = 0 the doublet is (M(+mubar), M(-mubar)) of
    the one-flavour operator."""
    w, U, lat = setup("4^4")
    psi = np.stack([doublet_source(w, 5), doublet_source(w, 7)])
    b = torch.from_numpy(psi).to(dev())
    out = torch.empty_like(b)
    lat.apply_Dh(out, b, 0.08, 0.03, nrhs=2)
    one = torch.empty_like(b[0])
    for k in range(2):
        lat.apply_Dh(one, b[k].contiguous(), 0.08, 0.03)
        assert torch.equal(one, out[k])
    lat.apply_Dh(one, b[0].contiguous(), 0.08, 0.0)
    lat.set_params(w.kappa, 0.08)
    up = torch.empty_like(b[0, 0])
    lat.apply_D(up, b[0, 0].contiguous(), flavour=1)
    dn = torch.empty_like(b[0, 1])
    lat.apply_D(dn, b[0, 1].contiguous(), flavour=-1)
    assert rel(one[0].cpu().numpy(), up.cpu().numpy()) < 1e-14
    assert rel(one[1].cpu().numpy(), dn.cpu().numpy()) < 1e-14
    lat.close()


MODES = [
    ("fp64", dict(mode=CG_FP64)),
    ("reliable_f32_18", dict(mode=CG_RELIABLE, sloppy_link=LINK18)),
    ("reliable_f32_12", dict(mode=CG_RELIABLE, sloppy_link=LINK12)),
    ("reliable_f32_8", dict(mode=CG_RELIABLE, sloppy_link=LINK8)),
]


@pytest.mark.parametrize("mode,kw", MODES)
@pytest.mark.parametrize("mubar,epsbar", PARAMS)
def test_solve_doublet_4x4x4x4(mode, kw, mubar, epsbar):
    w, U, lat = setup("4^4")
    phi = doublet_source(w)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_doublet(x, b, mubar, epsbar, tol=1e-10, **kw)
    assert oracle_residual(w, U, phi, x.cpu().numpy(), mubar, epsbar) < 1e-10
    assert info.true_rel_residual < 1e-10 and info.schur_rel_residual < 1e-10 and info.iters > 0
    lat.solve_doublet(x, b, mubar, epsbar, tol=1e-12, **kw)
    ref = oracle.solve_Mh(oracle.Lattice.cubic(w.T, w.L), U, phi, w.kappa, mubar, epsbar, tol=1e-12)
    assert ref.converged and rel(x.cpu().numpy(), ref.x) < 1e-9
    lat.close()


@pytest.mark.parametrize("mode,kw", [MODES[0], MODES[2]])
@pytest.mark.parametrize("name", ["8^4", "12^3x24", "16^3x32"])
def test_solve_doublet_larger_lattices(mode, kw, name):
    w, U, lat = setup(name)
    phi = doublet_source(w)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_doublet(x, b, 0.15, 0.19, tol=1e-10, **kw)
    res = oracle_residual(w, U, phi, x.cpu().numpy(), 0.15, 0.19)
    assert res < 1e-10 and info.true_rel_residual < 1e-10
    assert abs(res - info.true_rel_residual) < 1e-3 * res
    lat.close()


def test_solve_doublet_host_buffers_determinism_and_errors():
    w, U, lat = setup("4^4")
    phi = doublet_source(w)
    xh = np.zeros_like(phi)
    i1 = lat.solve_doublet(xh, phi, 0.1, 0.05, mode=CG_RELIABLE)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    i2 = lat.solve_doublet(x, b, 0.1, 0.05, mode=CG_RELIABLE)
    assert np.array_equal(x.cpu().numpy(), xh) and i1.iters == i2.iters
    z = torch.zeros_like(b)
    x.fill_(1.0)
    assert lat.solve_doublet(x, z, 0.1, 0.05).iters == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(TMError):  # singular site term: (2 kappa epsbar)^2 > 1 + (2 kappa mubar)^2
        lat.solve_doublet(x, b, 0.0, 4.0)
    with pytest.raises(TMError):
        lat.apply_Dh(x, b, 0.0, 4.0)
    with pytest.raises(TMError):
        lat.solve_doublet(x, b, 0.1, 0.05, mode=CG_SQRT_EPS)
    with pytest.raises(TMError):
        lat.solve_doublet(b, b, 0.1, 0.05)
    lat.close()
